"""maiter_sssp_noalloc: the SSSP entry point for callers that may not allocate
device memory (for example code handed buffers by a host framework's caching
allocator, or code that may run during a stream capture, where cudaMalloc is
not allowed).  Its working memory is a fixed array inside the library.

The test calls it through the C ABI with caller-owned device buffers and
checks its distances against the allocating entry point, maiter_run, on two
calls in a row (the second call must not see the first call's leftovers).
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import graphgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_N = 1 << 20


@pytest.fixture(scope="module")
def mt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_05785_b300 as m
    L = m.lib()
    P, i64 = ctypes.c_void_p, ctypes.c_int64
    L.maiter_sssp_noalloc.argtypes = [i64, i64, P, P, P, i64, P, P, i64, ctypes.c_int, P,
                                      ctypes.POINTER(ctypes.c_int64)]
    L.maiter_sssp_noalloc.restype = ctypes.c_int32
    return m


def noalloc(mt, n, m, rp, col, w, source, v, delta, stream=None):
    rounds = ctypes.c_int64(-1)
    st = mt.lib().maiter_sssp_noalloc(n, m, rp.data_ptr(), col.data_ptr(), w.data_ptr(), source,
                                      v.data_ptr(), delta.data_ptr(), 0, 0, stream,
                                      ctypes.byref(rounds))
    return st, rounds.value


@pytest.mark.parametrize("scale,ef", [(12, 8), (20, 16)])
def test_noalloc_matches_maiter_run_on_two_calls(mt, scale, ef):
    g = graphgen.rmat(scale, ef, weights=True)
    dev = torch.device("cuda", 0)
    rp = torch.from_numpy(g.row_ptr.astype(np.int32)).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    w = torch.from_numpy(g.w.view(np.int32)).to(dev)
    v = torch.empty(g.n, dtype=torch.int32, device=dev)
    delta = torch.empty(g.n, dtype=torch.int32, device=dev)
    G = mt.Graph.from_csr(g)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for s in graphgen.sssp_sources(g, 2):
        st, rounds = noalloc(mt, g.n, g.m, rp, col, w, int(s), v, delta, stream)
        assert st == mt.OK, mt.last_error()
        expect = mt.run(G, mt.OP_MIN_U32, source=int(s))
        got = v.cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(got, expect.state())
        assert rounds > 0


def test_noalloc_rejects_sizes_beyond_its_fixed_memory(mt):
    dev = torch.device("cuda", 0)
    small = torch.zeros(4, dtype=torch.int32, device=dev)
    st, _ = noalloc(mt, MAX_N + 1, 0, small, small, small, 0, small, small)
    assert st == mt.ERR_INVALID_ARG
    assert "1048576" in mt.last_error()
