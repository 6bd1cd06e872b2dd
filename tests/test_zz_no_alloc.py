"""maiter_sssp_noalloc: the SSSP entry point for callers that may not allocate
device memory (for example code whose device memory belongs to a host
framework's caching allocator, or a caller with a fixed memory budget).  Its
working memory is a fixed array inside the library.

The tests call it through the C ABI with caller-owned device buffers and check
its distances against the allocating entry point, maiter_run, and against the
oracle's Dijkstra, on two calls in a row (the second call must not see the
first call's leftovers); then its argument checks, its round cap, and a call
made while another stream is capturing.  This file is collected last on
purpose.
"""
import ctypes

import numpy as np
import pytest

import graphgen
import oracle

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


def noalloc(mt, n, m, rp, col, w, source, v, delta, stream=None, max_rounds=0, device=0,
            want_rounds=True):
    rounds = ctypes.c_int64(-1)
    st = mt.lib().maiter_sssp_noalloc(n, m, rp.data_ptr(), col.data_ptr(), w.data_ptr(), source,
                                      v.data_ptr(), delta.data_ptr(), max_rounds, device, stream,
                                      ctypes.byref(rounds) if want_rounds else None)
    return st, rounds.value


def device_csr(g, dev):
    rp = torch.from_numpy(g.row_ptr.astype(np.int32)).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    w = torch.from_numpy(g.w.view(np.int32)).to(dev)
    v = torch.empty(g.n, dtype=torch.int32, device=dev)
    delta = torch.empty(g.n, dtype=torch.int32, device=dev)
    return rp, col, w, v, delta


@pytest.mark.parametrize("scale,ef", [(12, 8), (20, 16)])
def test_noalloc_matches_maiter_run_and_dijkstra_on_two_calls(mt, scale, ef):
    g = graphgen.rmat(scale, ef, weights=True)
    dev = torch.device("cuda", 0)
    rp, col, w, v, delta = device_csr(g, dev)
    G = mt.Graph.from_csr(g)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for s in graphgen.sssp_sources(g, 2):
        st, rounds = noalloc(mt, g.n, g.m, rp, col, w, int(s), v, delta, stream)
        assert st == mt.OK, mt.last_error()
        got = v.cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(got, mt.run(G, mt.OP_MIN_U32, source=int(s)).state())
        np.testing.assert_array_equal(got, oracle.dijkstra(g, int(s)))
        assert rounds > 0


def test_noalloc_rejects_sizes_beyond_its_fixed_memory(mt):
    dev = torch.device("cuda", 0)
    small = torch.zeros(4, dtype=torch.int32, device=dev)
    st, _ = noalloc(mt, MAX_N + 1, 0, small, small, small, 0, small, small)
    assert st == mt.ERR_INVALID_ARG
    assert "1048576" in mt.last_error()


def test_noalloc_null_stream_and_null_rounds(mt):
    g = graphgen.rmat(6, 4, weights=True)
    dev = torch.device("cuda", 0)
    rp, col, w, v, delta = device_csr(g, dev)
    s = int(graphgen.sssp_sources(g, 1)[0])
    torch.cuda.synchronize()
    st, _ = noalloc(mt, g.n, g.m, rp, col, w, s, v, delta, stream=None, want_rounds=False)
    assert st == mt.OK, mt.last_error()
    np.testing.assert_array_equal(v.cpu().numpy().view(np.uint32), oracle.dijkstra(g, s))


def test_noalloc_device_side_csr_check(mt):
    g = graphgen.rmat(6, 4, weights=True)
    dev = torch.device("cuda", 0)
    rp, col, w, v, delta = device_csr(g, dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    bad_rp = rp.clone()
    i = int(np.argmax(np.diff(g.row_ptr)))          # a row with edges: make it decrease
    bad_rp[i + 1] = int(g.row_ptr[i]) - 1 if g.row_ptr[i] > 0 else 0
    bad_rp[i] = int(g.row_ptr[i + 1])
    st, _ = noalloc(mt, g.n, g.m, bad_rp, col, w, 0, v, delta, stream)
    assert st == mt.ERR_INVALID_ARG
    assert "row_ptr" in mt.last_error()
    bad_col = col.clone()
    bad_col[g.m // 2] = g.n                          # a target equal to n
    st, _ = noalloc(mt, g.n, g.m, rp, bad_col, w, 0, v, delta, stream)
    assert st == mt.ERR_INVALID_ARG
    assert "col" in mt.last_error()
    # a valid call afterwards still works (the flag word is cleared per call)
    s = int(graphgen.sssp_sources(g, 1)[0])
    st, _ = noalloc(mt, g.n, g.m, rp, col, w, s, v, delta, stream)
    assert st == mt.OK, mt.last_error()
    np.testing.assert_array_equal(v.cpu().numpy().view(np.uint32), oracle.dijkstra(g, s))


def test_noalloc_round_cap_leaves_a_readable_state(mt):
    g = graphgen.rmat(10, 8, weights=True)
    dev = torch.device("cuda", 0)
    rp, col, w, v, delta = device_csr(g, dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    s = int(graphgen.sssp_sources(g, 1)[0])
    st, rounds = noalloc(mt, g.n, g.m, rp, col, w, s, v, delta, stream, max_rounds=1)
    assert st == mt.ERR_NOT_CONVERGED
    assert rounds == 1
    # after one round the source is final and its out-neighbours hold their
    # one-edge distances as pending deltas; every state is an upper bound
    exact = oracle.dijkstra(g, s)
    vv = v.cpu().numpy().view(np.uint32)
    dd = delta.cpu().numpy().view(np.uint32)
    assert vv[s] == 0
    assert np.all(vv >= exact) and np.all(dd >= exact)
    nb = g.col[g.row_ptr[s]:g.row_ptr[s + 1]]
    assert np.all(np.minimum(vv[nb], dd[nb]) < 0xFFFFFFFF)


def test_noalloc_rejects_buffers_of_another_device(mt):
    g = graphgen.rmat(6, 4, weights=True)
    dev = torch.device("cuda", 0)
    rp, col, w, v, delta = device_csr(g, dev)
    # buffers live on device 0; naming device 1 is refused before any launch,
    # whether or not a device 1 exists
    st, _ = noalloc(mt, g.n, g.m, rp, col, w, 0, v, delta, device=1)
    assert st == mt.ERR_INVALID_ARG
    assert "device 0" in mt.last_error()
    host = torch.zeros(g.n + 1, dtype=torch.int32)
    st, _ = noalloc(mt, g.n, g.m, host, col, w, 0, v, delta)
    assert st == mt.ERR_INVALID_ARG
    assert "device pointers" in mt.last_error()


def test_noalloc_while_another_stream_captures(mt):
    g = graphgen.rmat(10, 8, weights=True)
    dev = torch.device("cuda", 0)
    rp, col, w, v, delta = device_csr(g, dev)
    s = int(graphgen.sssp_sources(g, 1)[0])
    side = torch.cuda.Stream(dev)                    # torch's pool streams are non-blocking
    cap = torch.cuda.Stream(dev)
    x = torch.zeros(4, device=dev)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cap, capture_error_mode="relaxed"):
        x.add_(1.0)
        # on the capturing stream: refused, and the capture stays intact
        st_cap, _ = noalloc(mt, g.n, g.m, rp, col, w, s, v, delta, stream=cap.cuda_stream)
        msg = mt.last_error()
        # on another (non-capturing) stream: runs to the exact distances
        st_side, _ = noalloc(mt, g.n, g.m, rp, col, w, s, v, delta, stream=side.cuda_stream)
    assert st_cap == mt.ERR_INVALID_ARG
    assert "capturing" in msg
    assert st_side == mt.OK
    side.synchronize()
    np.testing.assert_array_equal(v.cpu().numpy().view(np.uint32), oracle.dijkstra(g, s))
    graph.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0                        # only the replay added (capture is not run)
