"""Argument checks of the C ABI that return before any device work, run on
the CPU: every entry point rejects NULL handles, out-of-range sizes and
missing buffers with MAITER_ERR_INVALID_ARG and a message (thread-local,
maiter_last_error), and the destroy calls accept NULL."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def mt():
    import paper_1710_05785_b300 as m
    import paper_1710_05785_b300.build as b
    b.build()
    m.lib()
    return m


def rejected(mt, status, needle):
    assert status == mt.ERR_INVALID_ARG
    assert needle in mt.last_error()


def test_graph_create_checks_sizes_and_buffers(mt):
    L = mt.lib()
    rp = np.zeros(5, dtype=np.int64)
    col = np.zeros(4, dtype=np.int32)
    out = ctypes.c_void_p()
    P = lambda a: a.ctypes.data  # noqa: E731
    rejected(mt, L.maiter_graph_create(4, 0, P(rp), None, None, 0, None), "out is NULL")
    rejected(mt, L.maiter_graph_create(-1, 0, P(rp), None, None, 0, ctypes.byref(out)),
             "out of range")
    rejected(mt, L.maiter_graph_create(4, -3, P(rp), P(col), None, 0, ctypes.byref(out)),
             "out of range")
    rejected(mt, L.maiter_graph_create(4, 1 << 31, P(rp), P(col), None, 0, ctypes.byref(out)),
             "out of range")
    rejected(mt, L.maiter_graph_create(4, 0, None, None, None, 0, ctypes.byref(out)),
             "row_ptr is NULL")
    rejected(mt, L.maiter_graph_create(4, 4, P(rp), None, None, 0, ctypes.byref(out)),
             "col is NULL")
    assert not out.value


def test_run_update_and_readers_reject_null_handles(mt):
    L = mt.lib()
    p = mt.params_default()
    out = ctypes.c_void_p()
    rejected(mt, L.maiter_run(None, ctypes.byref(p), ctypes.byref(out)), "NULL argument")
    rejected(mt, L.maiter_graph_update(None, None, None, None, None), "NULL argument")
    buf = np.zeros(4, dtype=np.float64)
    rejected(mt, L.maiter_get_state(None, buf.ctypes.data, 4), "NULL result")
    rejected(mt, L.maiter_get_delta(None, buf.ctypes.data, 4), "NULL result")
    rejected(mt, L.maiter_get_stats(None, None), "NULL argument")


def test_batch_rejects_missing_arrays_and_empty_sets(mt):
    L = mt.lib()
    bp = mt.BatchParams()
    L.maiter_batch_params_default(ctypes.byref(bp))
    out = ctypes.c_void_p()
    rejected(mt, L.maiter_run_batch(None, 1, None, 1, ctypes.byref(bp), ctypes.byref(out)),
             "NULL argument")
    graphs = (ctypes.c_void_p * 1)(None)
    queries = (mt.QuerySpec * 1)()
    rejected(mt, L.maiter_run_batch(graphs, 0, queries, 1, ctypes.byref(bp), ctypes.byref(out)),
             "at least one graph")
    rejected(mt, L.maiter_run_batch(graphs, 1, queries, 1, ctypes.byref(bp), ctypes.byref(out)),
             "graph 0 is NULL")


def test_noalloc_rejects_sizes_beyond_its_fixed_memory(mt):
    L = mt.lib()
    f = L.maiter_sssp_noalloc
    P, i64 = ctypes.c_void_p, ctypes.c_int64
    f.argtypes = [i64, i64, P, P, P, i64, P, P, i64, ctypes.c_int, P, ctypes.POINTER(i64)]
    f.restype = ctypes.c_int32
    buf = np.zeros(8, dtype=np.uint32).ctypes.data
    rejected(mt, f(0, 0, buf, None, None, 0, buf, buf, 0, 0, None, None), "fixed working")
    rejected(mt, f((1 << 20) + 1, 0, buf, None, None, 0, buf, buf, 0, 0, None, None),
             "fixed working")
    rejected(mt, f(4, 0, buf, None, None, 4, buf, buf, 0, 0, None, None), "source")
    rejected(mt, f(4, 2, buf, None, None, 0, buf, buf, 0, 0, None, None), "NULL buffer")


def test_destroy_calls_accept_null(mt):
    L = mt.lib()
    for fn in (L.maiter_graph_destroy, L.maiter_result_destroy, L.maiter_batch_destroy,
               L.maiter_mlp_destroy):
        fn(None)


def test_errors_are_per_thread(mt):
    import threading
    L = mt.lib()
    seen = {}

    def other():
        seen["before"] = mt.last_error()
        L.maiter_get_stats(None, None)
        seen["after"] = mt.last_error()

    L.maiter_graph_create(-1, 0, None, None, None, 0, None)
    mine = mt.last_error()
    t = threading.Thread(target=other)
    t.start()
    t.join()
    assert seen["before"] == "" and "NULL argument" in seen["after"]
    assert mt.last_error() == mine          # untouched by the other thread
