"""The update kernel's bounded waits: failure detection without a GPU fault.

The batched kernel's producer warp and column warps hand record tiles to each
other through shared-memory barriers, and every wait on one is bounded.  These
tests set the bound to one poll with no suspension (gz_set_wait_limit), so the
waits run out almost at once: the kernel must stop on its own, leave the GPU
usable, and report GZ_ETIMEOUT (status 2 for the allocation-free call) once;
with the default bound restored, a reset handle gives the oracle's sketches
again.  Nothing here faults, traps or hangs the GPU: the kernel only stops
early.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2203_14927_b300 as gz
from paper_2203_14927_b300 import streams as S

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


@pytest.mark.parametrize("V", [5000, 70001])  # 32- and 64-bit edge indices
def test_bounded_wait_runs_out_reports_timeout_and_recovers(V):
    seed = 4
    u, v = S.random_stream(V, 200000, seed=V, n_distinct=80000)
    g = gz.Graph(V, seed, chunk_log2=16)
    g.set_wait_limit(1, 0)
    g.edge_update(_dev(u), _dev(v))
    with pytest.raises(gz.GzError) as err:
        g.sync()
    assert err.value.status == gz.GZ_ETIMEOUT
    g.sync()  # reported once
    g.set_wait_limit(0)
    g.reset()
    g.edge_update(_dev(u), _dev(v))
    g.sync()
    A, G = oracle.ingest(V, seed, u, v) if V <= 5000 else (None, None)
    if A is not None:
        a, gg = g.export_sketch()
        assert np.array_equal(a, A) and np.array_equal(gg, G)
    else:
        eu, ev = S.net_graph(V, u, v)
        for x in (0, 1, 77, V - 1):
            A1, G1 = oracle.sketch_node(V, seed, x, S.neighbors_from_edges(V, eu, ev, x))
            a, gg = g.export_sketch(x, x + 1)
            assert np.array_equal(a[0], A1) and np.array_equal(gg[0], G1), x
    g.close()


def test_allocation_free_call_reports_status_2_when_a_wait_runs_out():
    import torch

    V, seed = 3000, 6
    u, v = S.random_stream(V, 100000, seed=2, n_distinct=40000)
    g = gz.Graph(V, seed)  # supplies zeroed sketch memory
    ptr = g.info()["sketch_ptr"]
    stream = torch.cuda.current_stream().cuda_stream
    status = torch.full((1,), 9, dtype=torch.int32, device="cuda")
    du, dv = _dev(u), _dev(v)
    lib = gz.lib()

    def call():
        return lib.gz_sketch_update_noalloc(ctypes.c_void_p(ptr), V, seed, ctypes.c_void_p(du.data_ptr()),
                                            ctypes.c_void_p(dv.data_ptr()), du.numel(),
                                            ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(stream))

    assert lib.gz_set_wait_limit(None, 1, 0) == gz.GZ_OK
    try:
        assert call() == gz.GZ_OK
        torch.cuda.synchronize()
        assert int(status.item()) == 2
    finally:
        assert lib.gz_set_wait_limit(None, 0, 0) == gz.GZ_OK
    g.reset()
    assert call() == gz.GZ_OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    a, gg = g.export_sketch()
    A, G = oracle.ingest(V, seed, u, v)
    assert np.array_equal(a, A) and np.array_equal(gg, G)
    g.close()
