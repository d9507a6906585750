"""The allocation-free ingestion entry point gives the same sketches as
gz_edge_update.

Callers that cannot let a library allocate device memory (a host framework
whose caching allocator owns the device memory and accounts for every byte, a
latency-bound loop that may not call cudaMalloc, which can synchronise the
device) use gz_sketch_update_noalloc, which works in a fixed static scratch
array.  This test drives it through the C ABI on a handle's own sketch memory,
two calls in a row, and compares the exported sketches bit for bit with a
second handle fed the same batches through gz_edge_update (the tests of this
repository use exact equality for sketches).  It sits in a file of its own
that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import paper_2203_14927_b300 as gz
from paper_2203_14927_b300 import streams as S

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def _noalloc(ptr, V, seed, du, dv, status, stream):
    return gz.lib().gz_sketch_update_noalloc(
        ctypes.c_void_p(ptr), V, seed, ctypes.c_void_p(du.data_ptr()), ctypes.c_void_p(dv.data_ptr()),
        du.numel(), ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(stream))


@pytest.mark.parametrize("V", [5000, 70000])  # 32-bit and 64-bit edge indices
def test_noalloc_matches_edge_update_two_calls_in_a_row(V):
    import torch

    seed = 7
    u, v = S.random_stream(V, 400000, seed=V, n_distinct=150000)
    batches = [(u[:250000], v[:250000]), (u[250000:], v[250000:])]
    ref = gz.Graph(V, seed)
    tgt = gz.Graph(V, seed)  # supplies zeroed sketch memory and the export
    ptr = tgt.info()["sketch_ptr"]
    stream = torch.cuda.current_stream().cuda_stream
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    for bu, bv in batches:
        ref.edge_update(_dev(bu), _dev(bv))
        ref.sync()
        du, dv = _dev(bu), _dev(bv)
        assert _noalloc(ptr, V, seed, du, dv, status, stream) == gz.GZ_OK
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        a_ref, g_ref = ref.export_sketch()
        a_got, g_got = tgt.export_sketch()
        assert np.array_equal(a_got, a_ref) and np.array_equal(g_got, g_ref)
    ref.close()
    tgt.close()


def test_noalloc_rejects_bad_batches_and_sizes():
    import torch

    V, seed = 300, 3
    g = gz.Graph(V, seed)
    ptr = g.info()["sketch_ptr"]
    stream = torch.cuda.current_stream().cuda_stream
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    u, v = S.random_stream(V, 1000, seed=1)
    assert _noalloc(ptr, V, seed, _dev(u), _dev(v), status, stream) == gz.GZ_OK
    torch.cuda.synchronize()
    before = g.export_sketch()
    # a self loop discards the whole batch; status says so
    bu, bv = np.array([1, 2, 3], np.uint32), np.array([4, 2, 5], np.uint32)
    assert _noalloc(ptr, V, seed, _dev(bu), _dev(bv), status, stream) == gz.GZ_OK
    torch.cuda.synchronize()
    assert int(status.item()) == 1
    after = g.export_sketch()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    # sizes beyond the stated maxima are refused before anything is queued
    big = torch.zeros(1, dtype=torch.int32, device="cuda")
    lib = gz.lib()
    too_many = (1 << 20) + 1
    assert lib.gz_sketch_update_noalloc(ctypes.c_void_p(ptr), V, seed, ctypes.c_void_p(big.data_ptr()),
                                        ctypes.c_void_p(big.data_ptr()), too_many, None,
                                        ctypes.c_void_p(stream)) == gz.GZ_EINVAL
    assert lib.gz_sketch_update_noalloc(ctypes.c_void_p(ptr), (1 << 17) + 1, seed,
                                        ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(big.data_ptr()),
                                        1, None, ctypes.c_void_p(stream)) == gz.GZ_EINVAL
    g.close()
