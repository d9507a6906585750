"""GPU path vs the CPU oracle, through the C ABI.

Sketches must match bit for bit (integer XOR arithmetic, no tolerance), the
component labels exactly, and the per-round Boruvka samples and the spanning
forest exactly (both are fixed once the sketches are: Fig. cube_code's scan
order picks the sample, and the forest is the sequential acceptance order).
"""
import numpy as np
import pytest

import oracle
import paper_2203_14927_b300 as gz
from paper_2203_14927_b300 import streams as S

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def _gpu_graph(V, seed, u, v, on_device=True, **cfg):
    g = gz.Graph(V, seed, **cfg)
    if on_device:
        g.edge_update(_dev(u), _dev(v))
    else:
        g.edge_update(u, v)
    g.sync()
    return g


def _assert_same_sketches(g, A, G, lo=0, hi=None):
    a, gg = g.export_sketch(lo, hi)
    hi = g.V if hi is None else hi
    assert np.array_equal(a, A[lo:hi]), "alpha differs"
    assert np.array_equal(gg, G[lo:hi]), "gamma differs"


def _assert_same_query(g, A, G, seed):
    want = oracle.boruvka(g.V, seed, A, G)
    g.enable_trace(True)
    forest, labels, st = g.list_spanning_forest()
    assert np.array_equal(labels, want["labels"])
    assert st["rounds"] == want["rounds"]
    assert st["fails_last"] == want["fails_last"]
    trace = g.query_trace()
    assert np.array_equal(trace, want["samples"])
    assert np.array_equal(forest, want["forest"])
    labels2, ncc, st2 = g.connected_components()
    assert np.array_equal(labels2, want["labels"]) and ncc == want["n_components"]
    # untraced CC queries run as one CUDA graph (device-side round loop)
    g.enable_trace(False)
    for _ in range(2):
        labels3, ncc3, st3 = g.connected_components()
        assert np.array_equal(labels3, want["labels"]) and ncc3 == want["n_components"]
        assert st3["rounds"] == want["rounds"] and st3["fails_last"] == want["fails_last"]
        assert st3["fails_total"] == st2["fails_total"] and st3["exhausted"] == st2["exhausted"]
    return want


@pytest.mark.parametrize("kernel", ["batched", "plain"])
def test_planted_small_config_bit_exact(kernel):
    # V = 2^10, 8 planted G(n_i, 0.1) components, 20% extra pairs cycled so
    # that the stream has ~2e5 updates
    spec = S.PlantedSpec(V=1024, seed=11, n_comp=8, p=0.1, extra=0.2, cycles=74)
    u, v, comp = S.planted_stream(spec)
    assert 1.5e5 < len(u) < 2.5e5
    A, G = oracle.ingest(spec.V, 5, u, v)
    g = _gpu_graph(spec.V, 5, u, v, kernel=kernel)
    _assert_same_sketches(g, A, G)
    want = _assert_same_query(g, A, G, 5)
    assert np.array_equal(want["labels"], oracle.brute_cc(spec.V, u, v))


@pytest.mark.parametrize("smem_mode", [1, 2])
@pytest.mark.parametrize("V", [2, 3, 77, 1000, 4097])
def test_ragged_sizes_many_chunks_and_tiles(V, smem_mode):
    # chunk of 2^10 updates (many chunks + a ragged tail), tiles of 64 records
    # (heavy nodes split across CTAs), 3 shared-memory rows (deep rows go to
    # global memory directly), short segments through the direct path
    n = 5000 if V > 3 else 301
    u, v = S.random_stream(V, n, seed=V, n_distinct=max(1, n // 3))
    A, G = oracle.ingest(V, 42, u, v)
    g = _gpu_graph(V, 42, u, v, chunk_log2=10, tile_records=64, smem_rows=3, small_segment=3,
                   smem_mode=smem_mode)
    _assert_same_sketches(g, A, G)
    _assert_same_query(g, A, G, 42)


def test_hub_node_split_across_many_tiles():
    V = 600
    rng = np.random.default_rng(3)
    other = rng.integers(1, V, 20000)
    u = np.zeros(20000, np.uint32)
    v = other.astype(np.uint32)
    A, G = oracle.ingest(V, 8, u, v)
    for tile in (32, 1000, 4096):
        g = _gpu_graph(V, 8, u, v, tile_records=tile)
        _assert_same_sketches(g, A, G)


def test_kronecker_full_query_parity():
    spec = S.KronSpec(L=11, seed=4, target_edges=0.45 * 2048 * 2047 / 2, churn=0.1,
                      n_iso=20, slice_log2=18)
    u, v = spec.stream()
    A, G = oracle.ingest(spec.V, 9, u, v)
    g = _gpu_graph(spec.V, 9, u, v)
    _assert_same_sketches(g, A, G)
    want = _assert_same_query(g, A, G, 9)
    eu, ev = spec.final_edges()
    assert np.array_equal(want["labels"], oracle.cc_edges(spec.V, eu, ev))


def test_host_and_device_inputs_agree():
    # host input goes through two staging buffers on a copy stream (15 chunks
    # of 2^12 updates here, so both buffers are reused several times), and a
    # second call must not overwrite a buffer the first call's kernels read
    V = 3000
    u, v = S.random_stream(V, 60000, seed=2)
    g1 = _gpu_graph(V, 1, u, v, on_device=True)
    g2 = gz.Graph(V, 1, chunk_log2=12)
    half = len(u) // 2
    g2.edge_update(u[:half], v[:half])
    g2.edge_update(u[half:], v[half:])
    g2.sync()
    a1, b1 = g1.export_sketch()
    a2, b2 = g2.export_sketch()
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)


def test_graph_replay_and_direct_launches_agree():
    # 40 chunks of 2^11 updates: the handle replays its captured CUDA graph
    # from the 9th chunk on; with no_graph it launches every kernel itself
    V = 5000
    u, v = S.random_stream(V, 40 * 2048 - 77, seed=12)
    A, G = oracle.ingest(V, 6, u, v)
    g1 = _gpu_graph(V, 6, u, v, chunk_log2=11)
    g2 = _gpu_graph(V, 6, u, v, chunk_log2=11, no_graph=1)
    _assert_same_sketches(g1, A, G)
    _assert_same_sketches(g2, A, G)
    g1.profile_enable(True)  # the graph's event nodes are re-pointed when profiling
    g1.edge_update(_dev(u[:9000]), _dev(v[:9000]))
    p = g1.profile_read()
    assert p["batches"] == 5 and p["update_ms"] > 0


@pytest.mark.parametrize("smem_mode", [1, 2])
def test_smem_modes_bit_exact_kronecker(smem_mode):
    spec = S.KronSpec(L=12, seed=8, target_edges=0.4 * 4096 * 4095 / 2, churn=0.1, n_iso=30,
                      slice_log2=20)
    u, v = spec.stream()
    g = _gpu_graph(spec.V, 3, u, v, smem_mode=smem_mode, chunk_log2=20)
    rng = np.random.default_rng(smem_mode)
    for x in sorted(set(rng.integers(0, spec.V, 12).tolist()) | {0, 1}):
        A, G = oracle.sketch_node(spec.V, 3, x, spec.node_neighbors(x))
        a, gg = g.export_sketch(x, x + 1)
        assert np.array_equal(a[0], A) and np.array_equal(gg[0], G), x


def test_invalid_batch_is_discarded_whole():
    V = 100
    u, v = S.random_stream(V, 1000, seed=5)
    g = _gpu_graph(V, 3, u, v)
    before = g.export_sketch()
    bad_u = np.array([1, 2, 3, 4], np.uint32)
    bad_v = np.array([2, 3, 3, 5], np.uint32)  # a self loop
    g.edge_update(_dev(bad_u), _dev(bad_v))
    with pytest.raises(gz.GzError) as ei:
        g.sync()
    assert ei.value.status == gz.GZ_EINVAL
    g.sync()  # reported once
    after = g.export_sketch()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    g.edge_update(_dev(np.array([5], np.uint32)), _dev(np.array([100], np.uint32)))  # id >= V
    with pytest.raises(gz.GzError):
        g.sync()
    after = g.export_sketch()
    assert np.array_equal(before[0], after[0])


@pytest.mark.parametrize("pipelined", [True, False])
def test_host_input_slices_ramp_up_and_validate_each_slice(pipelined):
    # host input is cut into slices of 2^c/16, 2^c/4, then 2^c updates; a bad
    # update discards exactly its slice (here the second: updates 256..1279
    # at 2^c = 4096) and every other slice is applied
    V, seed = 500, 8
    u, v = S.random_stream(V, 12000, seed=9, n_distinct=6000)
    u[700] = v[700]  # a self loop in the second slice
    g = gz.Graph(V, seed, chunk_log2=12, no_pipeline=0 if pipelined else 1)
    g.edge_update(u, v)
    with pytest.raises(gz.GzError) as ei:
        g.sync()
    assert ei.value.status == gz.GZ_EINVAL
    keep = np.ones(len(u), bool)
    keep[256:256 + 1024] = False
    A, G = oracle.ingest(V, seed, u[keep], v[keep])
    _assert_same_sketches(g, A, G)
    g.close()


def test_empty_graph_single_edge_and_reset():
    V = 50
    g = gz.Graph(V, 1)
    labels, ncc, st = g.connected_components()
    assert ncc == V and np.array_equal(labels, np.arange(V))
    g.edge_update(_dev(np.array([7], np.uint32)), _dev(np.array([3], np.uint32)))
    forest, labels, st = g.list_spanning_forest()
    assert forest.tolist() == [[3, 7]] and labels[7] == 3
    g.reset()
    labels, ncc, _ = g.connected_components()
    assert ncc == V
    a, _ = g.export_sketch()
    assert not a.any()


WIDE_HUBS = [0, 1, 2, 65536, 70000]


def test_wide_indices_ragged_stream_sampled_nodes():
    # V^2 > 2^32 (64-bit edge indices, the kernel's wide record path), V not a
    # power of two, 2^18-update batches with a ragged last batch, the device
    # and host input paths; sampled node sketches (hubs spanning many tiles,
    # random nodes, the last node) equal the oracle's, labels the exact
    # components of the net graph
    V, seed = 70001, 9
    u, v = S.hub_stream(V, 600000, seed, WIDE_HUBS)
    eu, ev = S.net_graph(V, u, v)
    g = gz.Graph(V, seed, chunk_log2=18)
    g.edge_update(_dev(u[:400000]), _dev(v[:400000]))
    g.edge_update(u[400000:], v[400000:])
    g.sync()
    rng = np.random.default_rng(1)
    nodes = sorted(set(WIDE_HUBS) | set(rng.integers(0, V, 20).tolist()) | {3, V - 2})
    for x in nodes:
        A, G = oracle.sketch_node(V, seed, x, S.neighbors_from_edges(V, eu, ev, x))
        a, gg = g.export_sketch(x, x + 1)
        assert np.array_equal(a[0], A) and np.array_equal(gg[0], G), x
    labels, ncc, st = g.connected_components()
    assert st["fails_last"] == 0 and st["exhausted"] == 0
    assert np.array_equal(labels, oracle.cc_edges(V, eu.astype(np.uint32), ev.astype(np.uint32)))
    g.close()


def test_checkpoint_restore_resumes_exactly():
    V = 2500
    u, v = S.random_stream(V, 40000, seed=31)
    A, G = oracle.ingest(V, 14, u, v)
    g = gz.Graph(V, 14)
    g.edge_update(_dev(u[:15000]), _dev(v[:15000]))
    ck = g.checkpoint()
    assert bytes(ck[:8]) == b"GZB3CKP1"
    h = gz.Graph.restore(ck)
    for x in (g, h):
        x.edge_update(_dev(u[15000:]), _dev(v[15000:]))
        x.sync()
        _assert_same_sketches(x, A, G)
    assert np.array_equal(g.connected_components()[0], h.connected_components()[0])
    bad = ck.copy()
    bad[0] ^= 1
    with pytest.raises(gz.GzError):
        gz.Graph.restore(bad)
    with pytest.raises(gz.GzError):
        gz.Graph.restore(ck[: len(ck) - 1])


@pytest.mark.parametrize("on_device", [True, False])
def test_packed_index_updates_match_oracle(on_device):
    # gz_edge_update_idx: idx = min*V + max, several chunks and a ragged tail,
    # both endpoint orders in the source stream (the packed form is canonical)
    import torch
    V = 3000
    u, v = S.random_stream(V, 7000, seed=9, n_distinct=2500)
    lo, hi = np.minimum(u, v).astype(np.uint64), np.maximum(u, v).astype(np.uint64)
    idx = lo * np.uint64(V) + hi
    A, G = oracle.ingest(V, 17, u, v)
    g = gz.Graph(V, 17, chunk_log2=11)
    if on_device:
        g.edge_update_idx(torch.from_numpy(idx.view(np.int64)).cuda())
    else:
        g.edge_update_idx(idx)
    g.sync()
    _assert_same_sketches(g, A, G)


def test_packed_index_rejects_non_canonical():
    V = 50
    u, v = S.random_stream(V, 400, seed=4)
    g = _gpu_graph(V, 3, u, v)
    before = g.export_sketch()
    for bad in ([1 * V + 2, 7 * V + 3], [5 * V + 5], [V * V], [2 ** 63 + 1]):  # max<min, loop, >= V^2
        g.edge_update_idx(np.array([3 * V + 4] + bad, np.uint64))
        with pytest.raises(gz.GzError) as ei:
            g.sync()
        assert ei.value.status == gz.GZ_EINVAL
    after = g.export_sketch()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])


def test_queries_during_the_stream_see_each_prefix():
    # a CC query after every quarter of the stream (the experiment of Fig.
    # query): each sees exactly the sketches of the prefix ingested so far;
    # queries leave the sketches untouched, so ingestion simply continues
    spec = S.PlantedSpec(V=1024, seed=21, n_comp=8, p=0.1, extra=0.2, cycles=20)
    u, v, comp = S.planted_stream(spec)
    g = gz.Graph(spec.V, 5, chunk_log2=14)
    cuts = [len(u) * i // 4 for i in range(5)]
    for i in range(1, 5):
        g.edge_update(_dev(u[cuts[i - 1]:cuts[i]]), _dev(v[cuts[i - 1]:cuts[i]]))
        labels, ncc, st = g.connected_components()
        A, G = oracle.ingest(spec.V, 5, u[:cuts[i]], v[:cuts[i]])
        want = oracle.boruvka(spec.V, 5, A, G)
        assert np.array_equal(labels, want["labels"]), i
        assert np.array_equal(labels, oracle.brute_cc(spec.V, u[:cuts[i]], v[:cuts[i]])), i
    _assert_same_sketches(g, A, G)


def test_empty_component_stays_final_on_the_device():
    """The rule that a component sampled EMPTY is final, on the device: with
    the round-0 CubeSketches of 5 and 9 cleared in the device sketch array
    (and in the oracle's copy), the pair reports EMPTY in round 1 too and
    stays apart, sample for sample as the oracle does."""
    import torch

    class _Bytes:
        def __init__(self, ptr, nbytes):
            self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                             "version": 3}

    V, seed = 64, 3
    u = np.array([5, 20], np.uint32)
    v = np.array([9, 21], np.uint32)
    A, G = oracle.ingest(V, seed, u, v)
    A[[5, 9], 0] = 0
    G[[5, 9], 0] = 0
    g = _gpu_graph(V, seed, u, v)
    info = g.info()
    for node in (5, 9):  # CubeSketch 0 is the first 84R bytes of a node's sketch
        t = torch.as_tensor(_Bytes(info["sketch_ptr"] + node * info["node_bytes"], 84 * info["R"]),
                            device="cuda")
        t.zero_()
    torch.cuda.synchronize()
    want = _assert_same_query(g, A, G, seed)
    assert want["labels"][9] == 9 and want["labels"][21] == 20
    assert want["samples"][1][5] == -1 and want["samples"][1][9] == -1
