"""Sketches beyond HBM (cfg.device_sketch_mb): node shards in pinned host
memory, streamed through device slots per chunk, gathered per Boruvka round.
The results must equal the oracle's (and so an all-HBM handle's) bit for bit."""
import numpy as np
import pytest

import oracle
import paper_2203_14927_b300 as gz
from paper_2203_14927_b300 import streams as S

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


@pytest.mark.parametrize("budget_mb", [64, 1])  # 1364 resident nodes + 11 host shards; 20 + ~1000
def test_tiered_ingest_and_query_match_oracle(budget_mb):
    V = 5000
    u, v = S.random_stream(V, 30000, seed=3, n_distinct=9000)
    A, G = oracle.ingest(V, 8, u, v)
    g = gz.Graph(V, 8, chunk_log2=12, device_sketch_mb=budget_mb)
    total = gz.memory_bytes(V, chunk_log2=12, device_sketch_mb=budget_mb)
    assert total < V * A.shape[1] * 7 * A.shape[3] * 12  # less than all sketches in HBM
    g.edge_update(_dev(u[:20000]), _dev(v[:20000]))
    g.edge_update(u[20000:], v[20000:])  # host input path, several chunks
    g.sync()
    a, gg = g.export_sketch()
    assert np.array_equal(a, A) and np.array_equal(gg, G)
    a, gg = g.export_sketch(1200, 4100)  # a range across the resident boundary
    assert np.array_equal(a, A[1200:4100]) and np.array_equal(gg, G[1200:4100])
    want = oracle.boruvka(V, 8, A, G)
    labels, ncc, st = g.connected_components()
    assert np.array_equal(labels, want["labels"]) and st["rounds"] == want["rounds"]
    g.enable_trace(True)
    forest, labels, st = g.list_spanning_forest()
    assert np.array_equal(g.query_trace(), want["samples"])
    assert np.array_equal(forest, want["forest"])


def test_tiered_kronecker_checkpoint_and_reset():
    spec = S.KronSpec(L=11, seed=5, target_edges=4e5, churn=0.1, n_iso=10, slice_log2=16)
    u, v = spec.stream()
    A, G = oracle.ingest(spec.V, 2, u, v)
    g = gz.Graph(spec.V, 2, chunk_log2=16, device_sketch_mb=16)
    g.edge_update(_dev(u), _dev(v))
    g.sync()
    labels, ncc, st = g.connected_components()
    assert np.array_equal(labels, oracle.boruvka(spec.V, 2, A, G)["labels"])
    ck = g.checkpoint()
    for budget in (0, 8):  # restore into an all-HBM handle and into a tiered one
        h = gz.Graph.restore(ck, device_sketch_mb=budget)
        a, gg = h.export_sketch()
        assert np.array_equal(a, A) and np.array_equal(gg, G)
        h.close()
    g.reset()
    a, gg = g.export_sketch()
    assert not a.any() and not gg.any()
    # the device array of a tiered handle holds only some nodes: gz_info
    # withholds its pointer, so nothing can mistake it for the whole sketch
    assert g.info()["sketch_ptr"] is None
    g.close()


def test_tiered_wide_indices_match_all_hbm_and_oracle():
    # the windowed kernel on 64-bit edge indices (V^2 > 2^32): ~6,700 nodes
    # resident, the rest in pinned host memory; sampled node sketches from
    # both tiers equal the oracle's, labels and per-round samples equal an
    # all-HBM handle's
    V, seed = 70001, 9
    hubs = [0, 1, 2, 65536, 70000]
    u, v = S.hub_stream(V, 600000, seed, hubs)
    eu, ev = S.net_graph(V, u, v)
    g = gz.Graph(V, seed, chunk_log2=18, device_sketch_mb=512)
    g.edge_update(_dev(u[:400000]), _dev(v[:400000]))
    g.edge_update(u[400000:], v[400000:])
    g.sync()
    rng = np.random.default_rng(2)
    nodes = sorted(set(hubs) | set(rng.integers(0, V, 12).tolist()))
    for x in nodes:
        A, G = oracle.sketch_node(V, seed, x, S.neighbors_from_edges(V, eu, ev, x))
        a, gg = g.export_sketch(x, x + 1)
        assert np.array_equal(a[0], A) and np.array_equal(gg[0], G), x
    h = gz.Graph(V, seed, chunk_log2=18)
    h.edge_update(_dev(u), _dev(v))
    h.sync()
    a1, g1 = g.export_sketch(6000, 7500)  # across the resident boundary
    a2, g2 = h.export_sketch(6000, 7500)
    assert np.array_equal(a1, a2) and np.array_equal(g1, g2)
    g.enable_trace(True)
    h.enable_trace(True)
    f1, l1, s1 = g.list_spanning_forest()
    f2, l2, s2 = h.list_spanning_forest()
    assert np.array_equal(l1, l2) and np.array_equal(f1, f2)
    assert np.array_equal(g.query_trace(), h.query_trace())
    g.close()
    h.close()
