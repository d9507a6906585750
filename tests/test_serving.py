"""Serving many graphs on one GPU (gz_server): every graph's results in the
mix equal its results alone, memory admission keeps the resident bytes within
the budget, and requests that arrive while others run are admitted as slots
and memory free up.  Labels and sketches are integers, so "equal" is exact."""
import numpy as np
import pytest

import oracle
import paper_2203_14927_b300 as gz
from paper_2203_14927_b300 import streams as S

pytestmark = pytest.mark.gpu


def _graph_requests(i, rng):
    """A mixed workload: Kronecker or planted G(n,p), cut into update chunks
    with queries between them."""
    L = int(rng.integers(8, 12))
    V = 1 << L
    if i % 2 == 0:
        spec = S.KronSpec(L=L, seed=100 + i, target_edges=0.3 * V * (V - 1) / 2, churn=0.1,
                          n_iso=3, slice_log2=2 * L - 3)
        u, v = spec.stream()
    else:
        spec = S.PlantedSpec(V=V, seed=100 + i, n_comp=4, p=0.08, extra=0.2, cycles=2)
        u, v, _ = S.planted_stream(spec)
    cuts = np.sort(rng.choice(np.arange(1, len(u)), size=5, replace=False))
    parts = np.split(np.arange(len(u)), cuts)
    reqs = []
    for k, p in enumerate(parts):
        reqs.append(("u", u[p], v[p]))
        if k % 2 == 1 or k == len(parts) - 1:
            reqs.append(("q",))
    return V, 500 + i, reqs


def _alone(V, seed, reqs):
    """Labels and status of every query when the graph runs by itself."""
    g = gz.Graph(V, seed)
    out = []
    for r in reqs:
        if r[0] == "u":
            g.edge_update(r[1], r[2])
        else:
            labels, _, st = g.connected_components()
            out.append((labels, st["status"]))
    g.close()
    return out


def test_results_in_the_mix_equal_results_alone_and_budget_holds():
    rng = np.random.default_rng(42)
    graphs = [_graph_requests(i, rng) for i in range(8)]
    want = [_alone(V, seed, reqs) for V, seed, reqs in graphs]
    # a budget that fits only a few graphs at once, so admission must queue
    sizes = []
    for V, _, _ in graphs:
        import ctypes
        b = ctypes.c_size_t()
        gz.lib().gz_memory_bytes(V, None, ctypes.byref(b))
        sizes.append(b.value)
    budget = int(3.2 * max(sizes)) + (700 << 20)
    srv = gz.Server(hbm_budget=budget, slots=3, max_batch=2)
    gids = [srv.add_graph(V, seed) for V, seed, _ in graphs]
    # interleave the graphs' requests in a random order (per-graph order kept)
    cursors = [0] * len(graphs)
    qids = {}
    remaining = sum(len(r) for _, _, r in graphs)
    while remaining:
        i = int(rng.integers(0, len(graphs)))
        if cursors[i] == len(graphs[i][2]):
            continue
        r = graphs[i][2][cursors[i]]
        cursors[i] += 1
        remaining -= 1
        if r[0] == "u":
            # half the batches are lent without a copy (kept alive until polled)
            srv.submit_update(gids[i], r[1], r[2], copy=bool(i % 2))
        else:
            qids[srv.submit_query(gids[i])] = (i, sum(1 for x in graphs[i][2][:cursors[i]] if x[0] == "q") - 1)
        if cursors[i] == len(graphs[i][2]):
            srv.close_graph(gids[i])
    srv.drain()
    done = srv.poll(100000)
    bad = [(c["graph"], c["kind"], c["status"]) for c in done if c["kind"] == 0 and c["status"] != gz.GZ_OK]
    assert not bad, (bad[:4], srv.last_error())
    got = {}
    for c in done:
        if c["kind"] == 1:
            i, k = qids[c["req_id"]]
            got[(i, k)] = (c["labels"], c["status"])
            assert c["done_ms"] >= c["start_ms"] >= c["submit_ms"]
    for i, w in enumerate(want):
        for k, (lab, status) in enumerate(w):
            assert got[(i, k)][1] == status, (i, k, got[(i, k)][1], status)
            assert np.array_equal(got[(i, k)][0], lab), (i, k)
    st = srv.stats()
    assert st["peak_resident_bytes"] <= budget
    assert st["resident_bytes"] == 0 and st["pending_requests"] == 0
    srv.close()


def test_alone_results_match_the_oracle():
    rng = np.random.default_rng(7)
    V, seed, reqs = _graph_requests(1, rng)
    labels = _alone(V, seed, reqs)[-1][0]
    us = np.concatenate([r[1] for r in reqs if r[0] == "u"])
    vs = np.concatenate([r[2] for r in reqs if r[0] == "u"])
    assert np.array_equal(labels, oracle.brute_cc(V, us, vs))


def test_server_rejects_graph_beyond_budget_and_bad_ids():
    srv = gz.Server(hbm_budget=64 << 20, slots=1)
    with pytest.raises(gz.GzError):
        srv.add_graph(1 << 16, 1)  # ~5 GB of sketches
    assert gz.lib().gz_server_submit_query(srv._s, 99, None, None) == gz.GZ_EINVAL
    gid = srv.add_graph(64, 1)
    srv.close_graph(gid)
    assert gz.lib().gz_server_submit_query(srv._s, gid, None, None) == gz.GZ_EINVAL
    srv.close()


def _server_graph_bytes(V):
    """Device bytes the server reserves for a graph of V nodes (sketches,
    ingest scratch for 2^20-update batches, query scratch, host staging)."""
    import ctypes
    c = gz.Config()
    c.chunk_log2 = 20
    c.no_pipeline = 1
    b = ctypes.c_size_t()
    gz.lib().gz_memory_bytes(V, ctypes.byref(c), ctypes.byref(b))
    K, R = gz.geometry(V)
    return b.value + V * 96 + (V // 2 + 1) * 84 * R + (16 << 20)


def test_idle_graphs_are_evicted_and_restored_bit_for_bit():
    """A budget for one graph: a graph that waits for memory evicts the idle
    resident one (checkpoint to host), whose next request restores it; each
    graph's results still equal its results alone."""
    rng = np.random.default_rng(5)
    graphs = [_graph_requests(i, rng) for i in range(2)]
    want = [_alone(V, seed, reqs) for V, seed, reqs in graphs]
    budget = int(1.5 * max(_server_graph_bytes(V) for V, _, _ in graphs))
    srv = gz.Server(hbm_budget=budget, slots=2, max_batch=4)
    gids = [srv.add_graph(V, seed) for V, seed, _ in graphs]
    got = {0: [], 1: []}

    def run(i, reqs):
        for r in reqs:
            if r[0] == "u":
                srv.submit_update(gids[i], r[1], r[2])
            else:
                srv.submit_query(gids[i])
        srv.drain()
        for c in srv.poll(1000):
            assert c["status"] in (gz.GZ_OK, gz.GZ_ESKETCH_FAIL), srv.last_error()
            if c["kind"] == 1:
                got[c["graph"]].append((c["labels"], c["status"]))

    halves = [(r[: len(r) // 2], r[len(r) // 2:]) for _, _, r in graphs]
    run(0, halves[0][0])  # graph 0 resident, then idle
    run(1, halves[1][0])  # graph 1 waits, evicts graph 0
    run(0, halves[0][1])  # graph 0 restored from its checkpoint, graph 1 evicted
    run(1, halves[1][1])  # and back
    for i in range(2):
        srv.close_graph(gids[i])
    srv.drain()
    st = srv.stats()
    assert st["evictions"] >= 3, st
    assert st["peak_resident_bytes"] <= budget
    assert st["resident_bytes"] == 0 and st["evicted_graphs"] == 0
    srv.close()
    for i in range(2):
        assert len(got[i]) == len(want[i])
        for (lab, status), (wl, ws) in zip(got[i], want[i]):
            assert status == ws and np.array_equal(lab, wl), i
