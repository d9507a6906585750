"""The seeded stream generators follow the paper's stream rules (Section 6.1,
"Synthesizing Dense Graphs and Streams": (i) insert before delete, (ii) no two
consecutive updates of one type, (iii) a few disconnected nodes, (iv) the final
graph is exactly the input graph) and the Kronecker model it names."""
import itertools
import math

import numpy as np

from paper_2203_14927_b300 import streams as S


def test_kronecker_expected_edges_closed_form_matches_enumeration():
    for L in (3, 4, 5):
        V = 1 << L
        for s in (0.5, 7.0, 40.0):
            a, b, _, d = S.THETA
            brute = 0.0
            for u, v in itertools.combinations(range(V), 2):
                n11 = bin(u & v).count("1")
                n00 = L - bin(u | v).count("1")
                brute += min(1.0, s * a ** n00 * b ** (L - n00 - n11) * d ** n11)
            assert math.isclose(S._kron_expected_edges(L, s), brute, rel_tol=1e-12)


def test_feistel_order_is_a_permutation_of_ordered_pairs():
    spec = S.KronSpec(L=5, seed=3, target_edges=200.0, slice_log2=6)
    u, v = spec.position_pairs(np.arange(spec.V * spec.V, dtype=np.uint64))
    idx = u * np.uint64(spec.V) + v
    assert len(np.unique(idx)) == spec.V * spec.V


def test_kronecker_stream_rules_and_final_graph():
    spec = S.KronSpec(L=9, seed=5, target_edges=0.4 * 512 * 511 / 2, churn=0.1,
                      n_iso=8, slice_log2=13)
    us, vs = [], []
    for c in range(spec.n_chunks):
        u, v = spec.chunk(c)
        assert np.all(u < v)
        us.append(u)
        vs.append(v)
    u = np.concatenate(us)
    v = np.concatenate(vs)
    # (iv) the net graph is the final graph
    eu, ev = S.net_graph(spec.V, u, v)
    fu, fv = spec.final_edges()
    assert np.array_equal(eu, fu) and np.array_equal(ev, fv)
    # (i)/(ii) per pair: at most two updates, and a pair updated twice is a
    # churn pair (inserted first, deleted later)
    idx = u.astype(np.uint64) * spec.V + v
    vals, counts = np.unique(idx, return_counts=True)
    assert counts.max() <= 2
    twice = vals[counts == 2]
    cu, cv = (twice // spec.V).astype(np.uint32), (twice % spec.V).astype(np.uint32)
    assert spec.churn_pair(cu, cv).all()
    # (iii) isolated nodes have no final edge
    iso = np.nonzero(spec.isolated(np.arange(spec.V)))[0]
    assert len(iso) > 0
    assert not np.isin(fu, iso).any() and not np.isin(fv, iso).any()
    # realised size near the target (minus the isolated nodes' edges)
    assert abs(len(fu) / spec.target_edges - 1) < 0.1
    assert abs(len(twice) / (spec.churn * spec.target_edges) - 1) < 0.15


def test_kronecker_node_neighbors_match_final_edges():
    spec = S.KronSpec(L=8, seed=2, target_edges=9000.0, slice_log2=12)
    fu, fv = spec.final_edges()
    for x in (0, 1, 77, 255):
        want = S.neighbors_from_edges(spec.V, fu, fv, x)
        assert np.array_equal(spec.node_neighbors(x), want)


def test_kronecker_degrees_follow_the_initiator():
    # hubs are the nodes with few 1 bits (largest initiator entry a = 0.57)
    spec = S.KronSpec(L=10, seed=1, target_edges=60000.0, n_iso=0.0, slice_log2=16)
    fu, fv = spec.final_edges()
    deg = np.bincount(np.concatenate([fu, fv]), minlength=spec.V)
    pop = np.array([bin(x).count("1") for x in range(spec.V)])
    means = [deg[pop == k].mean() for k in range(11)]
    assert all(means[k] > means[k + 1] for k in range(9))


def test_planted_stream_net_graph_stays_inside_components():
    spec = S.PlantedSpec(V=1024, seed=3, n_comp=8, p=0.1, extra=0.2, cycles=3)
    u, v, comp = S.planted_stream(spec)
    assert np.all(u != v)
    eu, ev = S.net_graph(spec.V, u, v)
    assert np.all(comp[eu] == comp[ev])
    assert len(np.unique(comp)) == 8
    # stream length = |E| + 2 * cycles * extra * |E|
    assert len(u) == len(eu) + 2 * spec.cycles * int(round(spec.extra * len(eu)))


def test_random_stream_any_v():
    u, v = S.random_stream(3, 100, seed=1)
    assert np.all(u != v) and u.max() < 3 and v.max() < 3


def test_hub_stream_is_seeded_valid_and_hub_heavy():
    V, hubs = 70001, [0, 1, 2, 65536, 70000]
    u, v = S.hub_stream(V, 20000, 4, hubs)
    u2, v2 = S.hub_stream(V, 20000, 4, hubs)
    assert np.array_equal(u, u2) and np.array_equal(v, v2)
    assert len(u) > 19990 and (u != v).all() and u.max() < V and v.max() < V
    at_hub = np.isin(u, hubs) | np.isin(v, hubs)
    assert 0.45 < at_hub.mean() < 0.55
