"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (Table tab:size, the "one-tenth of sketch size" buffer), the
published SplitMix64 outputs, closed forms and pairwise independence of the
checksum h2, the scan order of Fig. cube_code's query on hand-built sketches,
the set definition of a bucket (Eq. 1-2) against the update loop (Fig.
cube_code), linearity (Definition def:l0), Lemma goodcheck, the membership law
behind Lemma goodset, and brute-force connected components checked in turn
against scipy's graph routine.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import oracle
from paper_2203_14927_b300 import streams as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def _idx(V, u, v):
    return min(u, v) * V + max(u, v)


# ----------------------------------------------------------------- hashing


def test_splitmix64_published_outputs():
    want = [int(r[0]) for r in _golden("splitmix64_1234567.txt")]
    got = [oracle.splitmix64_at(1234567, i) for i in range(5)]
    assert got == want


def _key_row(h1_pieces=(), h2_pieces=()):
    """One column's 256 key words with the given (k0, k1, k2) per piece."""
    k = np.zeros(oracle.KEY_WORDS, np.uint32)
    for i, t in enumerate(h1_pieces):
        k[3 * i:3 * i + 3] = t
    for i, t in enumerate(h2_pieces):
        k[128 + 3 * i:128 + 3 * i + 3] = t
    return k


def test_piece_geometry():
    # p = min(16, 33 - ceil(log2 V)); h1 covers the R - 1 = 2L - 1 depth bits,
    # h2 32 bits
    for V, want in [(2, (16, 1, 2)), (1000, (16, 2, 2)), (1 << 13, (16, 2, 2)), (70001, (16, 3, 2)),
                    (1 << 17, (16, 3, 2)), (1 << 18, (15, 3, 3)), (1 << 20, (13, 3, 3)),
                    (1 << 31, (2, 31, 16))]:
        assert oracle.pieces(V) == want, V


def test_hash_pieces_closed_forms():
    # With degenerate keys every piece reduces to a closed form: a constant
    # (the top p bits of k2), the low p bits of u or of v moved to the top, or
    # a sum whose carry crosses into the piece.  The concatenation
    # order (first piece most significant), the piece width, a transposed
    # pair, a wrong shift or a lost carry fails one of these.
    rng = np.random.default_rng(5)
    for V in (1000, 70001, 1 << 17, 1 << 20):
        p, m1, m2 = oracle.pieces(V)
        L = (V - 1).bit_length()
        edges = [(0, 1), (1, 2), (V - 2, V - 1), (0, V - 1)]
        edges += [tuple(sorted(rng.choice(V, 2, replace=False).tolist())) for _ in range(30)]
        consts = [int(t) for t in rng.integers(0, 2**32, 16, dtype=np.uint64)]
        for u, v in edges:
            e = u * V + v
            # constants only: h2 = the top p bits of each k2, concatenated, first 32 bits
            k = _key_row(h2_pieces=[(0, 0, c) for c in consts[:m2]])
            bits = "".join(format(c >> (32 - p), f"0{p}b") for c in consts[:m2])[:32]
            assert oracle.h2(V, k, e) == int(bits, 2)
            # word selection: k0 = 2^(32-p) puts u's low p bits at the top of piece 0
            k = _key_row(h2_pieces=[(1 << (32 - p), 0, 0), (0, 1 << (32 - p), 0)] + [(0, 0, 0)] * (m2 - 2))
            bits = (format(u % (1 << p), f"0{p}b") + format(v % (1 << p), f"0{p}b"))[:32].ljust(32, "0")
            assert oracle.h2(V, k, e) == int(bits, 2)
            # carry: top p bits of (u + 2^32 - 1) mod 2^32 are all ones iff u == 0
            k = _key_row(h2_pieces=[(1, 0, 2**32 - 1)] + [(0, 0, 0)] * (m2 - 1))
            top = ((u + 2**32 - 1) % 2**32) >> (32 - p)
            assert oracle.h2(V, k, e) >> (32 - p) == top
            # h1: col_hash bit i = the i-th bit of the H1 pieces from the top
            k = _key_row(h1_pieces=[(0, 0, c) for c in consts[:m1]])
            bits = "".join(format(c >> (32 - p), f"0{p}b") for c in consts[:m1])
            ch = oracle.h1(V, k, e)
            assert all((ch >> i) & 1 == int(bits[i]) for i in range(len(bits)))
            assert ch >> len(bits) == 0
            k = _key_row(h1_pieces=[(0, 1 << (32 - p), 0)] + [(0, 0, 0)] * (m1 - 1))
            ch = oracle.h1(V, k, e)
            bits = format(v % (1 << p), f"0{p}b")
            assert all((ch >> i) & 1 == int(bits[i]) for i in range(p)), (V, u, v)
        assert L == (V - 1).bit_length() and p == min(16, 33 - L)


def _chi2_uniform(counts):
    e = counts.sum() / counts.size
    return float(((counts - e) ** 2 / e).sum())


@pytest.mark.parametrize("V", [1000, 1 << 17, 1 << 20])
def test_h2_is_pairwise_independent(V):
    # Section 3.2 asks for h2 from a 2-wise independent family: for two
    # distinct edges and uniform keys, (h2(e), h2(f)) is uniform on pairs of
    # 32-bit words.  Checked on the top three and the low three output bits
    # (the latter fall in the last piece), for edges sharing u, sharing v,
    # sharing nothing, and differing by one or by a power of two.
    rng = np.random.default_rng(17)
    pairs = [((0, 1), (0, 2)), ((5, 9), (7, 9)), ((3, V - 1), (4, V - 2)), ((1, 2), (1, 2 + 256)),
             ((0, V // 2), (V // 2, V - 1)), ((11, 12), (13, 14))]
    n = 6400
    keys = rng.integers(0, 2**32, (n, oracle.KEY_WORDS), dtype=np.uint64).astype(np.uint32)
    limit = 63 + 6 * np.sqrt(2 * 63)  # chi-square, 63 degrees of freedom, far tail
    for (a, b), (c, d) in pairs:
        e, f = a * V + b, c * V + d
        top = np.zeros((8, 8))
        low = np.zeros((8, 8))
        for k in keys:
            he, hf = oracle.h2(V, k, e), oracle.h2(V, k, f)
            top[he >> 29, hf >> 29] += 1
            low[he & 7, hf & 7] += 1
        assert _chi2_uniform(top) < limit, (V, e, f, "top bits")
        assert _chi2_uniform(low) < limit, (V, e, f, "low bits")


@pytest.mark.parametrize("V", [1000, 1 << 17, 1 << 20])
def test_depth_bits_are_pairwise_independent(V):
    # Lemma goodset uses P[e in B_i] = 2^-i and pairwise independence of
    # membership (2-wise independent h1).  The first three H1 bits and the
    # three bits that straddle the first piece boundary (where a word or
    # carry mistake would correlate two edges) are jointly uniform.
    p, m1, _ = oracle.pieces(V)
    rng = np.random.default_rng(23)
    pairs = [((0, 1), (0, 2)), ((5, 9), (7, 9)), ((1, 2), (3, 4)), ((2, V - 1), (3, V - 1))]
    n = 6400
    keys = rng.integers(0, 2**32, (n, oracle.KEY_WORDS), dtype=np.uint64).astype(np.uint32)
    limit = 63 + 6 * np.sqrt(2 * 63)
    span = [0, 1, 2] if m1 == 1 else [p - 2, p - 1, p]
    for (a, b), (c, d) in pairs:
        e, f = a * V + b, c * V + d
        first = np.zeros((8, 8))
        cross = np.zeros((8, 8))
        for k in keys:
            he, hf = oracle.h1(V, k, e), oracle.h1(V, k, f)
            first[he & 7, hf & 7] += 1
            cross[sum(((he >> i) & 1) << t for t, i in enumerate(span)),
                  sum(((hf >> i) & 1) << t for t, i in enumerate(span))] += 1
        assert _chi2_uniform(first) < limit, (V, e, f)
        assert _chi2_uniform(cross) < limit, (V, e, f)


def test_checksum_is_not_xor_linear():
    # Lemma goodcheck needs h2(x) ^ h2(y) != h2(x ^ y) except with
    # probability ~2^-32; a GF(2)-linear checksum would pass every bucket.
    V = 1 << 17
    rng = np.random.default_rng(11)
    keys = oracle.keys(3, 1)
    hits = tried = 0
    for t in range(40000):
        a, b, c, d = (int(z) for z in rng.integers(0, V, 4))
        if a >= b or c >= d or (a, b) == (c, d):
            continue
        x, y = a * V + b, c * V + d
        z = x ^ y
        if z >= V * V or z // V >= z % V:
            continue  # x ^ y is not an edge: the decode check already rejects it
        tried += 1
        ck = keys[t % 7]
        hits += (oracle.h2(V, ck, x) ^ oracle.h2(V, ck, y)) == oracle.h2(V, ck, z)
    assert tried > 4000 and hits == 0


def test_row_membership_law():
    # P[e in nested row i] = 2^-i under the schedule's keys (Lemma goodset)
    V = 1 << 17
    K, R = oracle.geometry(V)
    keys = oracle.keys(99, K)
    rng = np.random.default_rng(2)
    n = 6000
    counts = np.zeros(6)
    for t in range(n):
        a, b = sorted(rng.choice(V, 2, replace=False).tolist())
        h = oracle.h1(V, keys[t % (K * 7)], a * V + b)
        for i in range(6):
            counts[i] += (h & ((1 << i) - 1)) == 0
    for i in range(6):
        q = 2.0 ** -i
        assert abs(counts[i] / n - q) < 5 * np.sqrt(q * (1 - q) / n) + 1e-9


# ----------------------------------------------------------------- geometry


def test_geometry_small_cases():
    assert oracle.geometry(2) == (2, 2)
    assert oracle.geometry(3) == (3, 4)
    assert oracle.geometry(1024) == (18, 20)
    with pytest.raises(ValueError):
        oracle.geometry(1)


def test_geometry_reproduces_table_tab_size():
    # node sketch = K * 7 * R buckets of 12 B (Section 5.1, "Sketch updates");
    # memory = sketches + leaf gutters of half a node sketch each.  The paper
    # reads process memory from `top`, so the computed size must lie at or
    # below each entry and within 4% of it; K-1 or K+1 CubeSketches per node
    # leave that band at one of the five sizes.
    for K_shift in (0, -1, 1):
        ok = True
        for log2v, gib in _golden("tab_size.txt"):
            V = 1 << int(log2v)
            K, R = oracle.geometry(V)
            total = V * (K + K_shift) * 7 * R * 12 * 1.5 / 2**30
            ok &= 0 <= 1 - total / float(gib) < 0.04
        assert ok == (K_shift == 0), K_shift


def test_geometry_reproduces_buffer_of_one_tenth_sketch():
    # Section 6.6: on kron17, 8.3 KB leaf-only buffers are "one-tenth of
    # sketch size"; Section 5: total ~ 280 V log^2 V bytes.
    V = 1 << 17
    K, R = oracle.geometry(V)
    node_bytes = K * 7 * R * 12
    assert abs(node_bytes / 10 / 8300 - 1) < 0.04
    assert abs(V * node_bytes / (280 * V * 17**2) - 1) < 0.08


# ----------------------------------------------------------------- update


def _bucket_definition(V, seed, edges):
    """Nested buckets from Eq. 1-2: alpha_{i,j} = XOR of the indices e of the
    vector with h1(e) = 0 mod 2^i (capped at row R-1), gamma likewise."""
    K, R = oracle.geometry(V)
    keys = oracle.keys(seed, K)
    A = np.zeros((V, K, 7, R), np.uint64)
    G = np.zeros((V, K, 7, R), np.uint32)
    for (u, v) in edges:
        e = _idx(V, u, v)
        for k in range(K):
            for j in range(7):
                col = k * 7 + j
                h = oracle.h1(V, keys[col], e)
                g = oracle.h2(V, keys[col], e)
                for i in range(R):
                    if h % (1 << i) == 0:
                        for node in (u, v):
                            A[node, k, j, i] ^= np.uint64(e)
                            G[node, k, j, i] ^= np.uint32(g)
    return A, G


@pytest.mark.parametrize("V", [3, 4, 5])
def test_update_loop_matches_bucket_definition_exhaustive(V):
    pairs = list(itertools.combinations(range(V), 2))
    subsets = range(1 << len(pairs))
    if V == 5:
        subsets = np.random.default_rng(0).choice(1 << len(pairs), 96, replace=False)
    for s in subsets:
        edges = [p for i, p in enumerate(pairs) if s >> i & 1]
        u = np.array([e[0] for e in edges], np.uint32)
        v = np.array([e[1] for e in edges], np.uint32)
        A, G = oracle.ingest(V, 17, u, v)
        A2, G2 = _bucket_definition(V, 17, edges)
        assert np.array_equal(A, A2) and np.array_equal(G, G2), (V, s)


def test_update_loop_matches_definition_random_larger_v():
    V = 37
    rng = np.random.default_rng(4)
    pairs = [p for p in itertools.combinations(range(V), 2) if rng.random() < 0.15]
    u = np.array([p[0] for p in pairs], np.uint32)
    v = np.array([p[1] for p in pairs], np.uint32)
    A, G = oracle.ingest(V, 5, u, v)
    A2, G2 = _bucket_definition(V, 5, pairs)
    assert np.array_equal(A, A2) and np.array_equal(G, G2)


def test_insert_then_delete_gives_zero_sketch():
    V = 200
    u, v = S.random_stream(V, 3000, seed=1, n_distinct=3000)
    uu = np.concatenate([u, v])  # each pair twice, orientation flipped
    vv = np.concatenate([v, u])
    A, G = oracle.ingest(V, 8, uu, vv)
    assert not A.any() and not G.any()


def test_sketch_of_symmetric_difference_is_xor():
    V = 150
    ua, va = S.random_stream(V, 2000, seed=2)
    ub, vb = S.random_stream(V, 2000, seed=3)
    A1, G1 = oracle.ingest(V, 9, ua, va)
    A2, G2 = oracle.ingest(V, 9, ub, vb)
    A3, G3 = oracle.ingest(V, 9, np.concatenate([ua, ub]), np.concatenate([va, vb]))
    assert np.array_equal(A1 ^ A2, A3) and np.array_equal(G1 ^ G2, G3)


def test_sketch_of_stream_equals_sketch_of_net_graph_any_order():
    V = 128
    u, v = S.random_stream(V, 5000, seed=4, n_distinct=900)
    A, G = oracle.ingest(V, 10, u, v)
    perm = np.random.default_rng(1).permutation(len(u))
    Ap, Gp = oracle.ingest(V, 10, u[perm], v[perm])
    assert np.array_equal(A, Ap) and np.array_equal(G, Gp)
    eu, ev = S.net_graph(V, u, v)
    for x in [0, 1, 17, 64, 127]:
        a, g = oracle.sketch_node(V, 10, x, S.neighbors_from_edges(V, eu, ev, x))
        assert np.array_equal(a, A[x]) and np.array_equal(g, G[x])


def test_invalid_update_is_rejected_whole():
    with pytest.raises(ValueError):
        oracle.ingest(10, 1, np.array([1, 2], np.uint32), np.array([2, 2], np.uint32))
    with pytest.raises(ValueError):
        oracle.ingest(10, 1, np.array([1], np.uint32), np.array([10], np.uint32))


# ----------------------------------------------------------------- query


def test_support_one_buckets_pass_checksum_lemma_goodcheck():
    V = 300
    K, R = oracle.geometry(V)
    keys = oracle.keys(21, K)
    u, v = S.random_stream(V, 800, seed=5, n_distinct=800)
    eu, ev = S.net_graph(V, u, v)
    A, G = oracle.ingest(V, 21, eu, ev)
    checked = 0
    for x in range(0, V, 7):
        nb = S.neighbors_from_edges(V, eu, ev, x)
        elems = [_idx(V, x, int(y)) for y in nb]
        for k in range(0, K, 3):
            for j in range(7):
                col = k * 7 + j
                depth = {}
                for e in elems:
                    h = oracle.h1(V, keys[col], e)
                    depth[e] = min((h & -h).bit_length() - 1 if h else 64, R - 1)
                for i in range(R):
                    members = [e for e in elems if depth[e] >= i]
                    if len(members) == 1:
                        assert int(A[x, k, j, i]) == members[0]
                        assert int(G[x, k, j, i]) == oracle.h2(V, keys[col], members[0])
                        checked += 1
    assert checked > 500


def test_query_single_element_and_empty_vector():
    V = 1000
    K, R = oracle.geometry(V)
    for (u, w) in [(0, 1), (3, 999), (500, 2)]:
        A, G = oracle.ingest(V, 3, np.array([u], np.uint32), np.array([w], np.uint32))
        for k in range(K):
            assert oracle.query_vector(V, 3, k, A[u, k], G[u, k]) == _idx(V, u, w)
    A, G = oracle.empty_sketches(V, 1)
    assert oracle.query_vector(V, 3, 0, A[0, 0], G[0, 0]) == oracle.EMPTY


def _good_bucket(V, kcol, u, w):
    """(alpha, gamma) of a bucket holding only edge {u, w}: it passes the
    checksum of its column (Lemma goodcheck, support one)."""
    e = _idx(V, u, w)
    return e, oracle.h2(V, kcol, e)


def _scan_fixture(V, seed, k, placed):
    """One CubeSketch (layout [j][row]) holding the good buckets `placed`
    {(j, row): (u, w)} and zeros elsewhere."""
    K, R = oracle.geometry(V)
    keys = oracle.keys(seed, K)
    A = np.zeros((7, R), np.uint64)
    G = np.zeros((7, R), np.uint32)
    for (j, row), (u, w) in placed.items():
        A[j, row], G[j, row] = _good_bucket(V, keys[k * 7 + j], u, w)
    return A, G


def test_query_scan_order_is_columns_then_rows_ascending():
    # Fig. cube_code's query loops over columns, and within a column over
    # its buckets from row 0 up; the first good bucket wins.  A row-major
    # scan, a deepest-row-first scan or a last-match scan picks another edge.
    V, seed = 1000, 12
    K, R = oracle.geometry(V)
    cases = [
        ({(0, 9): (1, 2), (1, 0): (3, 4)}, (1, 2)),            # column 0 before column 1
        ({(2, 1): (5, 6), (2, 6): (7, 8), (4, 0): (9, 10)}, (5, 6)),  # row 1 before row 6
        ({(3, R - 1): (11, 12), (3, 2): (13, 14)}, (13, 14)),  # the deepest row last
        ({(6, 0): (15, 16)}, (15, 16)),
    ]
    for k in (0, K - 1):
        for placed, want in cases:
            A, G = _scan_fixture(V, seed, k, placed)
            assert oracle.query_vector(V, seed, k, A, G) == _idx(V, *want), (k, placed)
    # a bucket that fails its checksum, or holds a non-edge, is passed over
    A, G = _scan_fixture(V, seed, 0, {(1, 3): (20, 21), (1, 5): (22, 23)})
    G[1, 3] ^= 1
    assert oracle.query_vector(V, seed, 0, A, G) == _idx(V, 22, 23)
    A[1, 5] = 7 * V + 3  # decodes to u > v: not an edge, whatever gamma holds
    G[1, 5] = 12345
    assert oracle.query_vector(V, seed, 0, A, G) == oracle.FAIL


def test_boruvka_sample_follows_the_scan_order():
    # The same order inside Boruvka: round 0 of a graph whose only nonzero
    # sketch is vertex 0's CubeSketch 0, with three good buckets whose edges
    # all leave {0}; the trace must hold the first in Fig. cube_code's order.
    V, seed = 64, 31
    K, R = oracle.geometry(V)
    alpha, gamma = oracle.empty_sketches(V)
    A, G = _scan_fixture(V, seed, 0, {(2, 1): (0, 5), (2, 6): (0, 3), (4, 0): (0, 7)})
    alpha[0, 0], gamma[0, 0] = A, G
    res = oracle.boruvka(V, seed, alpha, gamma)
    samples, labels = res["samples"], res["labels"]
    assert samples[0, 0] == _idx(V, 0, 5)
    assert all(samples[0, x] == oracle.EMPTY for x in range(1, V))
    assert labels[5] == 0 and labels[3] == 3 and labels[7] == 7
    # a good bucket whose edge stays inside the component is passed over
    # (the cut check): with {0, 5} merged, round 1 must skip (0, 5)
    A1, G1 = _scan_fixture(V, seed, 1, {(0, 0): (0, 5), (0, 4): (0, 9)})
    alpha[0, 1], gamma[0, 1] = A1, G1
    samples = oracle.boruvka(V, seed, alpha, gamma)["samples"]
    assert samples[1, 0] == _idx(V, 0, 9)


def test_query_returns_a_member_and_fails_rarely():
    # Lemma goodset: each CubeSketch fails with probability at most delta;
    # the paper takes delta = 1/100 (Section 4, l0size discussion).
    V = 1 << 12
    rng = np.random.default_rng(7)
    trials, fails = 400, 0
    for t in range(trials):
        x = int(rng.integers(0, V))
        deg = int(rng.integers(1, V - 1))
        nb = rng.choice(np.setdiff1d(np.arange(V), [x]), deg, replace=False).astype(np.uint32)
        A, G = oracle.sketch_node(V, 1000 + t, x, nb)
        members = {_idx(V, x, int(y)) for y in nb}
        r = oracle.query_vector(V, 1000 + t, t % 5, A[t % 5], G[t % 5])
        if r == oracle.FAIL:
            fails += 1
        else:
            assert r in members
    assert fails <= 4  # expected ~1e-4 * 400; delta = 1/100 would allow ~4


# ----------------------------------------------------------------- connected components


def _scipy_labels(V, eu, ev):
    m = sp.coo_matrix((np.ones(len(eu)), (eu, ev)), shape=(V, V))
    _, lab = connected_components(m, directed=False)
    # relabel to the minimum vertex id of each component
    mins = {}
    for x in range(V):
        mins.setdefault(lab[x], x)
    return np.array([mins[lab[x]] for x in range(V)], np.uint32)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_brute_cc_matches_scipy(seed):
    V = 700
    u, v = S.random_stream(V, 1500, seed=seed, n_distinct=500)
    eu, ev = S.net_graph(V, u, v)
    assert np.array_equal(oracle.brute_cc(V, u, v), _scipy_labels(V, eu, ev))
    assert np.array_equal(oracle.cc_edges(V, eu, ev), _scipy_labels(V, eu, ev))


def _check_forest(V, forest, eu, ev, labels):
    net = set(zip(eu.tolist(), ev.tolist()))
    for (a, b) in forest.tolist():
        assert (min(a, b), max(a, b)) in net
    assert len(forest) == V - len(np.unique(labels))
    # acyclic: union-find over the forest edges never joins a set to itself
    parent = list(range(V))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for (a, b) in forest.tolist():
        ra, rb = find(a), find(b)
        assert ra != rb
        parent[max(ra, rb)] = min(ra, rb)
    assert np.array_equal(np.array([find(x) for x in range(V)], np.uint32), labels)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_boruvka_matches_brute_force_planted(seed):
    spec = S.PlantedSpec(V=256, seed=seed, n_comp=8, p=0.1, extra=0.2, cycles=2)
    u, v, comp = S.planted_stream(spec)
    A, G = oracle.ingest(spec.V, seed, u, v)
    res = oracle.boruvka(spec.V, seed, A, G)
    want = oracle.brute_cc(spec.V, u, v)
    assert res["rc"] == 0
    assert np.array_equal(res["labels"], want)
    eu, ev = S.net_graph(spec.V, u, v)
    _check_forest(spec.V, res["forest"], eu, ev, want)
    # every sampled edge is a net edge that leaves its component
    net = set(zip(eu.tolist(), ev.tolist()))
    K, _ = oracle.geometry(spec.V)
    for r in range(res["rounds"]):
        for c, s in enumerate(res["samples"][r]):
            if s > 0:
                a, b = divmod(int(s), spec.V)
                assert (a, b) in net


def test_boruvka_random_sparse_graph_many_components():
    V = 500
    u, v = S.random_stream(V, 400, seed=9, n_distinct=400)
    A, G = oracle.ingest(V, 4, u, v)
    res = oracle.boruvka(V, 4, A, G)
    assert np.array_equal(res["labels"], oracle.brute_cc(V, u, v))
    assert res["n_components"] == len(np.unique(res["labels"]))


def test_boruvka_empty_graph_and_single_edge():
    V = 64
    A, G = oracle.empty_sketches(V)
    res = oracle.boruvka(V, 1, A, G)
    assert np.array_equal(res["labels"], np.arange(V, dtype=np.uint32))
    assert res["rounds"] == 1 and len(res["forest"]) == 0
    A, G = oracle.ingest(V, 1, np.array([5], np.uint32), np.array([9], np.uint32))
    res = oracle.boruvka(V, 1, A, G)
    lab = np.arange(V, dtype=np.uint32)
    lab[9] = 5
    assert np.array_equal(res["labels"], lab)
    assert res["forest"].tolist() == [[5, 9]]


def test_boruvka_kronecker_small():
    spec = S.KronSpec(L=9, seed=3, target_edges=0.3 * 512 * 511 / 2, churn=0.1,
                      n_iso=6, slice_log2=14)
    u, v = spec.stream()
    A, G = oracle.ingest(spec.V, 77, u, v)
    res = oracle.boruvka(spec.V, 77, A, G)
    eu, ev = spec.final_edges()
    want = oracle.cc_edges(spec.V, eu, ev)
    assert np.array_equal(res["labels"], want)
    _check_forest(spec.V, res["forest"], eu, ev, want)


@pytest.mark.parametrize("L,density,seed", [(9, 0.3, 1), (10, 0.45, 2), (11, 0.2, 3)])
def test_kron_components_shortcut_matches_brute_force(L, density, seed):
    from oracle.kron_cc import kron_components

    V = 1 << L
    spec = S.KronSpec(L=L, seed=seed, target_edges=density * V * (V - 1) / 2, n_iso=5, slice_log2=2 * L - 2)
    eu, ev = spec.final_edges()
    want = oracle.cc_edges(V, eu, ev)
    got = kron_components(spec, n_hubs=64)
    assert np.array_equal(got, want)
    assert len(np.unique(want)) > 1  # isolated vertices exist, so the check is not trivial


def test_paper_design_cpu_baseline_equals_oracle():
    # the OpenMP per-node-buffer baseline (Section 5.1's design) must produce
    # the oracle's sketches bit for bit, for every node range and chunking
    V = 300
    u, v = S.random_stream(V, 6000, seed=12, n_distinct=2000)
    A, G = oracle.ingest(V, 9, u, v)
    a, g = oracle.ingest_batched(V, 9, u, v, threads=4, chunk=777)
    assert np.array_equal(a, A) and np.array_equal(g, G)
    a, g = oracle.ingest_batched(V, 9, u, v, node_lo=37, node_hi=190, threads=3, chunk=1 << 20)
    assert np.array_equal(a, A[37:190]) and np.array_equal(g, G[37:190])
    with pytest.raises(ValueError):
        oracle.ingest_batched(V, 9, np.array([3], np.uint32), np.array([3], np.uint32))
    # 16-bit pieces at V = 2^17 (three depth pieces) and 14-bit pieces at
    # V = 2^19 (three checksum pieces): sampled nodes against the oracle
    for V in (1 << 17, 1 << 19):
        u, v = S.hub_stream(V, 4000, 5, [0, 1, V - 1])
        eu, ev = S.net_graph(V, u, v)
        a, g = oracle.ingest_batched(V, 4, u, v, node_lo=0, node_hi=2, threads=2, chunk=1000)
        for x in (0, 1):
            A1, G1 = oracle.sketch_node(V, 4, x, S.neighbors_from_edges(V, eu, ev, x))
            assert np.array_equal(a[x], A1) and np.array_equal(g[x], G1), (V, x)


def test_boruvka_empty_component_is_final():
    """A component whose sketch is entirely zero in a round takes no part in
    later rounds (it reports EMPTY), unless a sampled edge touches it.  With
    the round-0 CubeSketches of 5 and 9 cleared by hand, the pair (5, 9) is
    EMPTY in round 0; round 1 runs (20-21 merges) and, although 5's and 9's
    round-1 CubeSketches hold their edge, both report EMPTY again, so they
    stay apart.  Sampling them anew would join them."""
    V = 64
    u = np.array([5, 20], np.uint32)
    v = np.array([9, 21], np.uint32)
    A, G = oracle.ingest(V, 3, u, v)
    A[[5, 9], 0] = 0
    G[[5, 9], 0] = 0
    res = oracle.boruvka(V, 3, A, G)
    assert res["rounds"] == 2
    assert res["samples"][0][5] == -1 and res["samples"][0][9] == -1
    assert res["samples"][1][5] == -1 and res["samples"][1][9] == -1
    assert res["labels"][9] == 9 and res["labels"][21] == 20
    # untouched sketches: every component found, 5-9 joined in round 0
    A, G = oracle.ingest(V, 3, u, v)
    res = oracle.boruvka(V, 3, A, G)
    assert res["labels"][9] == 5 and res["labels"][21] == 20


def test_xor_of_every_node_sketch_is_zero():
    """Every edge index lands in the same bucket of both endpoints' sketches
    (depth and checksum depend on the index and the column only), so the XOR
    of all node sketches is zero for any stream; the query merges a component
    of more than V/2 members as the XOR of the nodes outside it."""
    V = 300
    u, v = S.random_stream(V, 5000, seed=17, n_distinct=2000)
    A, G = oracle.ingest(V, 8, u, v)
    assert np.any(A) and np.any(G)
    assert not np.any(np.bitwise_xor.reduce(A, axis=0))
    assert not np.any(np.bitwise_xor.reduce(G, axis=0))
    # and a strict subset's XOR equals its complement's
    inside = np.arange(V) < 200
    assert np.array_equal(np.bitwise_xor.reduce(A[inside], axis=0), np.bitwise_xor.reduce(A[~inside], axis=0))
