"""Seeded synthetic graph streams (inputs only: no sketch arithmetic here).

The paper evaluates on Graph500 Kronecker graphs turned into insert/delete
streams (Section 6.1, "Synthesizing Dense Graphs and Streams"; Table
tab:datasets) and on four public graphs that are not available here.  This
module stands in for both with counter-based generators, so that the same
stream can be produced on the host (numpy, this file) and on the device
(``gz_gen_kron_chunk`` in the CUDA library) and compared bit for bit.

Kronecker stream (V = 2^L):
  * edge probability of an unordered pair u < v is the stochastic-Kronecker
    product  p(u,v) = min(1, s * a^n00 * b^(n01+n10) * d^n11)  with the
    Graph500 initiator (a, b, b, d) = (0.57, 0.19, 0.19, 0.05), where nXY
    counts the bit positions with (u_bit, v_bit) = (X, Y);  s is solved so that
    the expected edge count hits the target (closed form over bit-pair counts);
  * the pair is an edge iff  mix64(idx ^ k_kron) >> 11  <  floor(p * 2^53),
    idx = u*V + v, so self loops and duplicates cannot occur (the paper prunes
    them);  the thresholds are a host-computed table T53[n00][n11];
  * rule (iii): nodes with  mix64(x ^ k_iso) >> 11 < floor(n_iso/V * 2^53)
    lose all their final edges;
  * churn: a non-final pair is inserted and later deleted iff
    mix64(idx ^ k_churn) >> 11 < floor(q * 2^53), q set so that the expected
    number of churn pairs is `churn` times the expected edge count;
  * order: positions 0..V^2-1 are mapped to ordered pairs by a 4-round
    Feistel permutation on the two L-bit halves; slice c covers positions
    [c*P, (c+1)*P); chunk c holds, in position order, the inserts of slice c
    followed by the deletes of the churn pairs of slice c-1, so every insert
    precedes its delete and updates of one edge alternate (rules (i), (ii));
    chunk S (S = number of slices) holds only the last deletes (rule (iv)).

mix64 is the SplitMix64 output function (Steele, Lea & Flood 2014).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1
THETA = (0.57, 0.19, 0.19, 0.05)

TAG_KRON, TAG_CHURN, TAG_ISO, TAG_FEISTEL = 1, 2, 3, 4  # Feistel uses 4..7


def mix64(z):
    """SplitMix64 output function on uint64 numpy arrays (wrapping)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def mix64_int(z: int) -> int:
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def tag_key(seed: int, tag: int) -> int:
    """Per-purpose 64-bit key: the tag-th SplitMix64 output from `seed`."""
    return mix64_int((seed + (tag + 1) * GOLDEN) & M64)


def u53(key: int, x) -> np.ndarray:
    """53 uniform bits of x under `key`."""
    return mix64(np.asarray(x, np.uint64) ^ np.uint64(key)) >> np.uint64(11)


def thresh53(p: float) -> int:
    """floor(min(max(p,0),1) * 2^53): x < thresh53(p) has probability p."""
    p = min(max(p, 0.0), 1.0)
    return int(math.floor(p * (1 << 53)))


# --------------------------------------------------------------------- Kronecker


def _kron_expected_edges(L: int, s: float, theta=THETA) -> float:
    """Expected number of unordered pairs u < v that are edges."""
    a, b, _, d = theta
    fact = math.factorial
    total = 0.0
    for n00 in range(L + 1):
        for n11 in range(L + 1 - n00):
            nx = L - n00 - n11
            mult = fact(L) // (fact(n00) * fact(nx) * fact(n11)) * (1 << nx)
            total += mult * min(1.0, s * a ** n00 * b ** nx * d ** n11)
    diag = sum(math.comb(L, n11) * min(1.0, s * a ** (L - n11) * d ** n11) for n11 in range(L + 1))
    return (total - diag) / 2.0


def kron_scale(L: int, target_edges: float, theta=THETA) -> float:
    """Solve s by bisection (on log s) so that the expected edge count is
    `target_edges`."""
    pairs = (1 << L) * ((1 << L) - 1) / 2
    if not 0 < target_edges < pairs:
        raise ValueError("target_edges must lie in (0, C(V,2))")
    lo, hi = -10.0, 200.0
    for _ in range(200):
        mid = (lo + hi) / 2
        if _kron_expected_edges(L, math.exp(mid), theta) < target_edges:
            lo = mid
        else:
            hi = mid
    return math.exp((lo + hi) / 2)


@dataclass(frozen=True)
class KronSpec:
    """A seeded Kronecker insert/delete stream on V = 2^L nodes."""

    L: int
    seed: int
    target_edges: float
    churn: float = 0.1
    n_iso: float = 100.0
    slice_log2: int = 26
    theta: tuple = THETA
    _d: dict = field(default_factory=dict, compare=False, repr=False)

    @property
    def V(self) -> int:
        return 1 << self.L

    def _derived(self) -> dict:
        if not self._d:
            L = self.L
            s = kron_scale(L, self.target_edges, self.theta)
            a, b, _, d = self.theta
            T = np.zeros((L + 1, L + 1), np.uint64)
            for n00 in range(L + 1):
                for n11 in range(L + 1 - n00):
                    nx = L - n00 - n11
                    T[n00, n11] = thresh53(s * a ** n00 * b ** nx * d ** n11)
            pairs = self.V * (self.V - 1) / 2
            q = self.churn * self.target_edges / max(pairs - self.target_edges, 1.0)
            self._d.update(
                s=s,
                table=T,
                t_iso=thresh53(self.n_iso / self.V),
                t_churn=thresh53(q),
                k_kron=tag_key(self.seed, TAG_KRON),
                k_churn=tag_key(self.seed, TAG_CHURN),
                k_iso=tag_key(self.seed, TAG_ISO),
                k_feistel=tuple(tag_key(self.seed, TAG_FEISTEL + i) for i in range(4)),
            )
        return self._d

    @property
    def n_slices(self) -> int:
        return max(1, (self.V * self.V) >> self.slice_log2)

    @property
    def n_chunks(self) -> int:
        return self.n_slices + 1

    @property
    def slice_len(self) -> int:
        return min(1 << self.slice_log2, self.V * self.V)

    def device_params(self) -> dict:
        """Everything the device generator needs (same values as used here)."""
        d = self._derived()
        return {
            "L": self.L,
            "slice_log2": int(math.log2(self.slice_len)),
            "k_feistel": d["k_feistel"],
            "k_kron": d["k_kron"],
            "k_churn": d["k_churn"],
            "k_iso": d["k_iso"],
            "t_iso": d["t_iso"],
            "t_churn": d["t_churn"],
            "table": d["table"].reshape(-1).copy(),
        }

    # -- pair predicates ---------------------------------------------------

    def isolated(self, x) -> np.ndarray:
        d = self._derived()
        return u53(d["k_iso"], x) < np.uint64(d["t_iso"])

    def kron(self, u, v) -> np.ndarray:
        d = self._derived()
        u = np.asarray(u, np.uint64)
        v = np.asarray(v, np.uint64)
        n11 = np.bitwise_count(u & v).astype(np.int64)
        n00 = self.L - np.bitwise_count(u | v).astype(np.int64)
        idx = np.minimum(u, v) * np.uint64(self.V) + np.maximum(u, v)
        return u53(d["k_kron"], idx) < d["table"][n00, n11]

    def final(self, u, v) -> np.ndarray:
        """Edge of the final graph (u != v)."""
        return self.kron(u, v) & ~self.isolated(u) & ~self.isolated(v)

    def churn_pair(self, u, v) -> np.ndarray:
        """Non-final pair that is inserted and later deleted."""
        d = self._derived()
        u = np.asarray(u, np.uint64)
        v = np.asarray(v, np.uint64)
        idx = np.minimum(u, v) * np.uint64(self.V) + np.maximum(u, v)
        return ~self.final(u, v) & (u53(d["k_churn"], idx) < np.uint64(d["t_churn"]))

    # -- order --------------------------------------------------------------

    def position_pairs(self, pos):
        """Feistel permutation of positions in [0, V^2) to ordered pairs."""
        d = self._derived()
        L = np.uint64(self.L)
        M = np.uint64(self.V - 1)
        pos = np.asarray(pos, np.uint64)
        left, right = pos >> L, pos & M
        for k in d["k_feistel"]:
            left, right = right, left ^ (mix64(right ^ np.uint64(k)) & M)
        return left, right

    def chunk(self, c: int):
        """Updates of chunk c (0 <= c <= n_slices) as (u, v) uint32 with u < v."""
        if not 0 <= c < self.n_chunks:
            raise IndexError(c)
        P = self.slice_len
        parts_u, parts_v = [], []
        if c < self.n_slices:
            u, v = self.position_pairs(np.arange(c * P, (c + 1) * P, dtype=np.uint64))
            m = u < v
            u, v = u[m], v[m]
            keep = self.final(u, v) | self.churn_pair(u, v)
            parts_u.append(u[keep])
            parts_v.append(v[keep])
        if c >= 1:
            u, v = self.position_pairs(np.arange((c - 1) * P, c * P, dtype=np.uint64))
            m = u < v
            u, v = u[m], v[m]
            keep = self.churn_pair(u, v)
            parts_u.append(u[keep])
            parts_v.append(v[keep])
        return (np.concatenate(parts_u).astype(np.uint32), np.concatenate(parts_v).astype(np.uint32))

    def stream(self):
        """The whole stream (small V only)."""
        us, vs = zip(*(self.chunk(c) for c in range(self.n_chunks)))
        return np.concatenate(us), np.concatenate(vs)

    def node_neighbors(self, x: int) -> np.ndarray:
        """Net neighbours of node x in the final graph, ascending."""
        y = np.arange(self.V, dtype=np.uint64)
        y = y[y != x]
        xs = np.full(y.shape, x, np.uint64)
        return y[self.final(xs, y)].astype(np.uint32)

    def final_edges(self, block: int = 1 << 22):
        """All final edges (u < v), small V only."""
        us, vs = [], []
        V = self.V
        for start in range(0, V * V, block):
            idx = np.arange(start, min(start + block, V * V), dtype=np.uint64)
            u, v = idx // np.uint64(V), idx % np.uint64(V)
            m = u < v
            u, v = u[m], v[m]
            f = self.final(u, v)
            us.append(u[f])
            vs.append(v[f])
        return np.concatenate(us).astype(np.uint32), np.concatenate(vs).astype(np.uint32)


def kron_for_updates(L: int, seed: int, n_updates: float, churn: float = 0.1,
                     chunk_updates: float = 2 ** 24, n_iso: float = 100.0) -> KronSpec:
    """Kronecker spec whose stream has about `n_updates` updates (final edges
    plus twice the churn pairs) and about `chunk_updates` updates per chunk."""
    target = n_updates / (1.0 + 2.0 * churn)
    per_pos = n_updates / float(1 << (2 * L))
    slice_log2 = int(round(math.log2(max(chunk_updates / per_pos, 1.0))))
    slice_log2 = max(10, min(slice_log2, 2 * L))
    return KronSpec(L=L, seed=seed, target_edges=target, churn=churn, n_iso=n_iso,
                    slice_log2=slice_log2)


# --------------------------------------------------------------------- planted G(n,p)


@dataclass(frozen=True)
class PlantedSpec:
    """`n_comp` planted components, each G(n_i, p); `extra` * |E| additional
    pairs (from all non-final pairs) are each toggled in `cycles` insert/delete
    cycles; the whole stream is shuffled with a seeded permutation."""

    V: int = 1024
    seed: int = 1
    n_comp: int = 8
    p: float = 0.1
    extra: float = 0.2
    cycles: int = 1


def planted_stream(spec: PlantedSpec):
    """Returns (u, v, comp): the update stream (uint32, random orientation)
    and the planted component of every node."""
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    V, C = spec.V, spec.n_comp
    w = rng.random(C) + 0.5
    sizes = np.maximum(2, np.floor(w / w.sum() * V).astype(np.int64))
    sizes[-1] = V - sizes[:-1].sum()
    perm = rng.permutation(V)
    comp = np.empty(V, np.int64)
    start = 0
    fu, fv = [], []
    for i, sz in enumerate(sizes):
        nodes = np.sort(perm[start:start + sz])
        comp[nodes] = i
        start += sz
        a, b = np.triu_indices(sz, 1)
        keep = rng.random(len(a)) < spec.p
        fu.append(nodes[a[keep]])
        fv.append(nodes[b[keep]])
    fu = np.concatenate(fu)
    fv = np.concatenate(fv)
    final_idx = set((fu * V + fv).tolist())
    n_extra = int(round(spec.extra * len(fu)))
    eu, ev = [], []
    seen = set()
    while len(eu) < n_extra:
        a, b = rng.integers(0, V, 2)
        if a == b:
            continue
        lo, hi = (a, b) if a < b else (b, a)
        key = int(lo) * V + int(hi)
        if key in final_idx or key in seen:
            continue
        seen.add(key)
        eu.append(lo)
        ev.append(hi)
    eu = np.asarray(eu, np.int64)
    ev = np.asarray(ev, np.int64)
    u = np.concatenate([fu] + [eu] * (2 * spec.cycles))
    v = np.concatenate([fv] + [ev] * (2 * spec.cycles))
    order = rng.permutation(len(u))
    u, v = u[order], v[order]
    flip = rng.random(len(u)) < 0.5
    u2 = np.where(flip, v, u)
    v2 = np.where(flip, u, v)
    return u2.astype(np.uint32), v2.astype(np.uint32), comp


def planted_sparse_stream(V: int, seed: int, n_updates: int, n_comp: int = 8, churn: float = 0.1):
    """Planted components at any scale: the final edges are uniform random
    pairs inside n_comp equal-ish components (G(n_i, p) with p set by the
    update budget), churn pairs are uniform over all pairs (inserted, later
    deleted); seeded shuffle.  Returns (u, v) uint32 and the component map."""
    rng = np.random.Generator(np.random.PCG64(seed))
    comp = rng.integers(0, n_comp, V)
    n_final = int(n_updates / (1 + 2 * churn))
    n_churn = int(n_final * churn)
    fu, fv = [], []
    for c in range(n_comp):
        nodes = np.nonzero(comp == c)[0]
        if len(nodes) < 2:
            continue
        m = int(n_final * len(nodes) / V * 1.05) + 1
        a = nodes[rng.integers(0, len(nodes), m)]
        b = nodes[rng.integers(0, len(nodes), m)]
        keep = a != b
        fu.append(np.minimum(a, b)[keep])
        fv.append(np.maximum(a, b)[keep])
    fu = np.concatenate(fu).astype(np.uint64)
    fv = np.concatenate(fv).astype(np.uint64)
    idx = np.unique(fu * np.uint64(V) + fv)[:n_final]
    a = rng.integers(0, V, n_churn).astype(np.uint64)
    b = rng.integers(0, V, n_churn).astype(np.uint64)
    keep = a != b
    cidx = np.unique(np.minimum(a, b)[keep] * np.uint64(V) + np.maximum(a, b)[keep])
    cidx = np.setdiff1d(cidx, idx, assume_unique=True)
    all_idx = np.concatenate([idx, cidx, cidx])
    all_idx = all_idx[rng.permutation(len(all_idx))]
    return ((all_idx // np.uint64(V)).astype(np.uint32), (all_idx % np.uint64(V)).astype(np.uint32), comp)


def random_stream(V: int, n: int, seed: int, n_distinct: int | None = None):
    """n updates over `n_distinct` random pairs (repeats toggle), any V >= 2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = n_distinct if n_distinct is not None else max(1, n // 2)
    a = rng.integers(0, V, m)
    b = rng.integers(0, V - 1, m)
    b = np.where(b >= a, b + 1, b)
    pick = rng.integers(0, m, n)
    return a[pick].astype(np.uint32), b[pick].astype(np.uint32)


def hub_stream(V: int, n: int, seed: int, hubs):
    """n updates (about): half `random_stream` pairs (repeats toggle), half
    with one endpoint drawn from `hubs` and the other uniform, shuffled; the
    hubs' node segments span many record tiles."""
    hubs = np.asarray(hubs, np.uint32)
    u1, v1 = random_stream(V, n // 2, seed=seed, n_distinct=n // 3)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    hu = hubs[rng.integers(0, len(hubs), n - n // 2)]
    hv = rng.integers(0, V, n - n // 2).astype(np.uint32)
    keep = hu != hv
    u = np.concatenate([u1, hu[keep]])
    v = np.concatenate([v1, hv[keep]])
    perm = rng.permutation(len(u))
    return u[perm], v[perm]


def net_graph(V: int, u, v):
    """Edges with an odd number of updates, as (u, v) with u < v, ascending idx."""
    u = np.asarray(u, np.uint64)
    v = np.asarray(v, np.uint64)
    idx = np.minimum(u, v) * np.uint64(V) + np.maximum(u, v)
    vals, counts = np.unique(idx, return_counts=True)
    odd = vals[counts % 2 == 1]
    return (odd // np.uint64(V)).astype(np.uint32), (odd % np.uint64(V)).astype(np.uint32)


def neighbors_from_edges(V: int, eu, ev, x: int) -> np.ndarray:
    eu = np.asarray(eu)
    ev = np.asarray(ev)
    return np.sort(np.concatenate([ev[eu == x], eu[ev == x]])).astype(np.uint32)
