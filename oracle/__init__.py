"""CPU oracle for the GraphZeppelin hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded restatement (``gz_oracle.c``) of CubeSketch
ingestion (Fig. cube_code, Eq. 1-2) and Boruvka connected components over node
sketches (Section 2.2; Lemma (CC I/O) proof), plus brute-force connected
components of the net graph (the adjacency-bit-vector check of Section 6.3).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline /
reference leg may import this package.  It shares no code with the CUDA
library in ``paper_2203_14927_b300``; both follow the same written definitions.
Parity pins for every function live in ``tests/test_oracle.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gz_oracle.c")
_SRC_BATCHED = os.path.join(_HERE, "gz_cpu_batched.c")
_SRC_L0 = os.path.join(_HERE, "gz_oracle_l0.c")
_LIB = os.path.join(_HERE, "libgz_oracle.so")

COLS = 7
EMPTY = -1
FAIL = -2
NOT_ROOT = -3
NOT_RUN = -4


def build(force: bool = False) -> str:
    """Compile gz_oracle.c (and the paper-design CPU baseline gz_cpu_batched.c,
    OpenMP) into libgz_oracle.so (plain gcc, -O2)."""
    srcs = [_SRC, _SRC_L0, _SRC_BATCHED]
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(s) for s in srcs):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fopenmp", "-shared",
                               "-fPIC", "-o", tmp, *srcs])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        u64, u32, sz, p = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_size_t, ctypes.c_void_p
        L.gzo_splitmix64_at.restype = u64
        L.gzo_splitmix64_at.argtypes = [u64, u64]
        L.gzo_h1.restype = u64
        L.gzo_h1.argtypes = [u32, p, u64]
        L.gzo_h2.restype = u32
        L.gzo_h2.argtypes = [u32, p, u64]
        L.gzo_pieces.restype = None
        L.gzo_pieces.argtypes = [u32, p, p, p]
        L.gzo_geometry.restype = ctypes.c_int
        L.gzo_geometry.argtypes = [u32, p, p]
        L.gzo_keys.restype = None
        L.gzo_keys.argtypes = [u64, u32, p]
        L.gzo_ingest.restype = ctypes.c_int
        L.gzo_ingest.argtypes = [u32, u64, sz, p, p, p, p]
        L.gzo_sketch_node.restype = ctypes.c_int
        L.gzo_sketch_node.argtypes = [u32, u64, u32, sz, p, p, p]
        L.gzo_query_vector.restype = ctypes.c_int64
        L.gzo_query_vector.argtypes = [u32, u64, u32, p, p]
        L.gzo_boruvka.restype = ctypes.c_int
        L.gzo_boruvka.argtypes = [u32, u64, p, p, p, p, p, p, p]
        L.gzo_brute_cc.restype = ctypes.c_int
        L.gzo_brute_cc.argtypes = [u32, sz, p, p, p]
        L.gzo_cc_edges.restype = ctypes.c_int
        L.gzo_cc_edges.argtypes = [u32, sz, p, p, p]
        L.gzo_l0_rows.restype = u32
        L.gzo_l0_rows.argtypes = [u64]
        L.gzo_mulmod61.restype = u64
        L.gzo_mulmod61.argtypes = [u64, u64]
        L.gzo_powmod61.restype = u64
        L.gzo_powmod61.argtypes = [u64, u64]
        L.gzo_l0_update.restype = ctypes.c_int
        L.gzo_l0_update.argtypes = [ctypes.c_int, u64, u64, sz, p, p, p]
        L.gzo_l0_query.restype = ctypes.c_int64
        L.gzo_l0_query.argtypes = [ctypes.c_int, u64, u64, p, p]
        L.gzb_ingest_batched.restype = ctypes.c_int
        L.gzb_ingest_batched.argtypes = [u32, u64, sz, p, p, u32, u32, p, p, ctypes.c_int, sz]
        L.gzb_max_threads.restype = ctypes.c_int
        L.gzb_max_threads.argtypes = []
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def geometry(V: int) -> tuple[int, int]:
    """(K, R): CubeSketches per node and rows per column."""
    K = np.zeros(1, np.uint32)
    R = np.zeros(1, np.uint32)
    if lib().gzo_geometry(V, _ptr(K), _ptr(R)) != 0:
        raise ValueError(f"V={V} must be >= 2")
    return int(K[0]), int(R[0])


KEY_WORDS = 256  # 32-bit key words per column: h1 pieces at [0, 128), h2 pieces at [128, 256)


def keys(seed: int, K: int) -> np.ndarray:
    """Hash keys of the 7K columns: a (7K, 256) uint32 array, row col holding
    the h1 pieces' keys in [0, 128) and the h2 pieces' keys in [128, 256)."""
    k = np.zeros((K * COLS, KEY_WORDS), np.uint32)
    lib().gzo_keys(seed, K, _ptr(k))
    return k


def pieces(V: int) -> tuple[int, int, int]:
    """(p, m1, m2): piece width 33 - ceil(log2 V) and the pieces of h1 and h2."""
    out = np.zeros(3, np.uint32)
    lib().gzo_pieces(V, _ptr(out[0:]), _ptr(out[1:]), _ptr(out[2:]))
    return int(out[0]), int(out[1]), int(out[2])


def splitmix64_at(seed: int, n: int) -> int:
    return int(lib().gzo_splitmix64_at(seed, n))


def h1(V: int, kcol, e: int) -> int:
    """col_hash of edge index e (u < v < V) under the keys of one column (a row
    of keys()): bit i is the i-th bit of H1 from its most significant end."""
    k = np.ascontiguousarray(kcol, np.uint32)
    return int(lib().gzo_h1(V, _ptr(k), e))


def h2(V: int, kcol, e: int) -> int:
    """Checksum of edge index e (u < v < V) under the keys of one column."""
    k = np.ascontiguousarray(kcol[128:], np.uint32)
    return int(lib().gzo_h2(V, _ptr(k), e))


def empty_sketches(V: int, nodes: int | None = None):
    """Zeroed nested-form sketches for `nodes` nodes (default V):
    alpha[node][k][j][row] u64 and gamma[node][k][j][row] u32."""
    K, R = geometry(V)
    n = V if nodes is None else nodes
    return (np.zeros((n, K, COLS, R), np.uint64), np.zeros((n, K, COLS, R), np.uint32))


def ingest_batched(V: int, seed: int, u, v, node_lo: int = 0, node_hi: int | None = None,
                   threads: int = 0, chunk: int = 1 << 22):
    """The paper's CPU design (per-node buffers applied by parallel workers,
    Section 5.1) over the stream (u, v), sketching nodes [node_lo, node_hi)
    only; nested form like ingest().  A timed baseline, not the oracle."""
    node_hi = V if node_hi is None else node_hi
    u = np.ascontiguousarray(u, np.uint32)
    v = np.ascontiguousarray(v, np.uint32)
    alpha, gamma = empty_sketches(V, node_hi - node_lo)
    rc = lib().gzb_ingest_batched(V, seed, len(u), _ptr(u), _ptr(v), node_lo, node_hi,
                                  _ptr(alpha), _ptr(gamma), threads, chunk)
    if rc != 0:
        raise ValueError(f"gzb_ingest_batched failed ({rc})")
    return alpha, gamma


# ---- single-vector l0 sketches (Fig. agm_code standard sampler, Fig. cube_code)

L0_CUBE, L0_STANDARD = 0, 1
P61 = (1 << 61) - 1


def l0_rows(n: int) -> int:
    return int(lib().gzo_l0_rows(n))


def l0_bytes(kind: int, n: int) -> int:
    """Bytes of one vector sketch: CubeSketch 7R x 12 padded to a multiple of 8
    (trailing zero bytes), standard 7R x 24."""
    R = l0_rows(n)
    return (84 * R + 7) // 8 * 8 if kind == L0_CUBE else 168 * R


def mulmod61(x: int, y: int) -> int:
    return int(lib().gzo_mulmod61(x, y))


def powmod61(r: int, e: int) -> int:
    return int(lib().gzo_powmod61(r, e))


def l0_update(kind: int, n: int, seed: int, x, delta=None, buckets=None) -> np.ndarray:
    """Apply updates (x[i], delta[i] = +-1) to one vector sketch; returns its
    bytes (a fresh zero sketch when buckets is None)."""
    x = np.ascontiguousarray(x, np.uint64)
    if buckets is None:
        buckets = np.zeros(l0_bytes(kind, n), np.uint8)
    dptr = None
    if delta is not None:
        delta = np.ascontiguousarray(delta, np.int32)
        dptr = _ptr(delta)
    rc = lib().gzo_l0_update(kind, n, seed, len(x), _ptr(x), dptr, _ptr(buckets))
    if rc != 0:
        raise ValueError("invalid l0 update")
    return buckets


def l0_query(kind: int, n: int, seed: int, buckets: np.ndarray):
    """(position, value) sampled from one vector sketch; position -1 = EMPTY,
    -2 = FAIL."""
    val = np.zeros(1, np.int64)
    pos = int(lib().gzo_l0_query(kind, n, seed, _ptr(buckets), _ptr(val)))
    return pos, int(val[0])


def max_threads() -> int:
    return int(lib().gzb_max_threads())


def ingest(V: int, seed: int, u, v, alpha=None, gamma=None):
    """Apply the stream (u[i], v[i]) to all V node sketches (nested form)."""
    u = np.ascontiguousarray(u, np.uint32)
    v = np.ascontiguousarray(v, np.uint32)
    if alpha is None:
        alpha, gamma = empty_sketches(V)
    rc = lib().gzo_ingest(V, seed, len(u), _ptr(u), _ptr(v), _ptr(alpha), _ptr(gamma))
    if rc != 0:
        raise ValueError(f"gzo_ingest returned {rc}")
    return alpha, gamma


def sketch_node(V: int, seed: int, node: int, nbrs):
    """Nested-form sketch of one node from its net neighbour list."""
    K, R = geometry(V)
    nbrs = np.ascontiguousarray(nbrs, np.uint32)
    a = np.zeros((K, COLS, R), np.uint64)
    g = np.zeros((K, COLS, R), np.uint32)
    rc = lib().gzo_sketch_node(V, seed, node, len(nbrs), _ptr(nbrs), _ptr(a), _ptr(g))
    if rc != 0:
        raise ValueError(f"gzo_sketch_node returned {rc}")
    return a, g


def query_vector(V: int, seed: int, k: int, A, G) -> int:
    """query_sketch of Fig. cube_code on one CubeSketch ([j][row] arrays)."""
    A = np.ascontiguousarray(A, np.uint64)
    G = np.ascontiguousarray(G, np.uint32)
    return int(lib().gzo_query_vector(V, seed, k, _ptr(A), _ptr(G)))


def boruvka(V: int, seed: int, alpha, gamma):
    """Boruvka over node sketches.  Returns a dict with labels (min vertex id
    per component), forest (n,2) in acceptance order, samples (K,V) per
    round and component, stats and the return code (1 = possible failure)."""
    K, _ = geometry(V)
    labels = np.zeros(V, np.uint32)
    forest = np.zeros(2 * max(V - 1, 1), np.uint32)
    nf = np.zeros(1, np.uint64)
    samples = np.zeros(K * V, np.int64)
    stats = np.zeros(4, np.uint64)
    rc = lib().gzo_boruvka(V, seed, _ptr(alpha), _ptr(gamma), _ptr(labels), _ptr(forest),
                           _ptr(nf), _ptr(samples), _ptr(stats))
    if rc < 0:
        raise ValueError(f"gzo_boruvka returned {rc}")
    n = int(nf[0])
    return {
        "labels": labels,
        "forest": forest[: 2 * n].reshape(n, 2).copy(),
        "samples": samples.reshape(K, V),
        "rounds": int(stats[0]),
        "fails_last": int(stats[1]),
        "exhausted": int(stats[2]),
        "n_components": int(stats[3]),
        "rc": rc,
    }


def brute_cc(V: int, u, v) -> np.ndarray:
    """Min-id component labels of the net graph of the stream (bit vector)."""
    u = np.ascontiguousarray(u, np.uint32)
    v = np.ascontiguousarray(v, np.uint32)
    labels = np.zeros(V, np.uint32)
    rc = lib().gzo_brute_cc(V, len(u), _ptr(u), _ptr(v), _ptr(labels))
    if rc != 0:
        raise ValueError(f"gzo_brute_cc returned {rc}")
    return labels


def cc_edges(V: int, u, v) -> np.ndarray:
    """Min-id component labels of the graph with the given edge list."""
    u = np.ascontiguousarray(u, np.uint32)
    v = np.ascontiguousarray(v, np.uint32)
    labels = np.zeros(V, np.uint32)
    rc = lib().gzo_cc_edges(V, len(u), _ptr(u), _ptr(v), _ptr(labels))
    if rc != 0:
        raise ValueError(f"gzo_cc_edges returned {rc}")
    return labels


def to_exact(alpha_nested: np.ndarray) -> np.ndarray:
    """Nested rows -> exact-depth rows (row i XOR row i+1): the inverse of the
    suffix-XOR that defines the nested form; used by tests only."""
    out = alpha_nested.copy()
    out[..., :-1] ^= alpha_nested[..., 1:]
    return out
