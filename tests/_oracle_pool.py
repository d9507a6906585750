"""Oracle node sketches for many nodes at once (test helper).

The CPU oracle is single-threaded C.  Tests that check hundreds or thousands
of node sketches run it in a pool of threads, one node per task: the oracle
call releases the interpreter lock (ctypes), so the nodes are sketched on all
host cores.  The oracle itself is unchanged; each node is sketched from its
net neighbour list, which linearity makes equal to sketching the stream."""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle


def sketch_nodes(V: int, seed: int, nodes, neighbors, threads: int | None = None) -> dict:
    """{x: (alpha, gamma)} = oracle.sketch_node(V, seed, x, neighbors(x)) for
    every x in nodes (nested form, [k][j][row])."""
    threads = threads or os.cpu_count() or 1
    oracle.lib()  # build and load once, before the pool starts

    def one(x):
        return int(x), oracle.sketch_node(V, seed, int(x), neighbors(int(x)))

    with ThreadPoolExecutor(max_workers=threads) as ex:
        return dict(ex.map(one, list(nodes)))


def hubs(L: int) -> list[int]:
    """The vertices with the fewest one bits (0 and the powers of two): the
    largest expected degrees under the Graph500 initiator, whose first
    entry (0.57) belongs to the (0, 0) bit pair."""
    return [0] + [1 << i for i in range(L)]


def first_mismatch(a, b):
    """Index of the first node whose sketch differs, or None."""
    diff = np.nonzero((a != b).reshape(len(a), -1).any(axis=1))[0]
    return int(diff[0]) if len(diff) else None
