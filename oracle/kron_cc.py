"""Exact connected components of a large seeded Kronecker graph -- TEST /
MEASUREMENT INFRASTRUCTURE ONLY (ground truth for the sketch-failure study).

Brute-force union-find over every final edge (the check of Section 6.3) costs
O(V^2) predicate evaluations and ~3e9 edges at V = 2^17.  The same components
follow exactly from far fewer edges:

  * hubs H = the `n_hubs` vertices with the fewest one bits (the largest
    expected degree under the Graph500 initiator), ties by id;
  * E_H = every final edge inside H, and C = the largest connected component
    of (H, E_H) (the core);
  * for each vertex x outside C with a final edge into C, one such edge;
  * for each remaining vertex x (no edge into C), every final edge of x.

The union of these edge sets has exactly the components of the final graph:
C is connected through E_H, a vertex adjacent to C lies in C's component, and
every edge of every other vertex is listed.
"""
from __future__ import annotations

import numpy as np

from . import cc_edges


def kron_components(spec, n_hubs: int = 1024, block: int = 1 << 22) -> np.ndarray:
    V = spec.V
    n_hubs = min(n_hubs, V)
    ids = np.arange(V, dtype=np.uint64)
    pop = np.bitwise_count(ids).astype(np.int64)
    order = np.lexsort((ids, pop))
    hubs = np.sort(order[:n_hubs]).astype(np.uint64)

    eu, ev = [], []
    # edges inside the hub set; the core is their largest component
    a, b = np.triu_indices(n_hubs, 1)
    hu, hv = hubs[a], hubs[b]
    f = spec.final(hu, hv)
    hub_u, hub_v = hu[f], hv[f]
    lab = cc_edges(V, hub_u.astype(np.uint32), hub_v.astype(np.uint32))
    roots, counts = np.unique(lab[hubs], return_counts=True)
    core = hubs[lab[hubs] == roots[np.argmax(counts)]]
    in_core = np.zeros(V, bool)
    in_core[core] = True
    eu.append(hub_u)
    ev.append(hub_v)

    # one core edge per other vertex, where one exists
    others = np.nonzero(~in_core)[0].astype(np.uint64)
    nc = len(core)
    rows = max(1, block // nc)
    lonely = []
    for s in range(0, len(others), rows):
        xs = others[s:s + rows]
        X = np.repeat(xs, nc)
        Y = np.tile(core, len(xs))
        fin = (spec.final(X, Y) & (X != Y)).reshape(len(xs), nc)
        has = fin.any(axis=1)
        first = fin.argmax(axis=1)
        eu.append(xs[has])
        ev.append(core[first[has]])
        lonely.append(xs[~has])

    # every edge of the vertices without a core neighbour
    for x in np.concatenate(lonely):
        nb = spec.node_neighbors(int(x)).astype(np.uint64)
        eu.append(np.full(len(nb), x, np.uint64))
        ev.append(nb)

    u = np.concatenate(eu).astype(np.uint32)
    v = np.concatenate(ev).astype(np.uint32)
    return cc_edges(V, u, v)
