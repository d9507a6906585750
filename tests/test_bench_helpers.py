"""Host-side helpers of bench.py (no GPU)."""
import numpy as np
import torch

import bench


def test_wide_index_fraction_counts_indices_of_2p32_or_more():
    rng = np.random.default_rng(5)
    for V in (1000, 65536, 65537, 70001, 1 << 17):
        u = rng.integers(0, V, 5000)
        v = (u + 1 + rng.integers(0, V - 1, 5000)) % V
        want = np.mean([min(a, b) * V + max(a, b) >= 1 << 32 for a, b in zip(u.tolist(), v.tolist())])
        got = bench.wide_index_fraction(torch.from_numpy(u.astype(np.int32)), torch.from_numpy(v.astype(np.int32)),
                                        V, torch, block=777)
        assert got == want, V


def test_wide_segment_fraction_counts_records_of_high_nodes():
    # the batched kernel's 64-bit column code runs on every record of a node
    # x >= floor((2^32 - V) / V) + 1; each update has two records
    rng = np.random.default_rng(6)
    for V in (1000, 65536, 70001, 1 << 17):
        u = rng.integers(0, V, 4000)
        v = (u + 1 + rng.integers(0, V - 1, 4000)) % V
        xn = ((1 << 32) - V) // V + 1
        want = 0.0
        if V * V > 1 << 32:
            # a node of a record can hold an index of 2^32 or more iff its
            # largest possible index x*V + V-1 reaches 2^32
            want = np.mean([x * V + V - 1 >= 1 << 32 for x in np.concatenate([u, v]).tolist()])
        got = bench.wide_segment_fraction(torch.from_numpy(u.astype(np.int32)),
                                          torch.from_numpy(v.astype(np.int32)), V, torch, block=555)
        assert abs(got - want) < 1e-12, V


def test_serve_schedule_orders_each_graph_and_closes_it_last():
    # two synthetic graphs: cut points of their update chunks
    graphs = [{"cuts": [10, 25, 40]}, {"cuts": [7]}]
    ev = bench.serve_schedule(graphs, 2.0)
    assert [e[0] for e in ev] == sorted(e[0] for e in ev)
    for gi, g in enumerate(graphs):
        mine = [e for e in ev if e[1] == gi]
        ups = [(e[3], e[4]) for e in mine if e[2] == "u"]
        assert ups == list(zip([0] + g["cuts"][:-1], g["cuts"]))  # chunks in order, covering the stream
        assert mine[-1][2] == "close" and mine[-2][2] == "q"      # a final query, then the close
    assert bench.serve_schedule(graphs, 2.0) == ev                 # seeded
