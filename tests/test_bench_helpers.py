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
