"""GPU path vs the CPU oracle at the benchmark sizes, in the benchmark's
launch configuration (autotune.DEFAULT: 2^26-update batches, 512-record tiles,
12 staged rows, shared-atomic deltas).

  * V = 2^13 Kronecker stream (~2e7 updates, 10% churn): every node sketch
    bit for bit, the per-round Boruvka samples, the spanning forest and the
    labels equal the oracle's.
  * V = 2^15 (~3e8 updates generated on the device): 256 seeded random nodes
    and every hub equal the oracle's; the plain per-update kernel gives the
    same device sketches as the batched kernel on the same stream, on every
    node; labels equal the exact components.
  * V = 2^17 (~4e9 updates, 64-bit edge indices): 256 random nodes and every
    hub; labels equal the exact components.
  * V = 2^20 (~8e9 updates, 123 GB of node sketches): 32 random nodes and
    a hub of three one bits; labels equal the exact components.

The oracle sketches single nodes from their net neighbour lists (linearity:
equal to sketching the stream), on all host cores (tests/_oracle_pool.py).
Sketches are integer XOR sums: equality is exact.
"""
import numpy as np
import pytest

import oracle
import paper_2203_14927_b300 as gz
from paper_2203_14927_b300 import streams as S

from _oracle_pool import first_mismatch, hubs, sketch_nodes

pytestmark = pytest.mark.gpu


def _device_stream(spec):
    """The whole stream of spec generated on the device: (u, v) int32 tensors."""
    import torch

    gen = gz.DeviceKronStream(spec)
    cap = int(spec.target_edges * (1 + 2 * spec.churn) * 1.08) + (1 << 26)
    U = torch.empty(cap, dtype=torch.int32, device="cuda")
    W = torch.empty(cap, dtype=torch.int32, device="cuda")
    n = 0
    for c in range(gen.n_chunks):
        n += gen.chunk_into(c, U.data_ptr() + 4 * n, W.data_ptr() + 4 * n, cap - n)
    gen.close()
    return U[:n], W[:n]


def _release():
    import torch

    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _check_sampled(g, spec, seed, nodes):
    ref = sketch_nodes(spec.V, seed, nodes, spec.node_neighbors)
    for x in nodes:
        a, gg = g.export_sketch(x, x + 1)
        A, G = ref[x]
        assert np.array_equal(a[0], A) and np.array_equal(gg[0], G), f"node {x}"


class _DeviceBytes:
    """A device byte range seen by torch (the library's raw sketch array)."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                         "version": 3}


def test_kron13_every_node_per_round_samples_and_forest():
    from paper_2203_14927_b300 import autotune

    seed = 77
    spec = S.kron_for_updates(13, 2024, 2.0e7, churn=0.1, chunk_updates=2 ** 24)
    U, W = _device_stream(spec)
    assert 1.7e7 < U.numel() < 2.3e7
    g = gz.Graph(spec.V, seed, **autotune.DEFAULT)
    g.edge_update(U, W)
    g.sync()
    a, gg = g.export_sketch()
    ref = sketch_nodes(spec.V, seed, range(spec.V), spec.node_neighbors)
    A = np.stack([ref[x][0] for x in range(spec.V)])
    G = np.stack([ref[x][1] for x in range(spec.V)])
    del ref
    assert first_mismatch(a, A) is None, f"alpha of node {first_mismatch(a, A)}"
    assert first_mismatch(gg, G) is None, f"gamma of node {first_mismatch(gg, G)}"
    want = oracle.boruvka(spec.V, seed, A, G)
    g.enable_trace(True)
    forest, labels, st = g.list_spanning_forest()
    assert np.array_equal(g.query_trace(), want["samples"])
    assert np.array_equal(forest, want["forest"])
    assert np.array_equal(labels, want["labels"])
    assert st["rounds"] == want["rounds"] and st["fails_last"] == want["fails_last"] == 0
    eu, ev = spec.final_edges()
    assert np.array_equal(labels, oracle.cc_edges(spec.V, eu, ev))
    g.close()
    _release()


def test_kron15_sampled_nodes_and_plain_kernel_on_the_same_stream():
    import torch

    from oracle.kron_cc import kron_components
    from paper_2203_14927_b300 import autotune

    seed = 15
    spec = S.kron_for_updates(15, 15, 3.0e8, churn=0.1, chunk_updates=2 ** 24)
    U, W = _device_stream(spec)
    assert 2.7e8 < U.numel() < 3.3e8
    g = gz.Graph(spec.V, seed, **autotune.DEFAULT)
    g.edge_update(U, W)
    g.sync()
    rng = np.random.default_rng(1515)
    nodes = sorted(set(rng.choice(spec.V, 256, replace=False).tolist()) | set(hubs(15)) | {spec.V - 1})
    _check_sampled(g, spec, seed, nodes)
    labels, ncc, st = g.connected_components()
    assert st["fails_last"] == 0 and st["exhausted"] == 0
    assert np.array_equal(labels, kron_components(spec))
    # the plain per-update kernel (the unbuffered baseline) on the same stream
    # leaves the same device sketches, node for node
    p = gz.Graph(spec.V, seed, kernel="plain", chunk_log2=26)
    p.edge_update(U, W)
    p.sync()
    ia, ip = g.info(), p.info()
    nbytes = spec.V * ia["node_bytes"]
    da = torch.as_tensor(_DeviceBytes(ia["sketch_ptr"], nbytes), device="cuda")
    dp = torch.as_tensor(_DeviceBytes(ip["sketch_ptr"], nbytes), device="cuda")
    assert torch.equal(da, dp)
    del da, dp, U, W
    p.close()
    g.close()
    _release()


def test_kron17_sampled_nodes_and_labels():
    # The benchmark's main workload at full size: V = 2^17 (64-bit edge
    # indices, so the kernel's wide record path), ~4e9 updates with 10% churn
    # generated on the device, ingested in one call.
    from oracle.kron_cc import kron_components
    from paper_2203_14927_b300 import autotune

    seed = 17
    spec = S.kron_for_updates(17, 17, 4.0e9, churn=0.1, chunk_updates=2 ** 24)
    U, W = _device_stream(spec)
    assert 3.6e9 < U.numel() < 4.4e9
    g = gz.Graph(spec.V, seed, **autotune.DEFAULT)
    g.edge_update(U, W)
    g.sync()
    del U, W
    _release()
    rng = np.random.default_rng(17)
    nodes = sorted(set(rng.choice(spec.V, 256, replace=False).tolist()) | set(hubs(17)) | {spec.V - 1})
    _check_sampled(g, spec, seed, nodes)
    labels, ncc, st = g.connected_components()
    assert st["fails_last"] == 0 and st["exhausted"] == 0
    assert np.array_equal(labels, kron_components(spec))
    g.close()
    _release()


def test_kron20_sampled_nodes_and_labels():
    # Beyond the paper's largest graph: V = 2^20, ~8e9 updates, 123 GB of
    # node sketches in HBM, 64-bit edge indices up to 2^40.
    from oracle.kron_cc import kron_components
    from paper_2203_14927_b300 import autotune

    seed = 20
    spec = S.kron_for_updates(20, 20, 8.0e9, churn=0.1, chunk_updates=2 ** 24)
    U, W = _device_stream(spec)
    assert 7.2e9 < U.numel() < 8.8e9
    g = gz.Graph(spec.V, seed, **autotune.DEFAULT)
    g.edge_update(U, W)
    g.sync()
    del U, W
    _release()
    rng = np.random.default_rng(20)
    nodes = sorted(set(rng.choice(spec.V, 32, replace=False).tolist()) | {(1 << 19) + 3, spec.V - 1})
    _check_sampled(g, spec, seed, nodes)
    labels, ncc, st = g.connected_components()
    assert st["fails_last"] == 0 and st["exhausted"] == 0
    # a core of 128 hubs: the components are exact for any core size, and the
    # smaller core keeps the ground truth quick at V = 2^20
    assert np.array_equal(labels, kron_components(spec, n_hubs=128))
    g.close()
    _release()
