"""Autotuner of the batched ingestion path.

Picks, for one GPU model and one V, the knobs of gz_config that change speed
but never results: the delta-update mode in shared memory (32-bit shared
atomics or load-xor-store), the records per work tile, the exact-depth rows staged in
shared memory, the resident CTAs per SM of the persistent kernel and the
partition chunk (updates per partition pass).  The search is coordinate
descent from the built-in defaults over a sample of the caller's device
stream, each candidate timed with CUDA events on the current stream; the
winner is cached in a JSON file keyed by (GPU name, V).

The paper tunes the analogous knobs of its CPU system by hand (gutter size,
Graph Worker count and group size, Sections 6.4 and 6.5).
"""
from __future__ import annotations

import json
import os

SPACE = {
    "smem_mode": [1, 2],
    "tile_records": [256, 512, 1024, 2048],
    "smem_rows": [12, 14, 16],
    "ctas_per_sm": [0, 2, 3],
    "chunk_log2": [24, 25, 26, 27],
}
DEFAULT = {"smem_mode": 1, "tile_records": 512, "smem_rows": 16, "ctas_per_sm": 0, "chunk_log2": 26}

CACHE = os.environ.get("GZ_TUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_configs.json"))


def _key(gpu: str, V: int) -> str:
    return f"{gpu}|V={V}"


def load(gpu: str, V: int) -> dict | None:
    try:
        with open(CACHE) as f:
            return json.load(f).get(_key(gpu, V))
    except Exception:
        return None


def store(gpu: str, V: int, entry: dict) -> None:
    try:
        with open(CACHE) as f:
            d = json.load(f)
    except Exception:
        d = {}
    d[_key(gpu, V)] = entry
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def measure(V: int, u, v, cfg: dict, seed: int = 1, reps: int = 2) -> float:
    """Updates/s of reset + gz_edge_update over the device sample (u, v)."""
    import torch

    import paper_2203_14927_b300 as gz

    g = gz.Graph(V, seed, **cfg)
    try:
        n = u.numel()
        g.edge_update(u[: min(n, 1 << 20)], v[: min(n, 1 << 20)])  # warm-up
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = float("inf")
        for _ in range(reps):
            g.reset()
            torch.cuda.synchronize()
            e0.record(stream)
            g.edge_update(u, v)
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1000.0)
        g.sync()
        return n / best
    finally:
        g.close()


def tune(V: int, u, v, seed: int = 1, passes: int = 2, use_cache: bool = True, log=None) -> dict:
    """Coordinate descent over SPACE; returns {"config": {...}, "rate": x, "tried": [...]}."""
    import torch

    gpu = torch.cuda.get_device_name()
    if use_cache:
        hit = load(gpu, V)
        if hit:
            return hit
    best = dict(DEFAULT)
    best_rate = measure(V, u, v, best, seed)
    tried = [(dict(best), best_rate)]
    for _ in range(passes):
        improved = False
        for name, values in SPACE.items():
            for val in values:
                if val == best[name]:
                    continue
                cand = dict(best)
                cand[name] = val
                try:
                    rate = measure(V, u, v, cand, seed)
                except Exception as exc:  # a candidate that does not fit is skipped
                    if log:
                        log(f"[tune] {cand}: {exc}")
                    continue
                tried.append((dict(cand), rate))
                if log:
                    log(f"[tune] {cand}: {rate / 1e9:.3f} G/s")
                if rate > best_rate * 1.01:
                    best, best_rate, improved = cand, rate, True
        if not improved:
            break
    entry = {"config": best, "rate": best_rate, "default_rate": tried[0][1],
             "tried": [[c, r] for c, r in tried], "sample_updates": int(u.numel())}
    store(gpu, V, entry)
    return entry
