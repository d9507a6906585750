#!/usr/bin/env python
"""Benchmark of the GraphZeppelin hot path on B300: CubeSketch edge updates/s
(whole job), HBM roofline of the batched update kernel, and Boruvka CC query
latency (p50/p99).

One step = zero the sketches, ingest the whole resident stream through
gz_edge_update (device pointers; the library partitions it into 2^24-update
chunks), then one gz_connected_components query.  Inputs are a seeded
Kronecker insert/delete stream generated on the device before timing; every
input (stream and sketches) is far larger than the 126 MB L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload kron17]
    python bench.py --impl reference      # the CPU oracle, timed on host cores
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2203_14927_b300 import streams as S  # noqa: E402

WORKLOADS = {
    # name: (log2 V, stream updates, churn, seed, description)
    "kron17": (17, 4.0e9, 0.1, 17, "V=2^17 Graph500-initiator Kronecker stream, ~4e9 updates, 10% churn"),
    "kron15": (15, 3.0e8, 0.1, 15, "V=2^15 Graph500-initiator Kronecker stream, ~3e8 updates, 10% churn"),
    "kron13": (13, 2.0e7, 0.1, 13, "V=2^13 Graph500-initiator Kronecker stream, ~2e7 updates, 10% churn"),
    # beyond the paper's largest graph (kron18): 123 GB of node sketches on one GPU
    "kron20": (20, 8.0e9, 0.1, 20, "V=2^20 Graph500-initiator Kronecker stream, ~8e9 updates, 10% churn"),
}
CHUNK_LOG2 = 24

# DRAM bytes per update of k_batched from one ncu capture (one-pass
# dram__bytes_read.sum + dram__bytes_write.sum, two full 2^26-update launches
# of this bench's own step); valid only for the kernel source it was taken with
# (kernel_sha) and its configuration.
TRAFFIC = {
    "kron17": {"sha": "ed532baf39b96e24",
               "cfg": {"smem_mode": 1, "tile_records": 512, "smem_rows": 16, "ctas_per_sm": 0, "chunk_log2": 26},
               "bytes_per_update": 140.92,
               # smsp__thread_inst_executed.sum per column update, same capture rules
               "thread_instr_per_column_update": 17.20,
               "source": "profiles/k_batched_kron17_dram.md"},
}


def kernel_sha() -> str:
    """Fingerprint of the batched kernel's device code: its section of
    gz_ingest.cu (from the "batched update" banner to the dispatch table) and
    gz_internal.cuh."""
    import hashlib

    d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2203_14927_b300", "csrc")
    with open(os.path.join(d, "gz_ingest.cu")) as fh:
        src = fh.read()
    lo = src.index("// ------------------------------------------------------------------ batched update")
    hi = src.index("using BatchedFn = void (*)(BatchedArgs);")
    h = hashlib.sha256(src[lo:hi].encode())
    with open(os.path.join(d, "gz_internal.cuh"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, cfg: dict, kernel: str):
    t = TRAFFIC.get(workload)
    if kernel != "batched" or not t:
        return None, "no ncu capture for this workload"
    if kernel_sha() != t["sha"]:
        return None, "kernel sources changed since the ncu capture"
    if any(cfg.get(k) != v for k, v in t["cfg"].items()):
        return None, f"ncu capture taken at config {t['cfg']}"
    return t, t["source"]


def nvtx_push(name: str):
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop():
    try:
        import torch
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle


def oracle_rate(spec: S.KronSpec, seed: int, budget_s: float, max_nodes: int = 64, first: int = 0):
    """The CPU oracle as it stands (single thread) sketching whole nodes of the
    same graph from their net neighbour lists; one stream update costs the
    oracle two node updates, so updates/s = (sum of degrees / 2) / seconds."""
    import oracle

    rng = np.random.default_rng(1234 + first)
    nodes = rng.integers(0, spec.V, max_nodes)
    spent, endpoint_updates, used = 0.0, 0, []
    for x in nodes:
        nb = spec.node_neighbors(int(x))
        t0 = time.perf_counter()
        oracle.sketch_node(spec.V, seed, int(x), nb)
        spent += time.perf_counter() - t0
        endpoint_updates += len(nb)
        used.append(int(x))
        if spent >= budget_s:
            break
    return endpoint_updates / 2.0 / spent, spent, used, endpoint_updates


def mem_available_bytes() -> int:
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def paper_design_rate(V: int, seed: int, u, v):
    """The paper's CPU design (per-node buffers, parallel workers; Section 5.1)
    on every host core, over the given stream prefix.  All V node sketches
    when host memory allows (3x their size available), else the first node
    range that fits (updates/s then counts the endpoint updates applied / 2)."""
    import oracle

    K, R = oracle.geometry(V)
    per_node = K * 7 * R * 12
    avail = mem_available_bytes()
    span = V if avail >= 3 * V * per_node else max(1024, min(V, avail // (4 * per_node)))
    inside = ((u < span).astype(np.int64) + (v < span).astype(np.int64)).sum()
    threads = oracle.max_threads()
    t0 = time.perf_counter()
    oracle.ingest_batched(V, seed, u, v, 0, span, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": float(inside) / 2.0 / dt, "unit": "updates/s", "cores": threads,
            "kind": "the paper's design: per-node buffers applied by parallel workers (OpenMP), "
                    "nested CubeSketch rows",
            "sample": f"first {len(u)} updates of the same stream, nodes [0, {span}) of {V} "
                      f"({int(inside)} endpoint updates, {dt:.1f} s)"}


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    L, n_upd, churn, seed, desc = WORKLOADS[args.workload]
    spec = S.kron_for_updates(L, seed, n_upd, churn=churn, chunk_updates=2 ** CHUNK_LOG2)
    per_step = max(0.5, args.ref_seconds / max(1, args.steps + args.warmup))
    for w in range(args.warmup):
        oracle_rate(spec, seed, per_step, first=100 + w)
    rates, times, nodes_all, eu = [], [], [], 0
    for s in range(args.steps):
        r, t, nodes, e = oracle_rate(spec, seed, per_step, first=s)
        rates.append(r)
        times.append(t)
        nodes_all += nodes
        eu += e
    value = eu / 2.0 / sum(times)
    sample = (f"oracle sketch_node over {len(nodes_all)} random nodes of the {args.workload} final graph "
              f"({eu} endpoint updates = {eu / 2:.0f} stream updates), single thread")
    out = {
        "impl": "reference", "metric": "edge_updates_per_sec", "value": value, "unit": "updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded Kronecker graph)",
        "config": {"workload": f"{args.workload}: {desc}", "V": spec.V},
        "cpu_baseline": {"value": value, "unit": "updates/s", "cores": 1, "kind": "oracle",
                         "sample": sample, "cpu": cpu_model()},
        "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- ranks


def max_over_ranks(ms: float, dist=None, device="cpu") -> float:
    """Slowest rank's time: the whole job finishes when the last replica does."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def wide_index_fraction(u, v, V: int, torch, block: int = 1 << 26) -> float:
    """Fraction of updates whose edge index min(u,v)*V + max(u,v) is 2^32 or
    more: both hashes of such an index need its high word (11 integer
    operations per column update instead of 7)."""
    n = u.numel()
    if V * V <= (1 << 32) or n == 0:
        return 0.0
    wide = 0
    for s in range(0, n, block):
        a = u[s:s + block].long()
        b = v[s:s + block].long()
        idx = torch.minimum(a, b) * V + torch.maximum(a, b)
        wide += int((idx >= (1 << 32)).sum())
    return wide / n


def wide_segment_fraction(u, v, V: int, torch, block: int = 1 << 26) -> float:
    """Fraction of partition records (one per endpoint of every update) that
    lie in the segment of a node x >= floor((2^32 - V) / V) + 1, the nodes
    whose edge indices can reach 2^32: the batched kernel runs its 64-bit
    column code on every record of such a segment."""
    n = u.numel()
    if V * V <= (1 << 32) or n == 0:
        return 0.0
    xn = ((1 << 32) - V) // V + 1
    wide = 0
    for s in range(0, n, block):
        wide += int((u[s:s + block].long() >= xn).sum()) + int((v[s:s + block].long() >= xn).sum())
    return wide / (2 * n)


def whole_job_rate(updates_per_rank_step: int, steps: int, world: int, ms_max: float) -> float:
    """Updates of all ranks over the slowest rank's time (weak scaling: every
    rank ingests its own graph of the same size)."""
    return world * updates_per_rank_step * steps / (ms_max / 1000.0)


# ----------------------------------------------------------------------------- GPU path


def generate_on_device(spec, torch, gz):
    gen = gz.DeviceKronStream(spec)
    # the expected stream length with a margin; the generator refuses a chunk
    # that would not fit (GZ_EINVAL), it never writes past the capacity
    est = spec.target_edges * (1 + 2 * spec.churn)
    cap = int(est * 1.08) + (1 << 26)
    U = torch.empty(cap, dtype=torch.int32, device="cuda")
    Vv = torch.empty(cap, dtype=torch.int32, device="cuda")
    off = 0
    for c in range(gen.n_chunks):
        n = gen.chunk_into(c, U.data_ptr() + 4 * off, Vv.data_ptr() + 4 * off, cap - off)
        off += n
    gen.close()
    return U, Vv, off


def run_ours(args, rank: int, world: int):
    import torch

    import paper_2203_14927_b300 as gz

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))

    L, n_upd, churn, seed, desc = WORKLOADS[args.workload]
    seed = seed + 1000 * rank  # independent replicas: each rank its own graph
    spec = S.kron_for_updates(L, seed, n_upd, churn=churn, chunk_updates=2 ** CHUNK_LOG2)
    t0 = time.time()
    U, Vv, total = generate_on_device(spec, torch, gz)
    torch.cuda.synchronize()
    log(f"[bench] rank {rank}: generated {total} updates on device in {time.time() - t0:.1f}s")
    u_all, v_all = U[:total], Vv[:total]
    f_wide = wide_index_fraction(u_all, v_all, spec.V, torch)
    f_wide_seg = wide_segment_fraction(u_all, v_all, spec.V, torch)
    int_peaks = {k: gz.int_peak(k) for k in ("imad", "lop3", "mixed", "clz", "atom_shared")}
    log("[bench] integer ceilings (T thread-instr/s): "
        + ", ".join(f"{k} {v / 1e12:.2f}" for k, v in int_peaks.items()))

    from paper_2203_14927_b300 import autotune

    cfg = dict(autotune.DEFAULT)
    tuned = None
    if args.kernel == "batched" and not args.no_tune:
        ns = min(total, 1 << 27)
        t0 = time.time()
        tuned = autotune.tune(spec.V, u_all[:ns], v_all[:ns], seed=seed, use_cache=False, log=log)
        cfg = dict(tuned["config"])
        log(f"[bench] autotuned in {time.time() - t0:.1f}s: {cfg} "
            f"({tuned['rate'] / 1e9:.3f} vs default {tuned['default_rate'] / 1e9:.3f} G/s on the sample)")
    if args.cfg:
        cfg.update(json.loads(args.cfg))
    if args.kernel == "plain":
        cfg = {"chunk_log2": CHUNK_LOG2}
    if args.device_sketch_mb:
        cfg["device_sketch_mb"] = args.device_sketch_mb
    g = gz.Graph(spec.V, seed=seed, kernel=args.kernel, **cfg)
    qtimes = []

    def step():
        g.reset()
        g.edge_update(u_all, v_all)
        labels, ncc, st = g.connected_components()
        qtimes.append(st["ms"])
        return ncc, st

    for _ in range(args.warmup):
        ncc, st = step()
        log(f"[bench] warmup step: components={ncc} rounds={st['rounds']} fails={st['fails_last']}")
    qtimes.clear()

    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g.profile_enable(True)
    with ClockSampler(dev) as clocks:
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ev0.record(stream)
        nvtx_push("timed")  # lets a profiler take the timed steps' kernels alone (--nvtx-include timed/)
        for _ in range(args.steps):
            ncc, st = step()
        nvtx_pop()
        ev1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    prof = g.profile_read()
    g.profile_enable(False)
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms, dist, "cuda")
    ms_per_step = ms_max / args.steps
    step_updates = total
    value = whole_job_rate(step_updates, args.steps, world, ms_max)
    clk = clocks.summary()

    # --- roofline of the dominant kernel (batched CubeSketch update) ---------
    peak, peak_kind = measured_peaks()
    launches = max(prof["batches"], 1)
    avg_ms = prof["update_ms"] / launches
    K, R = g.K, g.R
    upd_per_launch = prof["updates"] / launches
    sec = avg_ms / 1000.0
    s_total = spec.V * K * 84 * R
    col_updates = upd_per_launch * 2 * 7 * K
    # HBM, by the bytes the batched update must move per launch: its two
    # records per update (8 B) and a read-modify-write of every exact-depth
    # bucket a node segment changed (12 B each way; the kernel counts these
    # buckets as rows_flushed).  The full-sketch bound, one read and write of
    # every node sketch per chunk, overstates it whenever nodes touch few rows.
    rows_per_launch = prof["rows_flushed"] / launches
    captured, traffic_note = measured_traffic(args.workload, cfg, args.kernel)
    traffic = captured["bytes_per_update"] * upd_per_launch if captured else None
    hbm_bytes = 8.0 * upd_per_launch + 24.0 * rows_per_launch
    hbm = {"bound": "hbm", "achieved": hbm_bytes / sec / 1e9, "peak": peak, "unit": "GB/s",
           "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
           "bytes_per_launch": hbm_bytes, "touched_buckets_per_launch": rows_per_launch,
           "full_sketch_bytes_per_launch": 8.0 * upd_per_launch + 2.0 * s_total}
    hbm["frac"] = hbm["achieved"] / peak
    # Integer work, by the operations a column update needs under the piece
    # hashes: the depth piece (1 multiply-add) and its leading-zero count, the
    # two checksum pieces (2 multiply-adds) joined by one byte permute, and
    # one shared-memory XOR per bucket word (alpha lo, gamma; alpha hi for an
    # edge index of 2^32 or more, a fraction f_wide of the stream): 7 + f_wide
    # ops.  Each goes to one pipe, with its own measured ceiling on this GPU
    # (gz_int_peak): multiply-adds, leading-zero counts and shared atomics;
    # the issue ceiling bounds them all together.
    ops_per_cu = 7.0 + f_wide
    ops = col_updates * ops_per_cu
    issue_nominal = 148 * 4 * 32 * 2.032e9 / 1e12
    issue_peak = max(int_peaks[k] for k in ("imad", "lop3", "mixed")) / 1e12
    alu = {"bound": "alu", "pipe": "issue (all integer pipes)", "achieved": ops / sec / 1e12, "peak": issue_peak,
           "unit": "Tops/s",
           "peak_source": "measured: best of the integer probes "
                          + ", ".join(f"{k} {v / 1e12:.2f}" for k, v in int_peaks.items())
                          + f" T thread-ops/s (nominal issue {issue_nominal:.2f}: 148 SMs x 4 schedulers"
                            " x 32 lanes x 2.032 GHz)",
           "ops_per_launch": ops, "ops_per_column_update": ops_per_cu,
           "wide_index_fraction": f_wide, "wide_segment_fraction": f_wide_seg,
           "frac_of_nominal_issue": ops / sec / 1e12 / issue_nominal}
    alu["frac"] = alu["achieved"] / issue_peak
    imads = col_updates * 3.0
    imad_nominal = 148 * 4 * 16 * 2.032e9 / 1e12
    imad_peak = int_peaks["imad"] / 1e12
    imad = {"bound": "alu", "pipe": "integer multiply-add", "achieved": imads / sec / 1e12, "peak": imad_peak,
            "unit": "T IMAD/s", "peak_source": f"measured multiply-add chains (nominal {imad_nominal:.2f}:"
                                                " 148 SMs x 4 x 16-lane pipes x 2.032 GHz)",
            "imad_per_column_update": 3.0}
    imad["frac"] = imad["achieved"] / imad_peak
    clz_peak = int_peaks["clz"] / 1e12
    clz = {"bound": "alu", "pipe": "leading-zero count", "achieved": col_updates / sec / 1e12, "peak": clz_peak,
           "unit": "T clz/s", "peak_source": "measured leading-zero-count chains (nominal 4.81: 148 SMs x"
                                             " 16 lanes x 2.032 GHz)", "clz_per_column_update": 1.0}
    clz["frac"] = clz["achieved"] / clz_peak
    atom_peak = int_peaks["atom_shared"] / 1e12
    atoms = col_updates * (2.0 + f_wide)
    atom = {"bound": "alu", "pipe": "shared-memory atomics", "achieved": atoms / sec / 1e12, "peak": atom_peak,
            "unit": "T atomic XOR/s", "peak_source": "measured conflict-free 32-bit shared atomic XOR"
                                                     " (nominal 9.62: 148 SMs x 32 lanes x 2.032 GHz)",
            "atomics_per_column_update": 2.0 + f_wide}
    atom["frac"] = atom["achieved"] / atom_peak
    binding = max((hbm, alu, imad, clz, atom), key=lambda r: r["frac"])
    # context, not the roofline: the instructions the kernel executes (ncu)
    # against the same issue ceiling
    executed = None
    if captured:
        tpi = captured["thread_instr_per_column_update"]
        executed = {"bound": "alu", "pipe": "issue, executed instructions", "unit": "T thread-instr/s",
                    "achieved": col_updates * tpi / sec / 1e12, "peak": issue_peak,
                    "thread_instr_per_column_update": tpi, "source": captured["source"]}
        executed["frac"] = executed["achieved"] / issue_peak
    roofline = dict(binding)
    roofline.update({
        "kernel": "k_batched" if args.kernel == "batched" else "k_plain",
        "traffic": traffic,
        "traffic_source": traffic_note,
        "avg_launch_ms": avg_ms, "launches": launches, "updates_per_launch": upd_per_launch,
        "column_updates_per_s": col_updates / sec,
        "share_of_step": prof["update_ms"] / ms if ms > 0 else None,
        "partition_ms_per_launch": prof["partition_ms"] / launches,
        "all": {"hbm": hbm, "alu_issue": alu, "imad_pipe": imad, "clz_pipe": clz, "shared_atomics": atom},
        "executed_issue": executed,
    })

    # --- query latency -----------------------------------------------------------
    qs = [st["ms"]] if args.queries == 0 else []
    if args.trace_queries:
        g.enable_trace(True)  # host-driven rounds: a profiler lists every round's kernels
    qc = []  # the library's own clock around the call (graph launch to labels on the host)
    for _ in range(args.queries):
        t1 = time.perf_counter()
        labels, ncc, st = g.connected_components()
        qs.append((time.perf_counter() - t1) * 1000.0)
        qc.append(st["ms"])
    qs.sort()
    query = {"p50_ms": float(np.percentile(qs, 50)), "p99_ms": float(np.percentile(qs, 99)),
             "n": len(qs), "rounds": st["rounds"], "components": ncc, "fails_last": st["fails_last"],
             "in_step_ms": qtimes, "host_driven_trace": bool(args.trace_queries),
             "library_p50_ms": float(np.percentile(qc, 50)) if qc else None}

    # --- end to end through host buffers -------------------------------------
    e2e = None
    if not args.no_e2e:
        n_e2e = min(total, 1 << args.e2e_log2)
        hu = torch.empty(n_e2e, dtype=torch.int32, pin_memory=True)
        hv = torch.empty(n_e2e, dtype=torch.int32, pin_memory=True)
        hu.copy_(u_all[:n_e2e])
        hv.copy_(v_all[:n_e2e])
        hu_np, hv_np = hu.numpy(), hv.numpy()
        # raw pinned host -> device copy rate of the same buffers, for context
        dtmp = torch.empty(n_e2e, dtype=torch.int32, device="cuda")
        dtmp.copy_(hu, non_blocking=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dtmp.copy_(hu, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        h2d_gbs = 4 * n_e2e / (e0.elapsed_time(e1) / 1000.0) / 1e9
        del dtmp
        # the same handle, now fed from host memory (a second 2^20-node
        # graph would not fit beside the first one and the device stream)
        g.reset()
        g.edge_update(hu_np, hv_np)  # warm-up of the host path
        g.connected_components()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        reps = 2
        for _ in range(reps):
            g.reset()
            g.edge_update(hu_np, hv_np)
            labels, ncc_e, _ = g.connected_components()
        te = (time.perf_counter() - t1) / reps
        del hu, hv
        e2e = {"value": world * n_e2e / te, "unit": "updates/s", "h2d_bytes_per_step": 8 * n_e2e,
               "pinned_h2d_gbs": h2d_gbs,
               "d2h_bytes_per_step": 4 * spec.V + 32,
               "sample": f"first {n_e2e} updates of the same stream from pinned host memory "
                         f"(2^{int(math.log2(n_e2e))}), reset + gz_edge_update(host) + CC query with "
                         "labels read back, host wall clock"}

    # --- plain per-update kernel on a prefix of the same stream ---------------
    plain = None
    if not args.no_plain and args.kernel == "batched":
        n_pl = min(total, 1 << args.plain_log2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # the batched path on the prefix first, for a like-for-like ratio
        g.reset()
        e0.record(stream)
        g.edge_update(u_all[:n_pl], v_all[:n_pl])
        e1.record(stream)
        torch.cuda.synchronize()
        tb = e0.elapsed_time(e1) / 1000.0
        free_b, _ = torch.cuda.mem_get_info()
        if free_b < 1.1 * gz.memory_bytes(spec.V, kernel="plain", chunk_log2=CHUNK_LOG2):
            g.close()  # make room for the plain kernel's sketches
        gp = gz.Graph(spec.V, seed=seed, kernel="plain", chunk_log2=CHUNK_LOG2)
        gp.edge_update(u_all[:1 << 20], v_all[:1 << 20])
        torch.cuda.synchronize()
        gp.reset()
        e0.record(stream)
        gp.edge_update(u_all[:n_pl], v_all[:n_pl])
        e1.record(stream)
        torch.cuda.synchronize()
        tp = e0.elapsed_time(e1) / 1000.0
        gp.close()
        plain = {"value": n_pl / tp, "unit": "updates/s", "sample": f"first {n_pl} updates (2^{args.plain_log2})",
                 "batched_same_prefix": n_pl / tb, "speedup_batched_over_plain": tp / tb}

    # --- CPU oracle baseline ------------------------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        r, spent, nodes, eu = oracle_rate(spec, seed, args.cpu_seconds)
        cpu = {"value": r, "unit": "updates/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle sketch_node over {len(nodes)} random nodes of the same graph "
                         f"({eu} endpoint updates, {spent:.1f} s), single thread",
               "cpu": cpu_model(), "host_cores": host_cores()}
        n_pd = min(total, 1 << args.paper_design_log2)
        cpu["paper_design"] = paper_design_rate(spec.V, seed, u_all[:n_pd].cpu().numpy().view(np.uint32),
                                                v_all[:n_pd].cpu().numpy().view(np.uint32))
        log(f"[bench] paper-design CPU baseline: {cpu['paper_design']['value'] / 1e6:.2f} M updates/s "
            f"on {cpu['paper_design']['cores']} threads")

    if rank == 0:
        out = {
            "metric": "edge_updates_per_sec",
            "value": value,
            "unit": "updates/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_per_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "u64",
            "data": "synthetic: seeded Kronecker insert/delete stream generated on device",
            "config": {
                "workload": f"{args.workload}: {desc}",
                "V": spec.V, "K": K, "R": R, "updates_per_step": step_updates,
                "chunk_updates": 2 ** cfg.get("chunk_log2", CHUNK_LOG2), "kernel": args.kernel,
                "tuned": cfg if tuned else None,
                "tune_sample": {"rate": tuned["rate"], "default_rate": tuned["default_rate"],
                                "candidates": len(tuned["tried"])} if tuned else None,
                "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                "l2": "no flush needed: stream (%.1f GB) and sketches (%.1f GB) exceed the 126 MB L2"
                      % (8 * total / 1e9, spec.V * K * 84 * R / 1e9),
                "step": "reset sketches + ingest whole stream + one CC query",
                "sketches_beyond_hbm": None if not args.device_sketch_mb else
                f"{args.device_sketch_mb} MiB of sketches in HBM, the rest "
                f"({spec.V * K * 84 * R / 1e9 - args.device_sketch_mb * 2 ** 20 / 1e9:.1f} GB or more) in pinned host "
                "memory, streamed through three device shard slots per chunk",
            },
            "roofline": roofline,
            "query_ms": query,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "plain_kernel": plain,
            "gpu_launches": prof["kernel_launches"],
            "clocks": clk,
            "profile": prof,
        }
        if world == 1 and not args.no_serve_summary:
            g.close()
            del U, Vv, u_all, v_all
            torch.cuda.empty_cache()
            out["serving"] = serve_summary(args, torch, gz)
        print(json.dumps(out), flush=True)
    g.close()
    if dist:
        dist.destroy_process_group()


def serve_mix(n_graphs: int, planted_half: bool, torch, gz):
    """The serving mix: n_graphs graphs with V = 2^U{10..16} and 4 V log2(V)
    updates each, Kronecker streams (device generator) or, with planted_half,
    every second graph a planted G(n,p) stream; each cut into update chunks of
    2^U(16,20) updates.  Payloads are pinned host arrays, lent to the server."""
    rng = np.random.default_rng(2026)
    graphs = []
    for i in range(n_graphs):
        e = int(rng.integers(10, 17))
        V = 1 << e
        n_upd = int(4 * V * e)
        seed = 9000 + i
        if i % 2 == 0 or not planted_half:
            spec = S.kron_for_updates(e, seed, n_upd, churn=0.1, chunk_updates=2 ** 22, n_iso=8)
            U, Vv, tot = generate_on_device(spec, torch, gz)
            hu = torch.empty(tot, dtype=torch.int32, pin_memory=True)
            hv = torch.empty(tot, dtype=torch.int32, pin_memory=True)
            hu.copy_(U[:tot])
            hv.copy_(Vv[:tot])
            del U, Vv
            kind = "kronecker"
        else:
            u0, v0, _ = S.planted_sparse_stream(V, seed, n_upd)
            hu = torch.from_numpy(u0.view(np.int32)).pin_memory()
            hv = torch.from_numpy(v0.view(np.int32)).pin_memory()
            kind = "planted"
        u, v = hu.numpy().view(np.uint32), hv.numpy().view(np.uint32)
        cuts, pos = [], 0
        while pos < len(u):
            pos += int(2 ** rng.uniform(16, 20))
            cuts.append(min(pos, len(u)))
        graphs.append({"V": V, "seed": seed, "u": u, "v": v, "cuts": cuts, "kind": kind, "pin": (hu, hv)})
    return graphs


def serve_footprint(graphs, gz) -> float:
    import ctypes
    c = gz.Config()
    c.chunk_log2 = 20
    c.no_pipeline = 1
    tot = 0
    for g in graphs:
        b = ctypes.c_size_t()
        gz.lib().gz_memory_bytes(g["V"], ctypes.byref(c), ctypes.byref(b))
        tot += b.value
    return tot


def serve_schedule(graphs, window: float):
    """Poisson arrivals: each graph's update chunks spread over `window`
    seconds, a query after about one chunk in three and after the last."""
    r = np.random.default_rng(77)
    events = []
    for gi, g in enumerate(graphs):
        rate = len(g["cuts"]) / window
        t, lo = 0.0, 0
        for hi in g["cuts"]:
            t += r.exponential(1.0 / rate)
            events.append((t, gi, "u", lo, hi))
            lo = hi
            if r.random() < 1.0 / 3.0:
                events.append((t + 1e-9, gi, "q", 0, 0))
        events.append((t + 2e-9, gi, "q", 0, 0))
        events.append((t + 3e-9, gi, "close", 0, 0))
    events.sort(key=lambda x: x[0])
    return events


def serve_pass(srv, graphs, events, torch, gz, graph_cfg=None, one_at_a_time=False, paced=False) -> dict:
    """Run one pass of `events` through the server `srv` (the graphs are
    registered afresh and closed by the events); host wall clock."""
    gids = [srv.add_graph(g["V"], g["seed"], **(graph_cfg or {})) for g in graphs]
    torch.cuda.synchronize()
    total_updates = sum(len(g["u"]) for g in graphs)
    st0 = srv.stats()

    def submit(ev):
        _, gi, kind, lo, hi = ev
        g = graphs[gi]
        if kind == "u":
            srv.submit_update(gids[gi], g["u"][lo:hi], g["v"][lo:hi], copy=False)
        elif kind == "q":
            srv.submit_query(gids[gi])
        else:
            srv.close_graph(gids[gi])

    start = time.perf_counter()
    if one_at_a_time:
        for gi in range(len(graphs)):
            for ev in events:
                if ev[1] == gi:
                    submit(ev)
            srv.drain()
    else:
        for ev in events:
            if paced:
                now = time.perf_counter() - start
                if ev[0] > now:
                    time.sleep(ev[0] - now)
            submit(ev)
        srv.drain()
    elapsed = time.perf_counter() - start
    done = srv.poll(1 << 20)
    st = srv.stats()
    err = srv.last_error()
    bad = sum(1 for c in done if c["status"] not in (gz.GZ_OK, gz.GZ_ESKETCH_FAIL))
    q = sorted(c["done_ms"] - c["submit_ms"] for c in done if c["kind"] == 1)
    out = {"elapsed_s": elapsed, "updates_per_s": total_updates / elapsed,
           "query_p50_ms": float(np.percentile(q, 50)), "query_p99_ms": float(np.percentile(q, 99)),
           "queries": len(q), "requests": len(done), "errors": bad,
           "budget_gb": st["budget_bytes"] / 1e9, "evictions": st["evictions"] - st0["evictions"],
           "evict_ms": st["evict_ms"] - st0["evict_ms"], "restore_ms": st["restore_ms"] - st0["restore_ms"],
           "pinned_gb_new": (st["pinned_chunks"] - st0["pinned_chunks"]) * 0.25 * 2 ** 30 / 1e9}
    if bad:
        out["last_error"] = err
    return out


def serve_measure(graphs, budget_gb: float, slots: int, torch, gz, graph_cfg=None) -> dict:
    """One server, `slots` workers.  Capacity with every request queued at
    once and with the same requests served one graph at a time (a drain
    between graphs), then query latency with Poisson arrivals at half the
    measured capacity, under an HBM budget of budget_gb, and again under a
    budget that holds every graph.  Untimed passes first: module loads and
    query-graph captures, the device's memory pool grown to every graph, and
    the pinned host buffers that evictions reuse."""
    budget = int(budget_gb * 1e9)
    foot = serve_footprint(graphs, gz)
    ample = int(1.5 * foot) + (8 << 30)
    total_updates = sum(len(g["u"]) for g in graphs)
    events0 = serve_schedule(graphs, 1.0)
    # pinned host memory for two of the largest graphs' sketches, pinned before
    # the passes (a server that has run a while holds such a pool)
    big = max(gz.memory_bytes(g["V"], chunk_log2=20, no_pipeline=1) for g in graphs)
    srv = gz.Server(hbm_budget=ample, slots=slots, max_batch=8, host_pool_mb=int(2 * big / 2 ** 20) + 256)
    try:
        serve_pass(srv, graphs, events0, torch, gz, graph_cfg)  # warm-up
        srv.set_budget(budget)
        mixed = serve_pass(srv, graphs, events0, torch, gz, graph_cfg)
        seq = serve_pass(srv, graphs, events0, torch, gz, graph_cfg, one_at_a_time=True)
        window = max(1.0, total_updates / (0.5 * mixed["updates_per_s"]))
        paced_events = serve_schedule(graphs, window)
        serve_pass(srv, graphs, paced_events, torch, gz, graph_cfg, paced=True)  # warm-up: pinned buffers
        paced = serve_pass(srv, graphs, paced_events, torch, gz, graph_cfg, paced=True)
        srv.set_budget(ample)
        paced_ample = serve_pass(srv, graphs, paced_events, torch, gz, graph_cfg, paced=True)
        peak = srv.stats()["peak_resident_bytes"]
    finally:
        srv.close()
    return {"graphs": len(graphs), "total_updates": total_updates, "footprint_gb": foot / 1e9,
            "budget_gb": budget / 1e9, "slots": slots, "peak_resident_gb": peak / 1e9,
            "capacity_mixed": mixed, "capacity_one_at_a_time": seq,
            "mixed_over_one_at_a_time": seq["elapsed_s"] / mixed["elapsed_s"],
            "paced_window_s": window, "offered_load": "half of the mixed capacity, Poisson arrivals",
            "paced": paced, "paced_all_resident": paced_ample}


def serve_summary(args, torch, gz) -> dict:
    """A bounded serving figure for the main line: the serving mix with
    Kronecker streams only (the device generator keeps it to seconds)."""
    t0 = time.time()
    graphs = serve_mix(args.serve_graphs, False, torch, gz)
    m = serve_measure(graphs, args.serve_budget_gb, args.serve_slots, torch, gz)
    m["workload"] = (f"{len(graphs)} graphs, V = 2^U{{10..16}}, 4 V log2 V Kronecker updates each, update "
                     "chunks 2^U(16,20) and CC queries; all queued at once (capacity) or Poisson arrivals")
    m["wall_s"] = time.time() - t0
    log(f"[bench] serving summary in {m['wall_s']:.1f}s: mixed {m['capacity_mixed']['updates_per_s'] / 1e6:.0f} M/s"
        f", one at a time {m['capacity_one_at_a_time']['updates_per_s'] / 1e6:.0f} M/s, paced p50/p99 "
        f"{m['paced']['query_p50_ms']:.1f}/{m['paced']['query_p99_ms']:.1f} ms")
    return m


def run_serve(args, rank: int, world: int):
    """Serving: many independent graphs on one GPU (gz_server)."""
    import torch

    import paper_2203_14927_b300 as gz

    if rank != 0:
        return
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    t0 = time.time()
    graphs = serve_mix(args.serve_graphs, True, torch, gz)
    log(f"[serve] {len(graphs)} graphs, {sum(len(g['u']) for g in graphs)} updates, "
        f"generated in {time.time() - t0:.1f}s")
    graph_cfg = json.loads(args.cfg) if args.cfg else {}
    m = serve_measure(graphs, args.serve_budget_gb, args.serve_slots, torch, gz, graph_cfg)
    mixed, paced = m["capacity_mixed"], m["paced"]
    out = {
        "metric": "serve_aggregate_updates_per_sec", "value": mixed["updates_per_s"], "unit": "updates/s",
        "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": mixed["elapsed_s"] * 1000.0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic: seeded graphs, half Kronecker (device generator), half planted G(n,p)",
        "config": {"workload": f"serve: {len(graphs)} graphs, V = 2^U{{10..16}}, update chunks 2^U(16,20) "
                               "and CC queries as Poisson arrivals",
                   "graphs": len(graphs), "total_updates": m["total_updates"],
                   "footprint_gb": m["footprint_gb"], "budget_gb": m["budget_gb"], "slots": m["slots"]},
        "query_ms": {"p50_ms": paced["query_p50_ms"], "p99_ms": paced["query_p99_ms"], "n": paced["queries"],
                     "offered_load": m["offered_load"]},
        "serving": m,
    }
    print(json.dumps(out), flush=True)


def _truth(spec):
    from oracle.kron_cc import kron_components
    return kron_components(spec)


def run_failures(args, rank: int, world: int):
    """Sketch-failure rate: for each seed, ingest a V = 2^17 Kronecker stream
    and query; compare the labels with the exact components of the net graph
    (oracle, on the host cores, in a spawn-started pool)."""
    import multiprocessing as mp

    if rank != 0:
        return
    L, n_upd, churn, _, desc = WORKLOADS[args.fail_workload]
    seeds = [100 + i for i in range(args.seeds)]
    specs = [S.kron_for_updates(L, sd, n_upd, churn=churn, chunk_updates=2 ** CHUNK_LOG2) for sd in seeds]
    pool = mp.get_context("spawn").Pool(min(len(specs), max(1, host_cores() - 2)))
    truth_async = [pool.apply_async(_truth, (sp,)) for sp in specs]

    import torch

    import paper_2203_14927_b300 as gz
    from paper_2203_14927_b300 import autotune

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cfg = dict(autotune.DEFAULT)
    if args.cfg:
        cfg.update(json.loads(args.cfg))
    rows = []
    for sd, sp in zip(seeds, specs):
        U, Vv, tot = generate_on_device(sp, torch, gz)
        g = gz.Graph(sp.V, seed=sd, **cfg)
        g.edge_update(U[:tot], Vv[:tot])
        t0 = time.perf_counter()
        labels, ncc, st = g.connected_components()
        qms = (time.perf_counter() - t0) * 1000.0
        g.close()
        del U, Vv
        rows.append({"seed": sd, "updates": tot, "components": ncc, "rounds": st["rounds"],
                     "fails_last": st["fails_last"], "fails_total": st["fails_total"],
                     "exhausted": st["exhausted"], "query_ms": qms, "labels": labels})
        log(f"[failures] seed {sd}: {tot} updates, {ncc} components, rounds {st['rounds']}, "
            f"FAIL results {st['fails_total']}")
    wrong = 0
    for r, fut in zip(rows, truth_async):
        want = fut.get()
        r["correct"] = bool(np.array_equal(r.pop("labels"), want))
        r["true_components"] = int(len(np.unique(want)))
        wrong += not r["correct"]
    pool.close()
    out = {
        "metric": "sketch_failure_rate", "value": wrong / len(rows), "unit": "wrong queries / queries",
        "n_gpus": 1, "steps": len(rows), "warmup": 0, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic: seeded Kronecker streams generated on device",
        "config": {"workload": f"{args.fail_workload}: {desc}", "seeds": seeds,
                   "truth": "exact components of the net graph (oracle, hub-core shortcut checked against "
                            "union-find in tests)"},
        "fail_results_total": sum(r["fails_total"] for r in rows),
        "queries_with_fail_in_last_round": sum(1 for r in rows if r["fails_last"]),
        "per_seed": rows,
    }
    print(json.dumps(out), flush=True)


def run_stream_queries(args, rank: int, world: int):
    """Queries during the stream (the experiment of Fig. query): ingest the
    kron17 stream and issue a CC query after every tenth of it.  Each query
    first waits for the updates already queued (the flush of Section 5.2) and
    then runs Boruvka; both are reported, with the rate of the whole job."""
    import torch

    import paper_2203_14927_b300 as gz
    from paper_2203_14927_b300 import autotune

    if rank != 0:
        return
    torch.cuda.set_device(0)
    L, n_upd, churn, seed, desc = WORKLOADS["kron17"]
    spec = S.kron_for_updates(L, seed, n_upd, churn=churn, chunk_updates=2 ** CHUNK_LOG2)
    U, Vv, total = generate_on_device(spec, torch, gz)
    u_all, v_all = U[:total], Vv[:total]
    cfg = dict(autotune.DEFAULT)
    if args.cfg:
        cfg.update(json.loads(args.cfg))
    g = gz.Graph(spec.V, seed=seed, **cfg)
    cuts = [round(total * i / 10) for i in range(11)]

    def run(with_queries: bool):
        g.reset()
        torch.cuda.synchronize()
        rows = []
        t0 = time.perf_counter()
        for i in range(1, 11):
            g.edge_update(u_all[cuts[i - 1]:cuts[i]], v_all[cuts[i - 1]:cuts[i]])
            if with_queries:
                tq = time.perf_counter()
                labels, ncc, st = g.connected_components()
                wall = (time.perf_counter() - tq) * 1000.0
                rows.append({"fraction": i / 10, "updates": cuts[i], "components": ncc, "rounds": st["rounds"],
                             "query_ms": st["ms"], "wait_for_queued_ingest_ms": max(0.0, wall - st["ms"]),
                             "status": st["status"]})
        g.sync()
        return time.perf_counter() - t0, rows

    for _ in range(max(1, args.warmup)):
        run(True)
    t_plain, _ = run(False)
    t_q, rows = run(True)
    q = sorted(r["query_ms"] for r in rows)
    out = {
        "metric": "edge_updates_per_sec", "value": total / t_q, "unit": "updates/s", "n_gpus": 1,
        "steps": 1, "warmup": max(1, args.warmup), "ms_per_step": t_q * 1000.0, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic: seeded Kronecker insert/delete stream generated on device",
        "config": {"workload": f"kron17 with a CC query after every 10% of the stream: {desc}",
                   "V": spec.V, "updates": total, "cfg": cfg,
                   "timing": "host wall clock around the whole job (ingest calls + queries)"},
        "ingest_only_updates_per_s": total / t_plain,
        "query_overhead": t_q / t_plain - 1.0,
        "query_ms": {"p50_ms": float(np.percentile(q, 50)), "max_ms": q[-1], "n": len(q)},
        "per_query": rows,
        "paper": "Fig. query1: kron17, queries every 10% of the stream, 3.95e6 updates/s with 400-byte buffers",
    }
    g.close()
    print(json.dumps(out), flush=True)


# Fig. l0speedup, single-threaded CPU rates of the paper (updates/s):
# vector length -> (standard l0, CubeSketch)
PAPER_L0 = {10 ** 3: (223000, 7322000), 10 ** 4: (124000, 5180000), 10 ** 5: (54800, 4384000),
            10 ** 6: (29300, 3730000), 10 ** 7: (20900, 3177000), 10 ** 8: (16300, 2825000),
            10 ** 9: (13100, 2587000), 10 ** 10: (1350, 2272000), 10 ** 11: (918, 2108000),
            10 ** 12: (833, 1963000)}


def run_l0(args, rank: int, world: int):
    """Micro-benchmark of Fig. l0speedup on the GPU: ingestion rate of the
    standard l0 sampler (Fig. agm_code) and of CubeSketch into vector sketches
    of length n = 1e3 .. 1e12, many independent sketches at once (one thread
    per sketch column), with the CPU oracle's single-thread rates beside them."""
    import torch

    import oracle
    import paper_2203_14927_b300 as gz

    if rank != 0:
        return
    torch.cuda.set_device(0)
    dev = torch.device("cuda")
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    sketches, m, seed = sm * 256, 256, 42
    rows = []
    for e in range(3, 13):
        n = 10 ** e
        gen = torch.Generator(device=dev).manual_seed(e)
        x = torch.randint(1, n + 1, (sketches, m), device=dev, generator=gen, dtype=torch.int64)
        dl = (torch.randint(0, 2, (sketches, m), device=dev, generator=gen, dtype=torch.int32) * 2 - 1)
        R, bc, bs = gz.l0_geometry(n)
        rec = {"n": n, "rows": R}
        for kind, name, nb in ((gz.L0_CUBE, "cubesketch", bc), (gz.L0_STANDARD, "standard", bs)):
            buf = torch.zeros(sketches * nb, dtype=torch.uint8, device=dev)
            gz.l0_update(kind, n, seed, x, buf, dl)  # warm-up
            best = float("inf")
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                gz.l0_update(kind, n, seed, x, buf, dl)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1000.0)
            rec[f"gpu_{name}_updates_per_s"] = sketches * m / best
            # CPU oracle, single thread, bounded sample
            xs = x[0].cpu().numpy().view(np.uint64)
            ds = dl[0].cpu().numpy()
            t0, k = time.perf_counter(), 0
            while time.perf_counter() - t0 < args.l0_cpu_seconds:
                oracle.l0_update(kind, n, seed, xs, ds)
                k += len(xs)
            rec[f"cpu_oracle_{name}_updates_per_s"] = k / (time.perf_counter() - t0)
        rec["gpu_speedup_cube_over_standard"] = (rec["gpu_cubesketch_updates_per_s"]
                                                 / rec["gpu_standard_updates_per_s"])
        rec["paper_cpu_standard"], rec["paper_cpu_cubesketch"] = PAPER_L0[n]
        rows.append(rec)
        log(f"[l0] n=1e{e}: GPU cube {rec['gpu_cubesketch_updates_per_s'] / 1e9:.2f} G/s, "
            f"standard {rec['gpu_standard_updates_per_s'] / 1e9:.3f} G/s "
            f"({rec['gpu_speedup_cube_over_standard']:.1f}x)")
    out = {
        "metric": "l0_updates_per_sec", "value": rows[-1]["gpu_cubesketch_updates_per_s"], "unit": "updates/s",
        "n_gpus": 1, "steps": 3, "warmup": 1, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic: uniform positions, +-1 deltas",
        "config": {"workload": "Fig. l0speedup on the GPU: vector sketches of length 1e3..1e12, "
                               f"{sketches} sketches x {m} updates, 7 columns, thread per column",
                   "value": "CubeSketch rate at n = 1e12"},
        "per_length": rows,
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["serve", "failures", "stream_queries", "l0"],
                    default="kron17")
    ap.add_argument("--seeds", type=int, default=20)
    ap.add_argument("--fail-workload", choices=sorted(WORKLOADS), default="kron17")
    ap.add_argument("--serve-graphs", type=int, default=64)
    ap.add_argument("--no-serve-summary", action="store_true",
                    help="skip the bounded serving summary of the main line")
    ap.add_argument("--serve-budget-gb", type=float, default=24.0)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--kernel", choices=["batched", "plain"], default="batched")
    ap.add_argument("--queries", type=int, default=20)
    ap.add_argument("--trace-queries", action="store_true",
                    help="run the --queries extra CC queries host-driven with the per-round trace (for profiling)")
    ap.add_argument("--paper-design-log2", type=int, default=22,
                    help="stream prefix (log2 updates) for the OpenMP paper-design CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--l0-cpu-seconds", type=float, default=0.5)
    ap.add_argument("--ref-seconds", type=float, default=40.0)
    ap.add_argument("--e2e-log2", type=int, default=30)
    ap.add_argument("--plain-log2", type=int, default=26)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--cfg", default="", help="JSON gz_config overrides, e.g. '{\"smem_mode\": 1}'")
    ap.add_argument("--device-sketch-mb", type=int, default=0,
                    help="HBM budget for node sketches (MiB); the rest live in pinned host memory")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if args.workload in ("serve", "failures", "stream_queries", "l0"):
            args.workload = "kron17"
        run_reference(args, rank, world)
    elif args.workload == "serve":
        run_serve(args, rank, world)
    elif args.workload == "failures":
        run_failures(args, rank, world)
    elif args.workload == "stream_queries":
        run_stream_queries(args, rank, world)
    elif args.workload == "l0":
        run_l0(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
