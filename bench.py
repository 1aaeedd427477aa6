"""Benchmark: exact k-NN queries/s of the Random Ball Cover on one B300.

One step = one exact search (rbc_search) of the whole query batch of the
8-dim-subspace workload (n = 1,048,576 points in R^64, N(0, 0.01) noise,
m = 100,000 queries, n_r = 1024, k = 10, l2, bf16 storage, windowed plan):
stage one BF(Q, R), the own-list bound, pruning and sorted-list windows,
the tensor-core emission pass over (representative, query chunk) windows,
the exact re-rank with FP64 near-ties.  The index is built once before
timing.

Printed JSON line (rank 0): value = queries/s with inputs resident on the
device; e2e = the same call with host (pinned) buffers, copies inside the
timed region; roofline of the dominant kernel (the stage-two tcgen05
emission kernel);
cpu_baseline = the FP64 CPU oracle on a bounded query sample; the FP32
CUDA-core brute force over the same queries for comparison.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Serving mode (--serve): a resident index over the 12-dim sin/cos embedding
workload (n = 8,388,608 points in R^96, fp16 storage, n_r = 2896, k = 10)
behind the library's continuous-batching engine (rbc_server_*).  First the
engine's capacity is measured with a closed loop (64 requests outstanding),
then a Poisson stream of requests of log-uniform size in [1, 4096] queries
is offered at --serve-load (0.7) of that capacity for --serve-seconds (60).
The line reports the served queries/s and the p50 / p99 request latency
(submit to results in pinned host buffers), and checks sampled results
against the FP64 oracle and against the same requests searched alone.

    python bench.py --serve [--serve-seconds S] [--serve-load L]

Grouped mode (--group): 256 independent exact indexes (sizes log-uniform in
[1e3, 2e5], dimensions from {32, 64, 96, 128}, each on its own 8-dim
subspace with N(0, 0.01) noise, fp16 storage, n_r = round(sqrt(n))) with
ragged query batches (log-uniform in [16, 4096] per index), k = 5, searched
together by the grouped search (one persistent stage-two launch, one CUDA
graph per batch shape, autotuned work-item size).  The line reports the
total queries/s of the grouped search next to the same queries searched
index by index with rbc_search.

    python bench.py --group [--group-count N]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
METRIC = "exact k-NN queries/s (RBC BF16+rerank vs FP32 brute force), p50/p99 latency"
FALLBACK_PEAKS = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}
# DRAM bytes (read + write) of one main-pass launch of the emission kernel on
# the default workload, from an ncu capture of the current kernel; None
# whenever the kernel has changed since the counters were taken.
EMIT_TRAFFIC_BYTES = 807_752_960


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="subspace8-n1m-d64")
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--storage", default="bf16", choices=["bf16", "f16", "f32", "fp8"])
    ap.add_argument("--plan", default="window", choices=["window", "tile_union", "window_offset"],
                    help="exact-search stage two (bf16 / fp16 storage)")
    ap.add_argument("--cpu-sample", type=int, default=1000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ref-sample", type=int, default=200)
    ap.add_argument("--legs", default="all", choices=["all", "search"],
                    help="search: only the timed exact-search steps (for profiler launch lists)")
    ap.add_argument("--n", type=int, default=None, help="override the database size")
    ap.add_argument("--m", type=int, default=None, help="override the query batch size")
    ap.add_argument("--serve", action="store_true", help="serving measurement instead of batch search")
    ap.add_argument("--serve-workload", default="sincos12-n8m-d96")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-capacity-seconds", type=float, default=8.0)
    ap.add_argument("--serve-load", type=float, default=0.7)
    ap.add_argument("--serve-workers", type=int, default=3)
    ap.add_argument("--serve-max-batch", type=int, default=16384)
    ap.add_argument("--serve-check", type=int, default=24, help="rows checked against the oracle")
    ap.add_argument("--group", action="store_true", help="grouped multi-index search measurement")
    ap.add_argument("--group-count", type=int, default=256)
    ap.add_argument("--variants", action="store_true",
                    help="the other search modes on the same workload: exact L1 (CUDA cores) and "
                         "one-shot L2 (recall against the exact answer)")
    ap.add_argument("--oneshot-s", type=int, default=0, help="one-shot list size s (0: n_r)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_query_seed(rank: int) -> int:
    """Each rank searches its own query batch of the workload (weak scaling)."""
    return 1 + 1000 * rank


def ranks_max(value: float, device=None) -> float:
    """The largest value over the ranks of the default process group (the
    slowest rank's time); the value itself without one."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_qps(world: int, m: int, steps: int, elapsed_ms: float) -> float:
    """Whole-job queries/s: every rank searched m queries per step, the job
    took the slowest rank's time."""
    return world * m * steps / (elapsed_ms / 1000.0)


def load_peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return FALLBACK_PEAKS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_arrays(name: str, seed: int, m: int | None = None, query_seed: int | None = None,
                    n: int | None = None):
    w = synth.WORKLOADS[name]
    X, Q = synth.make_workload(w, seed=seed, n=n, m=m, query_seed=query_seed)
    return w, X, Q


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle (as it stands) on the host cores
# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle

    w, X, Q = workload_arrays(args.workload, 0)
    reps = oracle.sample_reps(len(X), w.n_r, 2)
    idx = oracle.build_exact(X, reps, "l2")
    cores = oracle.num_threads()
    S = args.ref_sample
    g = np.random.default_rng(7)
    times = []
    for step in range(args.warmup + args.steps):
        sel = np.sort(g.choice(len(Q), S, replace=False))
        t0 = time.perf_counter()
        oracle.search_exact(idx, Q[sel], args.k)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    total = sum(times)
    qps = S * len(times) / total
    out = {
        "impl": "reference",
        "metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        # the same workload and search as the GPU arm's line (its config keys
        # verbatim); the oracle computes that search's exact answer in FP64
        "config": {"workload": args.workload, "n": w.n, "m": w.m, "d": w.d, "n_r": w.n_r, "k": args.k,
                   "metric": "l2", "storage": args.storage, "plan": args.plan,
                   "noise_var": w.params.get("noise_var"),
                   "intrinsic_dim": w.params.get("k"), "parallelism": "replicas1",
                   "l2_flush": "inputs larger than L2 (bf16 database 128 MiB + FP32 copy 256 MiB)"},
        "method": "exact RBC search, FP64 CPU oracle",
        "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": cores, "kind": "oracle",
                         "sample": f"{S} random queries of {w.m} per step, full {w.n}-point database"},
        "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local):
    import torch

    import paper_1103_2635_b300 as rbc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    storage = {"bf16": rbc.BF16, "f16": rbc.F16, "f32": rbc.F32, "fp8": rbc.FP8E4M3}[args.storage]
    # each rank holds its own replica and its own query batch (weak scaling)
    w, X, Q = workload_arrays(args.workload, 0, query_seed=rank_query_seed(rank), n=args.n, m=args.m)
    Xd = torch.from_numpy(X).to(dev)
    Qd = torch.from_numpy(Q).to(dev)
    m, d, k = Q.shape[0], Q.shape[1], args.k
    st = torch.cuda.current_stream(dev)

    t0 = time.perf_counter()
    plan = {"window": rbc.PLAN_WINDOW, "tile_union": rbc.PLAN_TILE_UNION,
            "window_offset": rbc.PLAN_WINDOW_OFFSET}[args.plan]
    idx = rbc.rbc_build(Xd, w.n_r, metric=rbc.L2, seed=2, storage=storage, plan=plan)
    torch.cuda.synchronize(dev)
    build_s = time.perf_counter() - t0

    ids = torch.empty((m, k), dtype=torch.int64, device=dev)
    dist_ = torch.empty((m, k), dtype=torch.float32, device=dev)

    def step():
        rbc.rbc_search(idx, Qd, k, out_ids=ids, out_dist=dist_)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    launches_per_step = rbc.last_stats()["kernel_launches"]

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    # ---- device-resident timed region ----
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize(dev)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        evs[0].record(st)
        for i in range(args.steps):
            step()
            evs[i + 1].record(st)
        torch.cuda.synchronize(dev)
        barrier()
    launches = launches_per_step * args.steps
    elapsed_ms = evs[0].elapsed_time(evs[-1])
    step_ms = sorted(evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps))
    lat = {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
           "unit": "ms per batch of %d queries" % m}
    if world > 1:
        elapsed_ms = ranks_max(elapsed_ms, dev)
    stats = rbc.last_stats()
    qps = weak_scaling_qps(world, m, args.steps, elapsed_ms)
    if args.legs == "search":
        if rank == 0:
            print(json.dumps({"legs": "search", "value": qps, "unit": "queries/s",
                              "ms_per_step": elapsed_ms / args.steps, "n": len(X), "m": m, "k": k,
                              "gpu_launches": launches}), flush=True)
        return

    # ---- phase timing (separate pass: events around each phase) ----
    rbc.set_timing(True)
    ph = {"stage1_ms": 0.0, "stage2_ms": 0.0, "select_ms": 0.0, "fallback_ms": 0.0}
    pairs = 0
    nt = max(3, min(args.steps, 5))
    for _ in range(nt):
        step()
        s = rbc.last_stats()
        for key in ph:
            ph[key] += s[key] / nt
        pairs = s["pairs"]
    rbc.set_timing(False)

    # ---- end-to-end through the C ABI with host buffers ----
    Qh = torch.from_numpy(Q).pin_memory()
    ids_h = torch.empty((m, k), dtype=torch.int64).pin_memory()
    dist_h = torch.empty((m, k), dtype=torch.float32).pin_memory()
    Qh_np, ids_np, dist_np = Qh.numpy(), ids_h.numpy(), dist_h.numpy()
    for _ in range(2):
        rbc.rbc_search(idx, Qh_np, k, out_ids=ids_np, out_dist=dist_np)
    torch.cuda.synchronize(dev)
    e2e_steps = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        rbc.rbc_search(idx, Qh_np, k, out_ids=ids_np, out_dist=dist_np)
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    e2e_s = ranks_max(e2e_s, dev)  # the slowest rank
    e2e_qps = weak_scaling_qps(world, m, e2e_steps, e2e_s * 1e3)
    same = bool((ids_h.numpy() == ids.cpu().numpy()).all())

    # ---- plain FP32 CUDA-core brute force on the same queries ----
    fp32_m = min(m, 20000)
    Qs = Qd[:fp32_m].contiguous()
    rbc.bf_search(Qs, Xd, k, metric=rbc.L2, storage=rbc.F32)
    torch.cuda.synchronize(dev)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(st)
    bf_ids, bf_dist = rbc.bf_search(Qs, Xd, k, metric=rbc.L2, storage=rbc.F32)
    f1.record(st)
    torch.cuda.synchronize(dev)
    fp32_qps = fp32_m / (f0.elapsed_time(f1) / 1000.0)
    agree = float((bf_ids.cpu().numpy() == ids[:fp32_m].cpu().numpy()).all(axis=1).mean())

    # ---- dense BF16 brute force (tensor cores) on the same queries ----
    rbc.set_timing(True)
    bf16_ids, _ = rbc.bf_search(Qd, Xd, k, metric=rbc.L2, storage=rbc.BF16)
    torch.cuda.synchronize(dev)
    b0 = torch.cuda.Event(enable_timing=True)
    b1 = torch.cuda.Event(enable_timing=True)
    b0.record(st)
    rbc.bf_search(Qd, Xd, k, metric=rbc.L2, storage=rbc.BF16)
    b1.record(st)
    bst = rbc.last_stats()
    rbc.set_timing(False)
    torch.cuda.synchronize(dev)
    bf16_qps = m / (b0.elapsed_time(b1) / 1000.0)

    peaks, peak_src = load_peaks()
    flops_per_pair = 2 * d
    # dominant kernel: the stage-two tcgen05 emission kernel, timed with
    # events on its stream inside the library; algorithmic work = the
    # (query, window row) pairs of its work items x 2 d flops
    tflops = pairs * flops_per_pair / (ph["stage2_ms"] / 1000.0) / 1e12 if ph["stage2_ms"] > 0 else None
    # the kernel runs for milliseconds inside a short step: the burst peak
    peak = peaks.get("bf16_tflops")
    peak_sus = peaks.get("bf16_tflops_sustained", peak)
    dense_tflops = m * len(X) * flops_per_pair / (bst["stage2_ms"] / 1000.0) / 1e12 if bst["stage2_ms"] else None
    roofline = {
        "bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
        "frac": (tflops / peak) if tflops else None,
        "traffic": EMIT_TRAFFIC_BYTES if (args.workload == "subspace8-n1m-d64" and args.n is None
                                          and args.m is None and args.storage == "bf16"
                                          and args.plan == "window" and k == 10) else None,
        "kernel": "bf_tc_emit_kernel (stage two: query chunks x sorted-list windows)",
        "peak_source": f"{peak_src} bf16 burst (cuBLAS), of {peak_src}",
        "frac_of_sustained": (tflops / peak_sus) if tflops else None,
        "flops_per_launch": pairs * flops_per_pair, "launch_ms": ph["stage2_ms"],
        "dense_bf16_bf": {"achieved": dense_tflops, "frac": (dense_tflops / peak) if dense_tflops else None,
                          "launch_ms": bst["stage2_ms"]},
    }

    # ---- CPU oracle baseline on a bounded sample (rank 0, N = 1) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle

        S = min(args.cpu_sample, m)
        g = np.random.default_rng(11)
        sel = np.sort(g.choice(m, S, replace=False))
        reps = oracle.sample_reps(len(X), w.n_r, 2)
        oidx = oracle.build_exact(X, reps, "l2")
        t0 = time.perf_counter()
        o_ids, o_rho, _ = oracle.search_exact(oidx, Q[sel], k)
        cpu_s = time.perf_counter() - t0
        g_ids = ids.cpu().numpy()[sel]
        g_d = dist_.cpu().numpy()[sel].astype(np.float64)
        rel = np.abs(g_d - o_rho) / np.maximum(o_rho, 1e-30)
        cpu = {"value": S / cpu_s, "unit": "queries/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"{S} random queries of {m} (seed 11), exact RBC search (FP64) against the full "
                         f"{len(X)}-point database; index built outside the timed region",
               "parity_on_sample": {"rows_ids_equal": float((g_ids == o_ids).all(axis=1).mean()),
                                    "max_rel_dist_err": float(rel.max())}}

    out = {
        "metric": METRIC,
        "value": qps, "unit": "queries/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps, "latency": lat, "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
        "config": {"workload": args.workload, "n": len(X), "m": m, "d": d, "n_r": w.n_r, "k": k,
                   "metric": "l2", "storage": args.storage, "plan": args.plan,
                   "noise_var": w.params.get("noise_var"),
                   "intrinsic_dim": w.params.get("k"), "parallelism": f"replicas{world}",
                   "l2_flush": "inputs larger than L2 (bf16 database 128 MiB + FP32 copy 256 MiB)"},
        "clocks": clk.summary(),
        "gpu_launches": launches,
        "e2e": {"value": e2e_qps, "unit": "queries/s", "h2d_bytes_per_step": m * d * 4,
                "d2h_bytes_per_step": m * k * 12, "matches_device_run": same},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "fp32_bruteforce": {"value": fp32_qps, "unit": "queries/s", "queries": fp32_m,
                            "rows_equal_to_rbc": agree},
        "bf16_bruteforce": {"value": bf16_qps, "unit": "queries/s",
                            "rows_equal_to_rbc": float((bf16_ids.cpu().numpy() == ids.cpu().numpy()).all(axis=1).mean())},
        "speedup_vs_fp32_bruteforce": qps / fp32_qps,
        "phases_ms": ph,
        "stats": {"kept_reps_per_query": stats["kept_reps"] / m,
                  "examined_per_query": pairs / m if pairs else None,
                  "uncertified": stats["uncertified"], "fp64_ties": stats["fp64_ties"],
                  "boundary_ties": stats["boundary_ties"]},
        "build_s": build_s,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# serving: continuous batching under a Poisson request stream
# ---------------------------------------------------------------------------
def run_serve(args, rank, world, local):
    if rank != 0:
        return
    import threading

    import torch

    import paper_1103_2635_b300 as rbc

    torch.cuda.set_device(local)
    k = args.k
    w = synth.WORKLOADS[args.serve_workload]
    pool_m = 1 << 18
    X, Qpool = synth.make_workload(w, seed=0, n=args.n, m=pool_m)
    n = len(X)
    t0 = time.perf_counter()
    idx = rbc.rbc_build(torch.from_numpy(X).cuda(), w.n_r, seed=2, storage=rbc.F16)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    Qpin = torch.from_numpy(Qpool).pin_memory()
    ring = 1 << 22
    ids_ring = torch.empty((ring, k), dtype=torch.int64).pin_memory()
    dist_ring = torch.empty((ring, k), dtype=torch.float32).pin_memory()
    rng = np.random.default_rng(11)

    def draw_size():
        return int(min(4096, max(1, np.exp(rng.uniform(0.0, np.log(4097.0))))))

    mean_size = 4096 / np.log(4097.0)  # E[exp(U(0, ln 4097))] - 1/2 flooring, about 492
    srv = rbc.Server(idx, workers=args.serve_workers, max_batch=args.serve_max_batch, k_max=k)
    state = {"off": 0}
    pending = []
    lock = threading.Condition()
    kept = []  # (qstart, m, ticket-result slice) of a few requests for checks

    def submit(m):
        s = int(rng.integers(0, pool_m - m + 1))
        off = state["off"]
        if off + m > ring:
            off = 0
        state["off"] = off + m
        t = srv.submit(Qpin[s : s + m], k, ids_ring[off : off + m], dist_ring[off : off + m])
        return t, s, off, m

    def collector(stop):
        while True:
            with lock:
                while not pending and not stop["v"]:
                    lock.wait()
                if not pending and stop["v"]:
                    return
                t, s, off, m = pending.pop(0)
            ids, dist, info = srv.wait(t)
            if len(kept) < 64 and info["batch_requests"] > 1:
                kept.append((s, m, ids.numpy().copy(), dist.numpy().copy()))

    def run_phase(seconds, rate=None, depth=64):
        stop = {"v": False}
        th = threading.Thread(target=collector, args=(stop,))
        th.start()
        srv.stats(reset=True)
        t_start = time.perf_counter()
        submitted = q_sub = 0
        next_t = t_start
        while True:
            now = time.perf_counter()
            if now - t_start >= seconds:
                break
            if rate is None:  # closed loop: keep `depth` requests outstanding
                with lock:
                    backlog = len(pending)
                if backlog >= depth:
                    time.sleep(0.0002)
                    continue
            else:
                if now < next_t:
                    dt = next_t - now
                    if dt > 0.001:
                        time.sleep(dt - 0.0005)
                    continue
                next_t += rng.exponential(1.0 / rate)
            m = draw_size()
            item = submit(m)
            with lock:
                pending.append(item)
                lock.notify()
            submitted += 1
            q_sub += m
        offered_s = time.perf_counter() - t_start
        with lock:
            stop["v"] = True
            lock.notify()
        th.join()
        st = srv.stats(reset=False)
        return st, submitted, q_sub, offered_s

    # warm-up, then capacity (closed loop), then the Poisson stream
    run_phase(2.0)
    cap, _, _, _ = run_phase(args.serve_capacity_seconds)
    capacity = cap["queries_per_s"]
    rate = args.serve_load * capacity / mean_size  # requests per second
    dev = torch.cuda.current_device()
    with ClockSampler(dev) as clk:
        st, submitted, q_sub, offered_s = run_phase(args.serve_seconds, rate=rate)
    clocks = clk.summary()
    srv.close()

    # checks: sampled rows against the FP64 oracle; merged requests against
    # the same queries searched alone
    import oracle

    bad_alone = 0
    for s, m, ids, dist in kept[:16]:
        ia, da = rbc.rbc_search(idx, Qpin[s : s + m].cuda(), k)
        torch.cuda.synchronize()
        ia, da = ia.cpu().numpy(), da.cpu().numpy()
        same = np.array_equal(ids, ia) and np.allclose(dist, da, rtol=1e-5, atol=0)
        bad_alone += 0 if same else 1
    rows, got_i, got_d = [], [], []
    for s, m, ids, dist in kept:
        if len(rows) >= args.serve_check:
            break
        j = m // 2
        rows.append(s + j)
        got_i.append(ids[j])
        got_d.append(dist[j])
    parity = {"checked_rows": len(rows), "alone_vs_mix_requests": min(16, len(kept)),
              "alone_vs_mix_mismatch": bad_alone}
    if rows:
        o_ids, o_rho = oracle.bf(Qpool[rows], X, k)
        gi, gd = np.array(got_i), np.array(got_d, dtype=np.float64)
        parity["ids_equal_rows"] = int(np.sum(np.all(gi == o_ids, axis=1)))
        parity["max_rel_dist_err"] = float(np.max(np.abs(gd - o_rho) / np.maximum(o_rho, 1e-30)))
    line = {
        "metric": "serving: queries/s with p50/p99 request latency under a Poisson stream of "
                  "1-4096-query requests (exact k-NN, RBC fp16 + rerank)",
        "value": st["queries_per_s"], "unit": "queries/s", "higher_is_better": True,
        "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"], "max_ms": st["max_ms"],
        "queue_p50_ms": st["queue_p50_ms"], "queue_p99_ms": st["queue_p99_ms"],
        "capacity_qps": capacity, "capacity_p50_ms": cap["p50_ms"], "capacity_p99_ms": cap["p99_ms"],
        "offered_qps": q_sub / offered_s, "load": args.serve_load,
        "requests": st["requests"], "queries": st["queries"], "batches": st["batches"],
        "mean_batch_queries": st["mean_batch_queries"], "max_in_flight": st["max_in_flight"],
        "peak_reserved_bytes": st["peak_reserved_bytes"], "hbm_budget": st["hbm_budget"],
        "n_gpus": 1, "dtype": "f16", "data": "synthetic", "clocks": clocks, "parity": parity,
        "config": {"workload": args.serve_workload, "n": n, "d": w.d, "n_r": w.n_r, "k": k,
                   "storage": "f16", "workers": args.serve_workers,
                   "max_batch": args.serve_max_batch, "seconds": args.serve_seconds,
                   "request_sizes": "log-uniform [1, 4096]", "arrivals": "Poisson",
                   "build_s": build_s, "host_buffers": "pinned"},
    }
    print(json.dumps(line), flush=True)
    idx.close()


# ---------------------------------------------------------------------------
# grouped multi-index search
# ---------------------------------------------------------------------------
def run_group(args, rank, world, local):
    if rank != 0:
        return
    import torch

    import paper_1103_2635_b300 as rbc

    torch.cuda.set_device(local)
    k = 5
    rng = np.random.default_rng(4)
    Xs, Qs, idxs, meta = [], [], [], []
    t0 = time.perf_counter()
    for i in range(args.group_count):
        n = int(round(np.exp(rng.uniform(np.log(1e3), np.log(2e5)))))
        d = int(rng.choice([32, 64, 96, 128]))
        m = int(round(np.exp(rng.uniform(np.log(16), np.log(4096)))))
        mod = synth.SubspaceModel(d=d, k=8, noise_var=0.01, seed=10_000 + i)
        X, Q = mod.sample(n, 2 * i), mod.sample(m, 2 * i + 1)
        idx = rbc.rbc_build(torch.from_numpy(X).cuda(), int(round(np.sqrt(n))), seed=i,
                            storage=rbc.F16)
        Xs.append(X)
        Qs.append(Q)
        idxs.append(idx)
        meta.append((n, d, m))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    g = rbc.Group(idxs)
    Qd = [torch.from_numpy(Q).cuda() for Q in Qs]
    M = sum(len(Q) for Q in Qs)
    W = g.tune(Qd, k)
    stream = torch.cuda.current_stream()

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times = []
        for _ in range(steps):
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        return times

    dev = torch.cuda.current_device()
    with ClockSampler(dev) as clk:
        t_group = timed(lambda: g.search(Qd, k), args.steps, args.warmup)
    clocks = clk.summary()
    st = g.stats()
    t_seq = timed(lambda: [rbc.rbc_search(ix, Q, k) for ix, Q in zip(idxs, Qd)], max(3, args.steps // 3), 2)
    # e2e: each index's queries in pinned host memory, one pointer per index,
    # results into pinned host buffers
    Qh = [torch.from_numpy(np.ascontiguousarray(Q)).pin_memory() for Q in Qs]
    oi = torch.empty((M, k), dtype=torch.int64).pin_memory()
    od = torch.empty((M, k), dtype=torch.float32).pin_memory()
    t_e2e = timed(lambda: g.search(Qh, k, out_ids=oi, out_dist=od), max(3, args.steps // 3), 1)
    # parity: every index alone on the GPU, and the FP64 oracle on sampled rows
    # (this search is marked as an NVTX range, for profiler launch lists)
    torch.cuda.nvtx.range_push("group_search")
    ids, dist = g.search(Qd, k)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    import oracle

    alone_equal = 0
    for i in range(len(idxs)):
        ia, da = rbc.rbc_search(idxs[i], Qd[i], k)
        alone_equal += int(torch.equal(ia, ids[i]))
    sample_rows = ok_rows = 0
    max_err = 0.0
    for i in range(0, len(idxs), 16):
        rows = np.unique(np.linspace(0, len(Qs[i]) - 1, min(len(Qs[i]), 8)).astype(int))
        o_ids, o_rho = oracle.bf(Qs[i][rows], Xs[i], k)
        gi, gd = ids[i].cpu().numpy()[rows], dist[i].cpu().numpy()[rows].astype(np.float64)
        sample_rows += len(rows)
        ok_rows += int(np.sum(np.all(gi == o_ids, axis=1)))
        max_err = max(max_err, float(np.max(np.abs(gd - o_rho) / np.maximum(o_rho, 1e-30))))
    med = float(np.median(t_group))
    line = {
        "metric": "grouped exact k-NN queries/s over 256 independent RBC indexes (one persistent "
                  "stage-two launch, CUDA graph)",
        "value": M / (med / 1e3), "unit": "queries/s", "higher_is_better": True,
        "ms_per_step": med, "p99_ms": float(np.percentile(t_group, 99)), "steps": args.steps,
        "warmup": args.warmup, "n_gpus": 1, "dtype": "f16", "data": "synthetic",
        "sequential_rbc_search": {"value": M / (float(np.median(t_seq)) / 1e3), "unit": "queries/s",
                                  "ms_per_step": float(np.median(t_seq))},
        "e2e": {"value": M / (float(np.median(t_e2e)) / 1e3), "unit": "queries/s",
                "h2d_bytes_per_step": int(sum(Q.numel() * 4 for Q in Qh)),
                "d2h_bytes_per_step": int(M * k * 12)},
        "autotuned_work_item_points": W, "clocks": clocks,
        "stats": {kk: st[kk] for kk in ("tiles", "work_items", "uncertified", "fp64_ties", "graph_replays")},
        "parity": {"indexes_equal_to_rbc_search": alone_equal, "indexes": len(idxs),
                   "oracle_rows_equal": ok_rows, "oracle_rows": sample_rows,
                   "max_rel_dist_err": max_err},
        "config": {"workload": "256 subspace8 indexes, n log-uniform [1e3, 2e5], d in {32,64,96,128}",
                   "indexes": len(idxs), "total_points": int(sum(x[0] for x in meta)),
                   "total_queries": M, "k": k, "storage": "f16", "build_s": build_s,
                   "l2_flush": "padded fp32 rows of the group 4.9 GB > L2"},
    }
    print(json.dumps(line), flush=True)
    g.close()
    for ix in idxs:
        ix.close()


# ---------------------------------------------------------------------------
# the other search modes: exact L1 search and one-shot search
# ---------------------------------------------------------------------------
def run_variants(args, rank, world, local):
    """Exact L1 RBC (FP32, CUDA cores) against the L1 FP32 brute force, and
    one-shot RBC (Section 5.1, bf16) with its recall against the exact
    answer, on the same workload and query batch as the main bench line."""
    if rank != 0:
        return
    import torch

    import oracle
    import paper_1103_2635_b300 as rbc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w, X, Q = workload_arrays(args.workload, 0, query_seed=rank_query_seed(rank), n=args.n, m=args.m)
    Xd, Qd = torch.from_numpy(X).to(dev), torch.from_numpy(Q).to(dev)
    m, k = len(Q), args.k
    st = torch.cuda.current_stream(dev)

    def timed(fn, steps):
        for _ in range(args.warmup):
            out = fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            out = fn()
        e1.record(st)
        torch.cuda.synchronize(dev)
        return out, e0.elapsed_time(e1) / steps

    g = np.random.default_rng(11)
    sel = np.sort(g.choice(m, min(m, 200), replace=False))
    res = {}
    with ClockSampler(local) as clk:
        # exact L1
        idx1 = rbc.rbc_build(Xd, w.n_r, metric=rbc.L1, seed=2, storage=rbc.F32)
        (ids1, d1), ms1 = timed(lambda: rbc.rbc_search(idx1, Qd, k), args.steps)
        st1 = rbc.last_stats()
        bf_m = min(m, 20000)
        (bids, _), msb = timed(lambda: rbc.bf_search(Qd[:bf_m], Xd, k, metric=rbc.L1, storage=rbc.F32), 1)
        o_ids, o_rho = oracle.bf(Q[sel], X, k, "l1")
        g1 = ids1.cpu().numpy()
        rel = np.abs(d1.cpu().numpy()[sel].astype(np.float64) - o_rho) / np.maximum(o_rho, 1e-30)
        res["l1_exact"] = {
            "value": m / (ms1 / 1e3), "unit": "queries/s", "ms_per_step": ms1, "storage": "f32",
            "kept_reps_per_query": st1["kept_reps"] / m, "pairs_per_query": st1["pairs"] / m,
            "fp32_bruteforce_qps": bf_m / (msb / 1e3),
            "speedup_vs_fp32_bruteforce": (m / ms1) / (bf_m / msb),
            "rows_equal_to_bruteforce": float((bids.cpu().numpy() == g1[:bf_m]).all(axis=1).mean()),
            "oracle_sample": {"rows": len(sel), "rows_ids_equal": float((g1[sel] == o_ids).all(axis=1).mean()),
                              "max_rel_dist_err": float(rel.max())}}
        idx1.close()
        # one-shot L2 (and the exact answer it is compared with)
        s_ = args.oneshot_s or w.n_r
        idxe = rbc.rbc_build(Xd, w.n_r, metric=rbc.L2, seed=2, storage=rbc.BF16)
        ids_e, _ = rbc.rbc_search(idxe, Qd, k)
        ids_e = ids_e.cpu().numpy()
        idxe.close()
        t0 = time.perf_counter()
        idxo = rbc.rbc_build(Xd, w.n_r, metric=rbc.L2, seed=2, storage=rbc.BF16, mode=rbc.ONESHOT, s=s_)
        torch.cuda.synchronize(dev)
        build_s = time.perf_counter() - t0
        (ids_o, d_o), mso = timed(lambda: rbc.rbc_search(idxo, Qd, k), args.steps)
        go = ids_o.cpu().numpy()
        hits = sum(len(np.intersect1d(a, b)) for a, b in zip(go, ids_e))
        # parity of the one-shot answer with the oracle's one-shot search on the sample
        reps = oracle.sample_reps(len(X), w.n_r, 2)
        oo = oracle.build_oneshot(X, reps, s_, "l2")
        oo_ids, oo_rho = oracle.search_oneshot(oo, Q[sel], k)[:2]
        rel = np.abs(d_o.cpu().numpy()[sel].astype(np.float64) - oo_rho) / np.maximum(oo_rho, 1e-30)
        # Section 7.2's quality measure: the rank of the returned nearest
        # neighbour among all database points (0 = the true nearest)
        ranks = oracle.rank_of(Q[sel], X, go[sel, 0], "l2")
        res["oneshot"] = {
            "value": m / (mso / 1e3), "unit": "queries/s", "ms_per_step": mso, "storage": "bf16", "s": s_,
            "build_s": build_s, "recall_at_k_vs_exact": hits / (m * k),
            "rows_equal_to_exact": float((go == ids_e).all(axis=1).mean()),
            "rank_of_first_on_sample": {"mean": float(ranks.mean()), "exact_fraction": float((ranks == 0).mean())},
            "oracle_oneshot_sample": {"rows": len(sel),
                                      "rows_ids_equal": float((go[sel] == oo_ids).all(axis=1).mean()),
                                      "max_rel_dist_err": float(rel.max())}}
        idxo.close()
    line = {"mode": "variants", "workload": args.workload, "n": len(X), "m": m, "d": w.d, "n_r": w.n_r,
            "k": k, "steps": args.steps, "warmup": args.warmup, "n_gpus": 1, "data": "synthetic",
            "clocks": clk.summary(), **res}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.variants:
        run_variants(args, rank, world, local)
        return
    if args.group:
        run_group(args, rank, world, local)
        return
    if args.serve:
        run_serve(args, rank, world, local)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
