"""Benchmark: HDBSCAN* (default) / EMST throughput in Mpoints/s on one GB300, one JSON line.

Default workload (one step = one full wm_hdbscan call: k-d tree, core distances, MemoGFK rounds
of BCCP* + Kruskal, ordered dendrogram and reachability plot):
  n = 1,000,000 points in d = 3 from a mixture of 50 isotropic Gaussians (centres uniform in
  [0,100)^3, sigmas log-uniform in [0.1, 5], Dirichlet(1) weights) plus 5% uniform noise,
  FP32 coordinates, seed 0, minPts = 10, start point 0.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events on the call's
stream; a 256 MiB buffer is written between steps (outside the events) to flush the 129 MB L2.
value = points processed by all ranks / max-over-ranks time.  `e2e` repeats the step through the
same C ABI with host buffers (pinned input, host outputs), copies inside the timed region.

Multi-GPU: one independent replica per rank ("replicas only": the method has no exchange step),
weak scaling, no collective on the data path.

--impl reference times the FP64 CPU oracle (brute-force Prim etc.) on a bounded sample of the
same workload on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synthdata  # noqa: E402

METRIC = "EMST/HDBSCAN* Mpoints/s on 1 GB300 vs plain form; served p50/p99 latency"
FP32_LANES_PER_SM = 128
N_SM = 152

WORKLOADS = {
    "hdbscan-gmm-1m-3d": dict(problem="hdbscan", gen="gmm", n=1_000_000, d=3, min_pts=10, seed=0),
    "emst-uniform-10k-2d-fp64": dict(problem="emst", gen="uniform64", n=10_000, d=2, seed=0),
    "emst-uniform-10m-2d": dict(problem="emst", gen="uniform", n=10_000_000, d=2, seed=0),
    "emst-uniform-10m-3d": dict(problem="emst", gen="uniform", n=10_000_000, d=3, seed=0),
    "emst-varden-10m-3d": dict(problem="emst", gen="varden", n=10_000_000, d=3, seed=0),
}


def make_points(w):
    if w["gen"] == "gmm":
        return synthdata.gaussian_mixture(w["n"], w["d"], seed=w["seed"])
    if w["gen"] == "uniform64":
        return synthdata.uniform(w["n"], w["d"], seed=w["seed"], dtype=np.float64)
    if w["gen"] == "uniform":
        return synthdata.uniform(w["n"], w["d"], seed=w["seed"], dtype=np.float32)
    if w["gen"] == "varden":
        return synthdata.varden_blobs(w["n"], w["d"], seed=w["seed"])
    raise ValueError(w["gen"])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return self

        def reader():
            for line in self.proc.stdout:
                self.rows.append([c.strip() for c in line.split(",")])
        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def serving_mix(count, seed=0, n_lo=1_000, n_hi=200_000):
    """Requests shaped like the serving configuration: n log-uniform in [n_lo, n_hi], d in
    {2,3,5,7}, minPts in {10,50}, Gaussian-mixture or uniform points, EMST or HDBSCAN*."""
    g = np.random.Generator(np.random.PCG64(seed))
    jobs = []
    for i in range(count):
        n = int(np.exp(g.uniform(np.log(n_lo), np.log(n_hi))))
        d = int(g.choice([2, 3, 5, 7]))
        kind = "emst" if g.random() < 0.5 else "hdbscan"
        mp = int(g.choice([10, 50]))
        if g.random() < 0.5:
            x = synthdata.gaussian_mixture(n, d, seed=seed * 100003 + i)
        else:
            x = synthdata.uniform(n, d, seed=seed * 100003 + i, dtype=np.float32)
        jobs.append((kind, x, mp))
    return jobs


def batched_mix(count, seed=0, n_lo=64, n_hi=65536):
    """Instances shaped like the batched configuration: n log-uniform in [n_lo, n_hi], d in {2,3,5},
    half EMST and half HDBSCAN* (minPts in {5,10,50}), uniform or Gaussian-mixture points."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = int(np.exp(g.uniform(np.log(n_lo), np.log(n_hi))))
        d = int(g.choice([2, 3, 5]))
        mp = 1 if i % 2 == 0 else int(g.choice([5, 10, 50]))
        if g.random() < 0.5:
            x = synthdata.gaussian_mixture(n, d, seed=seed * 100003 + i)
        else:
            x = synthdata.uniform(n, d, seed=seed * 100003 + i, dtype=np.float32)
        out.append((x, min(mp, n), 0))
    return out


def run_batched(wm, torch, count, seed):
    """The batched configuration: all instances in one wm_batch call (device-resident inputs),
    and, on a 64-instance subset, one call per instance against one batched call."""
    inst = batched_mix(count, seed=seed)
    dev = [(torch.from_numpy(x).cuda(), mp, s) for x, mp, s in inst]
    pts = sum(len(x) for x, _, _ in inst)
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sum(ts) / len(ts)

    wm.batch(dev, raw=True)                                           # warm-up (arenas, caches)
    ms = timed(lambda: wm.batch(dev, raw=True), 2)
    sub = [dev[i] for i in np.random.default_rng(seed).choice(len(dev), size=min(64, len(dev)), replace=False)]
    sub_pts = sum(int(x.shape[0]) for x, _, _ in sub)

    def one_at_a_time():
        for x, mp, s in sub:
            if mp <= 1:
                wm.emst(x)
            else:
                wm.hdbscan(x, min_pts=mp, start=s)

    one_at_a_time()
    ms_single = timed(one_at_a_time, 1)
    ms_sub = timed(lambda: wm.batch(sub, raw=True), 2)
    return {"instances": len(inst), "points": pts, "ms": ms, "instances_per_s": len(inst) / (ms * 1e-3),
            "mpoints_per_s": pts / (ms * 1e-3) / 1e6,
            "subset": {"instances": len(sub), "points": sub_pts, "one_call_per_instance_ms": ms_single,
                       "batched_ms": ms_sub, "speedup": ms_single / ms_sub},
            "mix": "n log-uniform [64, 65536], d in {2,3,5}, half EMST and half HDBSCAN* (minPts in {5,10,50}), "
                   "uniform or gmm points; instances with equal minPts share one k-d forest and one set of "
                   "MemoGFK rounds (split by d where a dimension holds >= 2^20 points)"}


def run_serving(wm, jobs, workers, budget, rate_hz=None, seed=1):
    """Submits the jobs (all at once, or as a Poisson stream at rate_hz); returns latencies (ms)
    and the wall time (s)."""
    g = np.random.Generator(np.random.PCG64(seed))
    lat = []
    with wm.Server(hbm_budget_bytes=budget, workers=workers) as srv:
        t0 = time.perf_counter()
        tickets = []
        next_t = t0
        for kind, x, mp in jobs:
            if rate_hz:
                next_t += g.exponential(1.0 / rate_hz)
                delay = next_t - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            tickets.append(srv.submit(x, kind=kind, min_pts=mp))
        failed = 0
        for t in tickets:
            try:
                _, l = srv.wait(t)
                lat.append(l)
            except wm.WMError as e:
                failed += 1
                print(f"served job failed: {e}", file=sys.stderr)
        wall = time.perf_counter() - t0
        peak = srv.counters()
        peak["failed"] = failed
    return np.array(lat), wall, peak


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one bench step, summed over the
# kernel's launches, from the ncu launch list in profiles/launches_hdbscan_gmm_1m_3d.md (cold
# caches under ncu).  A figure is reported only while the kernel's source file is the one that
# was measured (sha256), and only for that workload; otherwise the traffic is null.
MEASURED_TRAFFIC = {
    "bccp": {"bytes": 649192704, "source": "paper_2104_01126_gb300/csrc/wspd.cu",
             "sha256": "37e646b38af4809f57ea97ef9ace2e0e1cdb91f8766807db17c6dbccce8f9518"},
    "getpairs": {"bytes": 2799996416, "source": "paper_2104_01126_gb300/csrc/wspd.cu",
                 "sha256": "37e646b38af4809f57ea97ef9ace2e0e1cdb91f8766807db17c6dbccce8f9518"},
    "knn": {"bytes": 299425792, "source": "paper_2104_01126_gb300/csrc/knn.cu",
            "sha256": "6ae5b2e070e73329be4943549c702cde3167fd62a2199c79ce797dcc00fb3410"},
}
TRAFFIC_WORKLOAD = "hdbscan-gmm-1m-3d"


def measured_traffic(key, workload):
    import hashlib
    t = MEASURED_TRAFFIC.get(key)
    if t is None or workload != TRAFFIC_WORKLOAD:
        return None
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), t["source"]), "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None
    return t["bytes"] if h == t["sha256"] else None


def load_peaks():
    """Measured peaks (MEASURED_PEAKS.json, written by the pool's driver), else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            j = json.load(f)
        return {"hbm_gbs": float(j["hbm_gbs"]), "hbm_basis": "measured (MEASURED_PEAKS.json copy bandwidth)"}
    except Exception:
        return {"hbm_gbs": 6800.0, "hbm_basis": "fallback 6.8 TB/s"}


def max_over_ranks(ms_local: float, dist, device=None) -> float:
    """The step time the job is charged: the maximum over ranks (replicas run independently)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms_local
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(points_per_rank: int, world_size: int, ms_max: float) -> float:
    """Mpoints/s of the whole job: points processed by all ranks over the max-over-ranks time."""
    return points_per_rank * world_size / (ms_max * 1e-3) / 1e6


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_step(w, xs):
    """One run of the FP64 oracle's exact k-d tree solvers (the same results as its brute force,
    pinned to it in tests/test_oracle.py) on the points xs."""
    import oracle
    if w["problem"] == "hdbscan":
        oracle.hdbscan_at_scale(xs, w["min_pts"], s=0)
    else:
        oracle.emst_at_scale(xs)


def run_reference(args, w, ws, rank):
    """The FP64 CPU oracle timed on the workload (its first 10^6 points at most; rank 0 only)."""
    if rank != 0:
        return
    import oracle
    x = make_points(w)
    ns = min(w["n"], args.ref_sample) if args.ref_sample > 0 else min(w["n"], 1_000_000)
    xs = np.ascontiguousarray(x[:ns])
    oracle.build()

    def step():
        oracle_step(w, xs)
    for _ in range(args.warmup if args.ref_warmup is None else args.ref_warmup):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    v = ns / t / 1e6
    cores = os.cpu_count()
    line = {"metric": METRIC, "impl": "reference", "value": v, "unit": "Mpoints/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, **{k: w[k] for k in w if k != "gen"}, "generator": w["gen"],
                       "sample_points": ns},
            "cpu_baseline": {"value": v, "unit": "Mpoints/s", "cores": cores, "kind": "oracle",
                             "sample": f"first {ns} of the {w['n']} points (the generator shuffles rows), "
                                       f"FP64 oracle (exact k-d tree k-NN and Boruvka, plus the dendrogram "
                                       f"and plot for HDBSCAN*), OpenMP on {cores} host threads"},
            "e2e": {"value": v, "unit": "Mpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(w, sample):
    import oracle
    oracle.build()
    x = make_points(w)
    sample = min(w["n"], sample) if sample > 0 else min(w["n"], 1_000_000)
    xs = np.ascontiguousarray(x[:sample])
    t0 = time.perf_counter()
    oracle_step(w, xs)
    t = time.perf_counter() - t0
    cores = os.cpu_count()
    return {"value": sample / t / 1e6, "unit": "Mpoints/s", "cores": cores, "kind": "oracle",
            "sample": f"first {sample} of the {w['n']} points, one run of the FP64 oracle's exact k-d tree "
                      f"solvers ({t:.1f} s, OpenMP on {cores} host threads)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hdbscan-gmm-1m-3d", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--cpu-sample", type=int, default=0, help="points for the CPU baseline (0: min(n, 1e6))")
    ap.add_argument("--ref-sample", type=int, default=0, help="points for --impl reference (0: min(n, 1e6))")
    ap.add_argument("--ref-warmup", type=int, default=None, help="warm-up runs of --impl reference (default: --warmup)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--batch-instances", type=int, default=4096)
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    ws, rank, local = dist_setup()

    if args.impl == "reference":
        run_reference(args, w, ws, rank)
        return

    import torch
    import paper_2104_01126_gb300 as wm
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wm.load()

    x = make_points(w)
    n, d = x.shape
    xd = torch.from_numpy(x).cuda()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step(inp):
        if w["problem"] == "hdbscan":
            return wm.hdbscan(inp, min_pts=w["min_pts"], start=0, precision=args.precision, return_stats=True)
        return wm.emst(inp, precision=args.precision, return_stats=True)

    for _ in range(args.warmup):
        step(xd)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = wm.kernel_launch_count()
    times, stats = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = step(xd)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            stats.append(r["stats"])
    torch.cuda.synchronize()
    launches = wm.kernel_launch_count() - l0
    if dist:
        dist.barrier()
    ms = sum(times) / len(times)
    ms_max = max_over_ranks(ms, dist, device="cuda")
    value = whole_job_value(n, ws, ms_max)

    # ---- roofline: the dominant single kernel (by live CUDA-event time) among those with counted work
    s0 = stats[-1]
    clocks = clk.summary()
    peaks = load_peaks()
    fp32_peak = N_SM * FP32_LANES_PER_SM * 2 * 2.070e9 / 1e12   # TFLOP/s at the maximum SM clock
    dp = 4 if d <= 4 else 8 if d <= 8 else 16
    kernels = []
    if s0.ms_getpairs > 0 and s0.getpairs_visits > 0:
        per = 8 + 2 * 16 + 2 * 16 + 2 * 8 * dp + 16
        gbs = s0.getpairs_visits * per / (s0.ms_getpairs * 1e-3) / 1e9
        kernels.append({"kernel": "findpair_dfs_kernel<1> (GetPairs traversal)", "bound": "hbm",
                        "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                        "traffic": measured_traffic("getpairs", args.workload), "ms": s0.ms_getpairs,
                        "launches": s0.getpairs_launches,
                        "work": f"{s0.getpairs_visits} visited node pairs x {per} B (pair, two links, two meta "
                                f"records holding the component labels, two boxes, two child pairs)",
                        "peak_basis": peaks["hbm_basis"]})
    if s0.ms_knn_kernel > 0:
        fl = s0.knn_evals * (3 * d - 1)
        tf = fl / (s0.ms_knn_kernel * 1e-3) / 1e12
        kernels.append({"kernel": "knn_fast_kernel", "bound": "alu", "achieved": tf, "peak": fp32_peak,
                        "unit": "TFLOP/s", "frac": tf / fp32_peak, "traffic": measured_traffic("knn", args.workload),
                        "ms": s0.ms_knn_kernel,
                        "launches": 1, "work": f"{s0.knn_evals} distance evaluations x {3 * d - 1} flop",
                        "peak_basis": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (max SM clock), derived"})
    if s0.ms_bccp > 0 and s0.bccp_evals > 0:
        per = 3 * d - 1 + (2 if w["problem"] == "hdbscan" else 0)
        tf = s0.bccp_evals * per / (s0.ms_bccp * 1e-3) / 1e12
        kernels.append({"kernel": "bccp_group/pair_tile/dual kernels (all BCCP classes)", "bound": "alu", "achieved": tf,
                        "peak": fp32_peak, "unit": "TFLOP/s", "frac": tf / fp32_peak,
                        "traffic": measured_traffic("bccp", args.workload), "ms": s0.ms_bccp, "launches": None,
                        "aggregate": True,
                        "note": "summed over every BCCP launch of the step (group, tile and dual-tree kernels); "
                                "traffic: DRAM bytes of those launches in one step",
                        "work": f"{s0.bccp_evals} distance evaluations x {per} flop",
                        "peak_basis": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (max SM clock), derived"})
    # the primary entry is the single kernel with the most live time per step; the BCCP entry
    # sums several kernels (size classes), so it is listed in "all" but not chosen
    roof = None
    singles = [k for k in kernels if not k.get("aggregate")]
    if singles:
        roof = dict(max(singles, key=lambda k: k["ms"]))
        roof["all"] = kernels

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(x).pin_memory()
        for _ in range(1):
            step(xh)
        et = []
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step(xh)
            torch.cuda.synchronize()
            et.append(time.perf_counter() - t0)
        e_ms = max_over_ranks(sum(et) / len(et) * 1e3, dist, device="cuda")
        h2d = n * d * x.dtype.itemsize
        if w["problem"] == "hdbscan":
            d2h = (n - 1) * 16 + n * 8 + (n - 1) * 24 + n * 4 + n * 8
        else:
            d2h = (n - 1) * 16 + 8
        e2e = {"value": whole_job_value(n, ws, e_ms), "unit": "Mpoints/s", "ms_per_step": e_ms,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---- the plain form: the same workload in FP64, one job at a time
    plain = None
    if not args.no_plain and args.precision == "fp32":
        saved = args.precision
        args.precision = "fp64"
        step(xd)
        torch.cuda.synchronize()
        pt = []
        for _ in range(max(1, min(args.steps, 2))):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(xd)
            e1.record(stream)
            e1.synchronize()
            pt.append(e0.elapsed_time(e1))
        args.precision = saved
        p_ms = max_over_ranks(sum(pt) / len(pt), dist, device="cuda")
        plain = {"value": whole_job_value(n, ws, p_ms), "unit": "Mpoints/s", "ms_per_step": p_ms,
                 "precision": "fp64", "note": "same workload, every distance in FP64, one job at a time"}

    # ---- served: continuous batching of a mixed request stream
    served = None
    if args.serve_requests > 0:
        jobs = serving_mix(args.serve_requests, seed=rank)
        pts = sum(len(x) for _, x, _ in jobs)
        budget = int(args.serve_budget_gb * (1 << 30))
        run_serving(wm, jobs[: min(8, len(jobs))], args.serve_workers, budget)     # warm-up
        lat_sat, wall_sat, peak_sat = run_serving(wm, jobs, args.serve_workers, budget)
        cap = len(jobs) / wall_sat
        rate = 0.5 * cap
        lat, wall, peak = run_serving(wm, jobs, args.serve_workers, budget, rate_hz=rate, seed=7 + rank)
        served = {"requests": len(jobs), "points": pts, "workers": args.serve_workers,
                  "hbm_budget_gb": args.serve_budget_gb,
                  "saturation": {"jobs_per_s": cap, "mpoints_per_s": pts / wall_sat / 1e6,
                                 "p50_ms": float(np.percentile(lat_sat, 50)),
                                 "p99_ms": float(np.percentile(lat_sat, 99)),
                                 "peak_running": peak_sat["peak_running"]},
                  "rate_hz": rate, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                  "mpoints_per_s": pts / wall / 1e6, "peak_running": peak["peak_running"],
                  "failed": peak["failed"] + peak_sat["failed"],
                  "mix": "n log-uniform [1e3, 2e5], d in {2,3,5,7}, minPts in {10,50}, gmm or uniform, "
                         "EMST or HDBSCAN*; Poisson arrivals at half the measured saturation rate"}

    batched = None
    if args.batch_instances > 0:
        batched = run_batched(wm, torch, args.batch_instances, seed=rank)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_sample)

    if rank == 0:
        cfg = {"workload": args.workload, "n": n, "d": d, "generator": w["gen"], "seed": w["seed"],
               "precision": args.precision, "l2": "256 MiB buffer written between timed steps",
               "parallelism": f"replicas{ws}"}
        if w["problem"] == "hdbscan":
            cfg["min_pts"] = w["min_pts"]
        phases = {k: round(getattr(s0, k), 3) for k in ("ms_build_tree", "ms_core_dist", "ms_wspd", "ms_bccp",
                                                       "ms_kruskal", "ms_dendrogram", "ms_knn_kernel",
                                                       "ms_tile_kernel", "ms_getpairs")}
        counters = {k: int(getattr(s0, k)) for k in ("rounds", "pairs_retrieved", "bccp_evals", "bccp_tile_evals",
                                                    "bccp_dual_evals", "knn_evals", "fp64_rechecks",
                                                    "candidate_edges", "tree_depth", "tile_launches",
                                                    "getpairs_launches", "getpairs_visits", "getrho_visits",
                                                    "rho_shrinks", "max_pending_pairs")}
        line = {"metric": METRIC, "value": value, "unit": "Mpoints/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
                "config": cfg, "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roof,
                "cpu_baseline": cpu, "plain_form": plain, "served": served, "batched": batched,
                "phases_ms": phases,
                "counters": counters,
                "step_ms": [round(t, 3) for t in times]}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
