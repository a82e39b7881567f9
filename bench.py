"""Benchmark: EMST / HDBSCAN* throughput in Mpoints/s on one GB300, one JSON line.

Headline workload (one step = eight full wm_emst calls, one per point set): the EMST at scale,
n = 10,000,000 points in d = 2, 3, 5 and 7 from two generators, i.i.d. uniform in [0,1)^d and
variable-density blobs (1,000 Gaussian blobs, sigmas log-uniform over three decades, Zipf(1.1)
sizes), FP32 coordinates, seed 0, FP32 screening with FP64 winners.  value = the points of all
eight calls over the summed time of the eight calls (Mpoints/s), across all ranks.

Timing: W untimed warm-up steps, then K steps; each call is bracketed by CUDA events on the
call's stream, and a 256 MiB buffer is written before every call (outside the events) to flush
the 129 MB L2.  `e2e` repeats the calls through the same C ABI from pinned host buffers into host
outputs, copies inside the timed region.  Further keys: `roofline` (the kernel with the most
device time, every kernel's figures in `roofline.all`), `cpu_baseline` (the FP64 oracle on a
sample), `plain_form` (the same workloads with every distance in FP64), `cfg2` (HDBSCAN* on 10^6
Gaussian-mixture points), `served` (a Poisson rate sweep of mixed requests against the plain
one-job-at-a-time FP64 server) and `batched` (4,096 small instances in one call).

Multi-GPU: one independent replica per rank ("replicas only": the method has no exchange step),
weak scaling, no collective on the data path.

--impl reference times the FP64 CPU oracle (exact k-d tree solvers) on a bounded sample of each
workload on this host's cores.
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

SCALE_DIMS = (2, 3, 5, 7)
SCALE_GENS = ("uniform", "varden")
WORKLOADS = {f"emst-{g}-10m-{d}d": dict(problem="emst", gen=g, n=10_000_000, d=d, seed=0)
             for g in SCALE_GENS for d in SCALE_DIMS}
WORKLOADS["hdbscan-gmm-1m-3d"] = dict(problem="hdbscan", gen="gmm", n=1_000_000, d=3, min_pts=10, seed=0)
WORKLOADS["emst-uniform-10k-2d-fp64"] = dict(problem="emst", gen="uniform64", n=10_000, d=2, seed=0)
# the headline: the largest single-GPU configuration, all eight 10^7-point sets
SUITES = {"emst-10m-suite": [f"emst-{g}-10m-{d}d" for g in SCALE_GENS for d in SCALE_DIMS]}
CFG2 = "hdbscan-gmm-1m-3d"


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


def workload_names(name):
    return SUITES.get(name, [name])


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


# ------------------------------------------------------------------------------ request mixes
def serving_pool(size, seed=0, n_lo=1_000, n_hi=2_000_000):
    """Point sets shaped like the serving configuration: n log-uniform in [n_lo, n_hi], d in
    {2,3,5,7}, Gaussian-mixture or uniform points; each comes with a problem (EMST or HDBSCAN*)
    and minPts in {10, 50}."""
    g = np.random.Generator(np.random.PCG64(seed))
    pool = []
    for i in range(size):
        n = int(np.exp(g.uniform(np.log(n_lo), np.log(n_hi))))
        d = int(g.choice([2, 3, 5, 7]))
        kind = "emst" if g.random() < 0.5 else "hdbscan"
        mp = int(g.choice([10, 50]))
        if g.random() < 0.5:
            x = synthdata.gaussian_mixture(n, d, seed=seed * 100003 + i)
        else:
            x = synthdata.uniform(n, d, seed=seed * 100003 + i, dtype=np.float32)
        pool.append((kind, x, mp))
    return pool


def request_stream(pool, count, seed):
    """count requests drawn uniformly (seeded) from the pool."""
    g = np.random.Generator(np.random.PCG64(seed))
    return [pool[int(i)] for i in g.integers(0, len(pool), size=count)]


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


def run_serving(wm, jobs, workers, budget, rate_hz=None, seed=1, precision="fp32"):
    """Submits the jobs (all at once, or as a Poisson stream at rate_hz); returns latencies (ms),
    the wall time (s) and the server's counters."""
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
            tickets.append(srv.submit(x, kind=kind, min_pts=mp, precision=precision))
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


def serving_sweep(wm, args, rank):
    """The serving configuration: Poisson arrivals at rates swept around the continuous-batching
    server's saturation, against the plain form (one job at a time, every distance in FP64) at
    the lowest rate."""
    pool = serving_pool(args.serve_pool, seed=rank)
    budget = int(args.serve_budget_gb * (1 << 30))
    run_serving(wm, pool[:8], args.serve_workers, budget)                       # warm-up
    sat_jobs = request_stream(pool, args.serve_requests, seed=11 + rank)
    lat, wall, peak = run_serving(wm, sat_jobs, args.serve_workers, budget)
    cap = len(sat_jobs) / wall
    pts_per_job = float(np.mean([len(x) for _, x, _ in sat_jobs]))
    out = {"pool": args.serve_pool, "requests_per_rate": args.serve_requests, "workers": args.serve_workers,
           "hbm_budget_gb": args.serve_budget_gb,
           "saturation": {"jobs_per_s": cap, "mpoints_per_s": cap * pts_per_job / 1e6,
                          "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                          "peak_running": peak["peak_running"], "failed": peak["failed"]},
           "rates": [],
           "mix": "n log-uniform [1e3, 2e6], d in {2,3,5,7}, minPts in {10,50}, gmm or uniform points, "
                  "EMST or HDBSCAN*; each request drawn from a pool of generated point sets; Poisson arrivals"}
    fracs = [float(f) for f in args.serve_rates.split(",") if f]
    for i, f in enumerate(fracs):
        jobs = request_stream(pool, args.serve_requests, seed=100 + 7 * i + rank)
        rate = f * cap
        lat, wall, peak = run_serving(wm, jobs, args.serve_workers, budget, rate_hz=rate, seed=7 + i + rank)
        pts = sum(len(x) for _, x, _ in jobs)
        out["rates"].append({"fraction_of_saturation": f, "rate_hz": rate, "requests": len(jobs),
                             "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                             "mpoints_per_s": pts / wall / 1e6, "peak_running": peak["peak_running"],
                             "failed": peak["failed"]})
    if args.serve_plain_requests > 0 and fracs:
        f = min(fracs)
        jobs = request_stream(pool, args.serve_plain_requests, seed=100 + rank)
        rate = f * cap
        lat, wall, peak = run_serving(wm, jobs, 1, budget, rate_hz=rate, seed=7 + rank, precision="fp64")
        pts = sum(len(x) for _, x, _ in jobs)
        out["plain_form"] = {"fraction_of_saturation": f, "rate_hz": rate, "requests": len(jobs), "workers": 1,
                             "precision": "fp64", "p50_ms": float(np.percentile(lat, 50)),
                             "p99_ms": float(np.percentile(lat, 99)), "mpoints_per_s": pts / wall / 1e6,
                             "note": "the same request stream at the lowest swept rate, served one job at a "
                                     "time with every distance in FP64"}
    return out


def run_ablation(wm, torch, call, timed_pass, release):
    """MemoGFK (the default) against GFK (the full WSPD materialised, Algorithm 2) and EMST-Naive
    on the EMST of 10^7 uniform points in 3-D; and, on the HDBSCAN* workload, the disjunctive
    separation of Sec. 3.1.2 against the geometric one of the GanTao baseline (the full WSPD of
    each counted by the GFK form).  One warm-up and one timed call per method."""
    def run(w, x, method):
        def fn():
            if w["problem"] == "hdbscan":
                return wm.hdbscan(x, min_pts=w["min_pts"], start=0, method=method, return_stats=True)
            return wm.emst(x, method=method, return_stats=True)
        fn()
        stream = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        s = r["stats"]
        return {"ms": e0.elapsed_time(e1), "wspd_pairs": int(s.wspd_pairs), "bccp_pairs": int(s.pairs_retrieved),
                "bccp_evals": int(s.bccp_evals), "rounds": int(s.rounds),
                "traversal_visits": int(s.getpairs_visits + s.getrho_visits), "candidate_edges": int(s.candidate_edges)}
    out = {}
    w = WORKLOADS["emst-uniform-10m-3d"]
    x = torch.from_numpy(make_points(w)).cuda()
    out["emst-uniform-10m-3d"] = {m: run(w, x, m) for m in ("memogfk", "gfk", "naive")}
    del x
    release()
    w = WORKLOADS[CFG2]
    x = torch.from_numpy(make_points(w)).cuda()
    out[CFG2] = {m: run(w, x, m) for m in ("memogfk", "gantao", "gfk", "gfk-geometric")}
    del x
    release()
    out["note"] = ("every method returns the same tree (tests/test_gpu_methods.py checks it); wspd_pairs: size of the materialised WSPD (GFK forms); "
                   "bccp_pairs: pairs whose BCCP was evaluated (MemoGFK counts a pair again in each round that "
                   "retrieves it)")
    return out


# ------------------------------------------------------------------------------ rooflines
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per unit of work of a kernel, from an
# ncu capture of a smaller case of the same kernel, scaled to the bench's launches by their units
# (the node-pair visits of a traversal, the distance evaluations of the k-NN kernel).  A figure is
# reported only while the kernel's source file is the measured version (sha256), else null.
# Captured on emst-uniform-10m-3d run at n = 2x10^6 (--points 2000000), every traversal launch of
# one call (90 GetPairs, 54 GetRho): 8.962 GB over 110,660,742 visits and 1.088 GB over
# 19,169,412 visits.
MEASURED_TRAFFIC = {
    "getpairs": {"bytes_per_unit": 80.99, "source": "paper_2104_01126_gb300/csrc/wspd.cu",
                 "sha256": "027e4fa02ba56ff6c3a2110c7325f5a8fa9cbdd99ca7ec172ad17532d667af12"},
    "getrho": {"bytes_per_unit": 56.75, "source": "paper_2104_01126_gb300/csrc/wspd.cu",
               "sha256": "027e4fa02ba56ff6c3a2110c7325f5a8fa9cbdd99ca7ec172ad17532d667af12"},
}


def measured_traffic(key, units):
    import hashlib
    t = MEASURED_TRAFFIC.get(key)
    if t is None or not units:
        return None
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), t["source"]), "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None
    return t["bytes_per_unit"] * units if h == t["sha256"] else None


def load_peaks():
    """Measured peaks (MEASURED_PEAKS.json, written by the pool's driver), else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            j = json.load(f)
        return {"hbm_gbs": float(j["hbm_gbs"]), "hbm_basis": "of measured (MEASURED_PEAKS.json copy bandwidth)"}
    except Exception:
        return {"hbm_gbs": 6800.0, "hbm_basis": "of fallback 6.8 TB/s"}


def visit_bytes(d):
    """Algorithmic bytes of one visited node pair of a WSPD traversal: the pair (8 B), two link
    records (2 x 16 B), two meta records holding the component labels (2 x 16 B), two boxes
    (2 x 2 x DP x 4 B, DP = d rounded up to 4, 8 or 16) and at most two child pairs (16 B)."""
    dp = 4 if d <= 4 else 8 if d <= 8 else 16
    return 8 + 32 + 32 + 16 * dp + 16


def kernel_rooflines(runs, peaks, fp32_peak, fp32_basis, hdb=False):
    """Per-kernel roofline entries summed over runs = [(d, stats), ...]: the traversals against
    HBM (algorithmic bytes per visited pair), the BCCP and k-NN kernels against the measured FP32
    FMA peak (3d-1 flop per distance evaluation, +2 under mutual reachability)."""
    def tot(f):
        return sum(f(d, s) for d, s in runs)

    ks = []

    def hbm(name, key, visits, ms, launches):
        if ms <= 0 or tot(lambda d, s: visits(s)) <= 0:
            return
        byts = tot(lambda d, s: visits(s) * visit_bytes(d))
        gbs = byts / (ms * 1e-3) / 1e9
        ks.append({"kernel": name, "bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                   "frac": gbs / peaks["hbm_gbs"], "ms": ms, "launches": launches,
                   "traffic": (measured_traffic(key, tot(lambda d, s: visits(s))) / launches
                               if launches and measured_traffic(key, 1) else None),
                   "traffic_total": measured_traffic(key, tot(lambda d, s: visits(s))),
                   "work": f"{tot(lambda d, s: visits(s))} visited node pairs x {visit_bytes(runs[0][0])} B "
                           f"(d = {runs[0][0]}; the byte count grows with d)",
                   "peak_basis": peaks["hbm_basis"]})

    def alu(name, evals, ms, launches, extra=0):
        if ms <= 0:
            return
        ev = tot(lambda d, s: evals(s))
        if ev <= 0:
            return
        fl = tot(lambda d, s: evals(s) * (3 * d - 1 + extra))
        tf = fl / (ms * 1e-3) / 1e12
        ks.append({"kernel": name, "bound": "alu", "achieved": tf, "peak": fp32_peak, "unit": "TFLOP/s",
                   "frac": tf / fp32_peak, "ms": ms, "launches": launches, "traffic": None,
                   "work": f"{ev} distance evaluations x (3d-1{'+2' if extra else ''}) flop",
                   "peak_basis": fp32_basis})

    hbm("findpair_dfs_kernel<1> (GetPairs traversal)", "getpairs", lambda s: s.getpairs_visits,
        tot(lambda d, s: s.ms_getpairs), tot(lambda d, s: s.getpairs_launches))
    hbm("findpair_dfs_kernel<0> (GetRho traversal)", "getrho", lambda s: s.getrho_visits,
        tot(lambda d, s: s.ms_getrho), None)
    x = 2 if hdb else 0
    alu("bccp_group_kernel<1/8> (tiny and small pairs)",
        lambda s: s.bccp_evals - s.bccp_tile_evals - s.bccp_dual_evals, tot(lambda d, s: s.ms_bccp_group), None, x)
    alu("bccp_pair_tile_kernel (medium and big pairs)", lambda s: s.bccp_tile_evals,
        tot(lambda d, s: s.ms_tile_kernel), None, x)
    alu("bccp_dual_kernel (huge pairs, pruned dual-tree)", lambda s: s.bccp_dual_evals,
        tot(lambda d, s: s.ms_bccp_dual), None, x)
    alu("knn_fast_kernel (core distances)", lambda s: s.knn_evals, tot(lambda d, s: s.ms_knn_kernel),
        len(runs))
    if not ks:
        return None
    roof = dict(max(ks, key=lambda k: k["ms"]))
    roof["all"] = ks
    return roof


# ------------------------------------------------------------------------------ multi-rank helpers
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


# ------------------------------------------------------------------------------ the oracle arm
def oracle_step(w, xs):
    """One run of the FP64 oracle's exact k-d tree solvers (the same results as its brute force,
    pinned to it in tests/test_oracle.py) on the points xs."""
    import oracle
    if w["problem"] == "hdbscan":
        oracle.hdbscan_at_scale(xs, w["min_pts"], s=0)
    else:
        oracle.emst_at_scale(xs)


def oracle_samples(names, sample):
    """The first `sample` points of each workload (the generators shuffle rows)."""
    out = []
    for nm in names:
        w = WORKLOADS[nm]
        x = make_points(w)
        ns = min(w["n"], sample)
        out.append((nm, w, np.ascontiguousarray(x[:ns])))
        del x
    return out


def run_reference(args, ws, rank):
    """The FP64 CPU oracle timed on a bounded sample of each workload (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    names = workload_names(args.workload)
    sample = args.ref_sample if args.ref_sample > 0 else (30_000 if len(names) > 1 else 1_000_000)
    samples = oracle_samples(names, sample)
    oracle.build()

    def step():
        for _, w, xs in samples:
            oracle_step(w, xs)
    for _ in range(args.warmup if args.ref_warmup is None else args.ref_warmup):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    pts = sum(len(xs) for _, _, xs in samples)
    v = pts / t / 1e6
    cores = os.cpu_count()
    desc = (f"the first {sample} points of each of {len(names)} workloads ({pts} points; the generators "
            f"shuffle rows), FP64 oracle (exact k-d tree k-NN and Boruvka, plus the dendrogram and plot for "
            f"HDBSCAN*), OpenMP on {cores} host threads")
    line = {"metric": METRIC, "impl": "reference", "value": v, "unit": "Mpoints/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "workloads": names, "sample_points_per_workload": sample},
            "cpu_baseline": {"value": v, "unit": "Mpoints/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": "Mpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(names, sample):
    import oracle
    oracle.build()
    samples = oracle_samples(names, sample)
    t0 = time.perf_counter()
    for _, w, xs in samples:
        oracle_step(w, xs)
    t = time.perf_counter() - t0
    pts = sum(len(xs) for _, _, xs in samples)
    cores = os.cpu_count()
    return {"value": pts / t / 1e6, "unit": "Mpoints/s", "cores": cores, "kind": "oracle",
            "sample": f"the first {sample} points of each of {len(names)} workloads ({pts} points), one run of "
                      f"the FP64 oracle's exact k-d tree solvers ({t:.1f} s, OpenMP on {cores} host threads)"}


# ------------------------------------------------------------------------------ our arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="emst-10m-suite", choices=sorted(WORKLOADS) + sorted(SUITES))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--cpu-sample", type=int, default=100_000, help="points per workload for the CPU baseline")
    ap.add_argument("--ref-sample", type=int, default=0,
                    help="points per workload for --impl reference (0: 30,000 per workload of a suite)")
    ap.add_argument("--ref-warmup", type=int, default=None, help="warm-up runs of --impl reference (default: --warmup)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cfg2", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=1000, help="requests per swept rate (0: no serving)")
    ap.add_argument("--serve-rates", default="0.5,1.0,2.0", help="arrival rates as fractions of saturation")
    ap.add_argument("--serve-pool", type=int, default=64, help="distinct point sets the requests draw from")
    ap.add_argument("--serve-plain-requests", type=int, default=200)
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    ap.add_argument("--batch-instances", type=int, default=4096)
    ap.add_argument("--no-ablation", action="store_true")
    ap.add_argument("--points", type=int, default=0,
                    help="run the workload's generator and dimension at this n instead (profiling captures "
                         "of a smaller case; the line then says so in config.points)")
    args = ap.parse_args()
    ws, rank, local = dist_setup()

    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import torch
    import paper_2104_01126_gb300 as wm
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wm.load()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    fp32_peak, fma_ms = wm.fp32_fma_peak()
    fp32_basis = (f"of measured: FFMA probe (independent FMA chains on every SM, best of 5 after a warm-up, "
                  f"{fma_ms:.3f} ms, CUDA events, clocks as found)")
    peaks = load_peaks()

    def call(w, inp, precision):
        if w["problem"] == "hdbscan":
            return wm.hdbscan(inp, min_pts=w["min_pts"], start=0, precision=precision, return_stats=True)
        return wm.emst(inp, precision=precision, return_stats=True)

    def timed_pass(items, precision):
        """One step: every workload once, each call bracketed by CUDA events after an L2 flush."""
        ms, st = [], []
        for w, xd in items:
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = call(w, xd, precision)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            st.append(r["stats"])
        return ms, st

    def e2e_pass(items_host, steps):
        """The same calls through the C ABI from pinned host buffers into host outputs."""
        et = []
        for _ in range(steps):
            tot = 0.0
            for w, xh in items_host:
                flush.fill_(1)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                call(w, xh, args.precision)
                torch.cuda.synchronize()
                tot += time.perf_counter() - t0
            et.append(tot * 1e3)
        return sum(et) / len(et)

    def io_bytes(w, x):
        n, d = x.shape
        h2d = n * d * x.dtype.itemsize
        if w["problem"] == "hdbscan":
            d2h = (n - 1) * 16 + n * 8 + (n - 1) * 24 + n * 4 + n * 8
        else:
            d2h = (n - 1) * 16 + 8
        return h2d, d2h

    # ---- the headline workloads, device resident
    names = workload_names(args.workload)
    sel = [dict(WORKLOADS[nm], n=args.points) if args.points else WORKLOADS[nm] for nm in names]
    host = [(w, make_points(w)) for w in sel]
    dev = [(w, torch.from_numpy(x).cuda()) for w, x in host]
    n_total = sum(int(x.shape[0]) for _, x in host)
    for _ in range(args.warmup):
        timed_pass(dev, args.precision)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = wm.kernel_launch_count()
    steps_ms, per_wl = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            ms, st = timed_pass(dev, args.precision)
            steps_ms.append(sum(ms))
            per_wl.append(ms)
    torch.cuda.synchronize()
    launches = wm.kernel_launch_count() - l0
    if dist:
        dist.barrier()
    ms_step = sum(steps_ms) / len(steps_ms)
    ms_max = max_over_ranks(ms_step, dist, device="cuda")
    value = whole_job_value(n_total, ws, ms_max)
    clocks = clk.summary()
    runs = [(w["d"], s) for (w, _), s in zip(dev, st)]
    roof = kernel_rooflines(runs, peaks, fp32_peak, fp32_basis, hdb=any(w["problem"] == "hdbscan" for w, _ in dev))
    screen_err = max(s.max_rel_screen_err for s in st)
    workloads = {}
    for i, ((w, x), s) in enumerate(zip(host, st)):
        nm = names[i]
        workloads[nm] = {"n": int(x.shape[0]), "d": int(x.shape[1]), "generator": w["gen"],
                         "ms": round(statistics.mean(p[i] for p in per_wl), 3),
                         "mpoints_per_s": x.shape[0] / (statistics.mean(p[i] for p in per_wl) * 1e-3) / 1e6,
                         "phases_ms": {k: round(getattr(s, k), 3) for k in (
                             "ms_build_tree", "ms_core_dist", "ms_wspd", "ms_getrho", "ms_getpairs", "ms_bccp",
                             "ms_bccp_group", "ms_tile_kernel", "ms_bccp_dual", "ms_kruskal", "ms_dendrogram",
                             "ms_knn_kernel")},
                         "counters": {k: int(getattr(s, k)) for k in (
                             "rounds", "pairs_retrieved", "bccp_evals", "bccp_tile_evals", "bccp_dual_evals",
                             "bccp_tile_evals_skipped", "bccp_pairs_above", "knn_evals", "fp64_rechecks",
                             "candidate_edges", "tree_depth", "getpairs_launches", "getpairs_visits",
                             "getrho_visits", "rho_shrinks")},
                         "max_rel_screen_err": s.max_rel_screen_err}
    del dev
    torch.cuda.empty_cache()

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        items_host = [(w, torch.from_numpy(x).pin_memory()) for w, x in host]
        e2e_pass(items_host[:1], 1)
        e_ms = max_over_ranks(e2e_pass(items_host, max(1, min(args.steps, 2))), dist, device="cuda")
        h2d = sum(io_bytes(w, x)[0] for w, x in host)
        d2h = sum(io_bytes(w, x)[1] for w, x in host)
        e2e = {"value": whole_job_value(n_total, ws, e_ms), "unit": "Mpoints/s", "ms_per_step": e_ms,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        del items_host

    # ---- the plain form: every distance in FP64, one job at a time
    plain = None
    if not args.no_plain and args.precision == "fp32":
        dev = [(w, torch.from_numpy(x).cuda()) for w, x in host]
        timed_pass(dev[:1], "fp64")
        pms, _ = timed_pass(dev, "fp64")
        p_ms = max_over_ranks(sum(pms), dist, device="cuda")
        plain = {"value": whole_job_value(n_total, ws, p_ms), "unit": "Mpoints/s", "ms_per_step": p_ms,
                 "precision": "fp64", "per_workload_ms": {nm: round(t, 3) for nm, t in zip(names, pms)},
                 "note": "the same workloads, every distance evaluated in FP64, one job at a time"}
        del dev
        torch.cuda.empty_cache()

    # ---- configuration 2: HDBSCAN* on 10^6 Gaussian-mixture points
    cfg2 = None
    if not args.no_cfg2 and CFG2 not in names:
        w = WORKLOADS[CFG2]
        x = make_points(w)
        xd = torch.from_numpy(x).cuda()
        timed_pass([(w, xd)], args.precision)
        timed_pass([(w, xd)], args.precision)
        cms, cst = [], None
        for _ in range(max(3, args.steps)):
            ms, st2 = timed_pass([(w, xd)], args.precision)
            cms += ms
            cst = st2[0]
        c_ms = max_over_ranks(statistics.mean(cms), dist, device="cuda")
        pms, _ = timed_pass([(w, xd)], "fp64")
        xh = torch.from_numpy(x).pin_memory()
        ce = max_over_ranks(e2e_pass([(w, xh)], 3), dist, device="cuda")
        h2d, d2h = io_bytes(w, x)
        cfg2 = {"workload": CFG2, "n": w["n"], "d": w["d"], "min_pts": w["min_pts"], "generator": w["gen"],
                "value": whole_job_value(w["n"], ws, c_ms), "unit": "Mpoints/s", "ms_per_step": c_ms,
                "step_ms": [round(t, 3) for t in cms],
                "e2e": {"value": whole_job_value(w["n"], ws, ce), "unit": "Mpoints/s", "ms_per_step": ce,
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "plain_form": {"value": whole_job_value(w["n"], ws, pms[0]), "unit": "Mpoints/s",
                               "ms_per_step": pms[0], "precision": "fp64"},
                "roofline": kernel_rooflines([(w["d"], cst)], peaks, fp32_peak, fp32_basis, hdb=True),
                "max_rel_screen_err": cst.max_rel_screen_err,
                "phases_ms": {k: round(getattr(cst, k), 3) for k in (
                    "ms_build_tree", "ms_core_dist", "ms_knn_kernel", "ms_wspd", "ms_getrho", "ms_getpairs",
                    "ms_bccp", "ms_kruskal", "ms_dendrogram")},
                "counters": {k: int(getattr(cst, k)) for k in (
                    "rounds", "pairs_retrieved", "bccp_evals", "knn_evals", "fp64_rechecks", "candidate_edges",
                    "getpairs_visits", "getrho_visits")}}
        del xd, xh
        torch.cuda.empty_cache()

    # ---- ablation: the paper's method against GFK and EMST-Naive (EMST, uniform 3-D, 10^7 points),
    # and the disjunctive separation against GanTao's geometric one (the HDBSCAN* workload)
    ablation = None
    if not args.no_ablation:
        ablation = run_ablation(wm, torch, call, timed_pass, release=wm.release_cache)

    served = serving_sweep(wm, args, rank) if args.serve_requests > 0 else None
    batched = run_batched(wm, torch, args.batch_instances, seed=rank) if args.batch_instances > 0 else None

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(names, args.cpu_sample)

    if rank == 0:
        cfg = {"workload": args.workload, "workloads": names, "n_per_workload": [int(x.shape[0]) for _, x in host],
               "points_per_step": n_total, "seed": 0, "precision": args.precision,
               "coordinates": "FP32", "l2": "256 MiB buffer written before every timed call",
               "parallelism": f"replicas{ws}"}
        if args.points:
            cfg["points"] = args.points
        line = {"metric": METRIC, "value": value, "unit": "Mpoints/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
                "config": cfg, "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roof,
                "cpu_baseline": cpu, "max_rel_screen_err": screen_err,
                "screen_error_band": "a priori 2^-19 = 1.9e-6 relative for FP32 coordinates",
                "fp32_peak_tflops": fp32_peak, "plain_form": plain, "workloads": workloads, "cfg2": cfg2,
                "served": served, "batched": batched, "ablation": ablation,
                "step_ms": [round(t, 3) for t in steps_ms]}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
