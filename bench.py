#!/usr/bin/env python3
"""Core-ALS sweep throughput on one GB300 (row-solves/s).

Workload: the 100k-user x 20k-item rating matrix with 10M observed cells
(Zipf(1.0) user and item popularity, integer 1-5 ratings from a rank-32
truth plus N(0, 0.5^2) noise; 9M train / 1M test), n_f = 32,
lambda = 0.05, CES budget r = 0.25, the paper's asymmetric estimator
(Eq. core_ui) in FP32. Synthetic, seeded; no dataset is read.

A step is one full sweep of Algorithm 2 (all users, then all items) plus
the test-RMSE evaluation. value = (n_u + n_m) row solves per sweep / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (under torchrun) every rank runs an independent replica of the
workload on its own GPU (the method needs an exchange of the whole updated
factor between half-sweeps to shard one problem; that path is not built).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2509_18024_gb300 import synth  # noqa: E402

WORKLOAD = "zipf_100k"
METRIC = "ALS time-to-RMSE & row-solves/s, core vs full, FP32 vs mixed; % of roofline"
UNIT = "row-solves/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP32 FMA roof: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (maximum SM clock).
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--budget", type=float, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--precision", choices=["fp32", "tf32", "bf16", "fp32_tc"], default="fp32")
    ap.add_argument("--refine", type=int, default=None,
                    help="refinement steps for --workload zipf_1m (default: the precision's automatic count)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--workload", choices=["zipf_100k", "zipf_1m", "warmstart", "batch64"], default="zipf_100k",
                    help="zipf_1m: the 1M x 100k, 10^8-cell matrix drawn on the device, fitted at --nf; "
                         "warmstart: the learned warm start on 100k x 20k matrices (5 training, 5 held-out seeds); "
                         "batch64: 64 independent problems of mixed sizes and widths in one batch")
    ap.add_argument("--nf", type=int, default=None,
                    help="model width for --workload zipf_1m (default 64) or --capture-case (default 32)")
    ap.add_argument("--capture-case", choices=sorted(synth.CAPTURE_CASES), default=None,
                    help="run one half-sweep of a small single-bucket case three times (for ncu captures)")
    ap.add_argument("--sketch", choices=["slice", "factor"], default="slice",
                    help="factor: the fast variant (CES once on the whole design factor)")
    ap.add_argument("--no-large", action="store_true", help="skip the 10^8-cell n_f = 128 records")
    ap.add_argument("--no-sim", action="store_true", help="skip the simulation-design metrics")
    ap.add_argument("--no-probes", action="store_true", help="skip the roofline probes")
    ap.add_argument("--no-warm", action="store_true", help="skip the learned warm-start record")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-problem batch record")
    return ap.parse_args()


def workload_config(w, r):
    return {"workload": f"{WORKLOAD}: {w['n_u']} users x {w['n_m']} items, {w['nnz']} observed "
                        f"(Zipf {w['zipf_s']}), n_f={w['f']}, lambda={w['lam']}, r={r}, asymmetric Eq. core_ui",
            "n_u": w["n_u"], "n_m": w["n_m"], "nnz": w["nnz"], "n_f": w["f"], "lambda": w["lam"], "budget": r,
            "gram": "asym", "reg": "weighted", "train_frac": 0.9, "precision": "fp32"}


# ----------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.15)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------- CPU oracle leg
def oracle_sample(p, M0, lam, r, n_user_rows, n_item_rows, seed):
    """Time the FP64 oracle on random rows of both sides; return rows/s of a
    whole sweep extrapolated by observed entries, and what was run."""
    import oracle
    rng = np.random.default_rng(seed)
    U0 = synth.init_factor(p.n_u, p.f, 2000)
    t_sweep = 0.0
    done = 0
    for csr, Y, k in ((p.train_rows, M0, n_user_rows), (p.train_cols, U0, n_item_rows)):
        rows = np.sort(rng.choice(csr.n_rows, size=min(k, csr.n_rows), replace=False))
        L = np.diff(csr.indptr)
        t0 = time.perf_counter()
        oracle.half_sweep(csr.indptr, csr.indices, csr.values, Y, lam, r, oracle.GRAM_ASYM, rows=rows)
        dt = time.perf_counter() - t0
        t_sweep += dt * csr.nnz / max(int(L[rows].sum()), 1)
        done += len(rows)
    return (p.n_u + p.n_m) / t_sweep, done, t_sweep


def small_leg(M0_seed=1000, seed=1):
    """The oracle-sized workload ('small': 1000 x 500, n_f = 10, 5 % of the
    cells, lambda 0.1, r = 0.5) timed whole: the GPU sweep (CUDA events) and
    the FP64 oracle's full sweep on all host cores and on one core, from the
    same M^(0), with the test RMSE of both after the same sweeps."""
    import torch
    import oracle
    from paper_2509_18024_gb300 import core_als
    w = dict(synth.WORKLOADS["small"])
    p = synth.make_workload("small", seed=seed)
    M0 = synth.init_factor(p.n_m, p.f, M0_seed)
    sweeps = w["sweeps"]
    eng = core_als.CoreALS(p.f, w["lam"], w["budget"])
    Ru, Ri = core_als.DeviceCSR.from_host(p.train_rows), core_als.DeviceCSR.from_host(p.train_cols)
    M = torch.as_tensor(M0).cuda()
    U = torch.empty((p.n_u, p.f), device="cuda")
    eng.sweep(Ru, Ri, U, M)  # plans and workspace
    M.copy_(torch.as_tensor(M0))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(sweeps):
        eng.sweep(Ru, Ri, U, M)
    b.record()
    torch.cuda.synchronize()
    gpu_ms = a.elapsed_time(b) / sweeps
    test = tuple(np.asarray(t) for t in (p.test_u, p.test_m, p.test_r))
    gpu_rmse = oracle.rmse(*test, U.cpu().numpy().astype(np.float64), M.cpu().numpy().astype(np.float64))
    eng.close()
    oracle.build()
    res = {}
    all_cores = oracle.num_threads()
    for cores in (all_cores, 1):
        oracle.set_threads(cores)
        try:
            t0 = time.perf_counter()
            Uo, Mo = oracle.fit(p.train_rows, p.train_cols, M0, w["lam"], w["budget"], sweeps)
            dt = time.perf_counter() - t0
        finally:
            oracle.set_threads(all_cores)
        res[f"oracle_{'all' if cores == all_cores else 'one'}_cores"] = {
            "cores": cores, "ms_per_sweep": 1e3 * dt / sweeps,
            "row_solves_per_s": (p.n_u + p.n_m) * sweeps / dt}
        oracle_rmse = oracle.rmse(*test, Uo, Mo)
    return {"workload": f"small: {p.n_u} x {p.n_m}, {p.train_rows.nnz} training cells, n_f={p.f}, "
                        f"lambda={w['lam']}, r={w['budget']}, {sweeps} sweeps from the same M^(0)",
            "gpu": {"ms_per_sweep": gpu_ms, "row_solves_per_s": (p.n_u + p.n_m) / (gpu_ms * 1e-3),
                    "test_rmse": gpu_rmse},
            **res, "oracle_test_rmse": oracle_rmse,
            "rmse_rel_diff": abs(gpu_rmse - oracle_rmse) / oracle_rmse}


def reference_arm(args, p, w, M0, r):
    import oracle
    oracle.build()
    threads = oracle.num_threads()
    per_user, per_item = 8000, 1600
    for q in range(args.warmup):
        oracle_sample(p, M0, w["lam"], r, per_user // 4, per_item // 4, 100 + q)
    rates, t_total = [], 0.0
    for q in range(args.steps):
        t0 = time.perf_counter()
        rate, done, _ = oracle_sample(p, M0, w["lam"], r, per_user, per_item, 1000 + q)
        t_total += time.perf_counter() - t0
        rates.append(rate)
    value = float(statistics.median(rates))
    sample = (f"each step: one half-sweep of {per_user} random user rows and {per_item} random item rows "
              f"(new rows per step), extrapolated to a full sweep by observed entries")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, r),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- GPU arm
def replica_value(ms, rows, steps, world, device):
    """Whole-job throughput of `world` independent replicas: every rank
    solved `rows` rows per step for `steps` timed steps in `ms` (its own CUDA
    events); the job's time is the slowest rank's, taken by an all-reduce
    MAX over the process group (no other exchange). Returns (ms, value)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * rows * steps / (ms / 1e3)


def gpu_arm(args, p, w, M0, r, rank, world, local_rank):
    import torch
    from paper_2509_18024_gb300 import core_als
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    f, lam = w["f"], w["lam"]
    Ru = core_als.DeviceCSR.from_host(p.train_rows, dev)
    Ri = core_als.DeviceCSR.from_host(p.train_cols, dev)
    tu, tm, tr = (torch.as_tensor(a).to(dev) for a in (p.test_u, p.test_m, p.test_r))
    eng = core_als.CoreALS(f, lam, r, gram_mode="asym", precision=PRECISIONS[args.precision], sketch=args.sketch)
    M = torch.as_tensor(M0).to(dev)
    U = torch.empty((p.n_u, f), dtype=torch.float32, device=dev)
    tuning = None
    if not args.no_autotune:
        tuning = eng.autotune(Ru, Ri, U, M, trials=3)
    eng.prepare(Ru)
    eng.prepare(Ri)
    sse = torch.zeros(1, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def step(e=eng):
        e.half_sweep(Ru, M, U)
        e.half_sweep(Ri, U, M)
        e.sse_async(tu, tm, tr, U, M, sse)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = eng.launch_count
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for q in range(args.steps):
            flush.zero_()
            evs[q][0].record(stream)
            step()
            evs[q][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches = eng.launch_count - launches0
    ms = sum(a.elapsed_time(b) for a, b in evs)
    # Per-kernel times from separate profiled steps (CUDA events around every
    # launch; the handle then runs each half-sweep on one stream, so each
    # launch is timed alone).
    prof_steps = max(3, min(args.steps, 10))
    eng.profile(True)
    for q in range(prof_steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    fam = {}
    for name in KERNEL_FAMILIES:
        t, n = eng.kernel_time(name)
        if n:
            fam[name] = (t, n)
    eng.profile(False)
    ms, value = replica_value(ms, p.n_u + p.n_m, args.steps, world, dev)
    test_rmse = float(np.sqrt(sse.item() / len(p.test_r)))

    if rank != 0:
        return None

    # Dominant kernel and its roofline (CES + masked Gram on CUDA cores):
    # algorithmic FP32 flops of Eq. core_ui's assembly per launch.
    top = max(fam, key=lambda k: fam[k][0])
    t_top, n_top = fam[top]
    avg_s = t_top / n_top / 1e3
    roof = roofline(top, avg_s, p, f, r, n_top / prof_steps, getattr(args, "ffma_peak", None))

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": {"fp32": "f32", "fp32_tc": "f32 (split tf32)", "tf32": "tf32/f32",
                                          "bf16": "bf16/f32"}[args.precision], "data": "synthetic (seeded Zipf rating matrix; no dataset)",
           "config": dict(workload_config(w, r), l2="flushed between steps (256 MB write)",
                          parallelism="replicas" if world > 1 else "single GPU", precision=args.precision,
                          schedule=tuning if tuning else "default (not autotuned)"),
           "gpu_launches": launches, "roofline": roof, "clocks": clk.summary(),
           "kernels_ms_per_step": {k: v[0] / prof_steps for k, v in fam.items()},
           "kernels_timing": f"{prof_steps} separate profiled steps, each launch alone on the stream",
           "test_rmse_after_timed_sweeps": test_rmse}
    return out, eng, (Ru, Ri, tu, tm, tr), dev


KERNEL_FAMILIES = ("cta_rows", "warp_rows", "solve_rows", "split_init", "split_hist", "split_eqcount",
                   "split_cut", "split_gram", "split_reduce", "sse", "sum_partials")


# DRAM traffic of the dominant kernel family, from the one-pass ncu capture
# summarised in profiles/cta_rows_zipf100k_traffic.md (dram__bytes_read.sum +
# dram__bytes_write.sum, summed over the k_cta_rows launches of one sweep;
# `roofline.traffic` is that sum over the sweep's measured launches). It
# holds only for the kernel's sources it was taken from: `roofline.traffic`
# is null once they hash differently.
TRAFFIC = {"kernel": "cta_rows", "bytes_per_sweep": 183.0e6, "sources_sha256_16": "3854a07198f97238",
           "sources": ("als_device.cuh", "als_rows.cuh", "als_tc.cuh")}


def kernel_sources_hash(files=TRAFFIC["sources"]):
    import hashlib
    pkg = os.path.join(ROOT, "paper_2509_18024_gb300", "csrc")
    h = hashlib.sha256()
    for fn in files:
        h.update(fn.encode())
        with open(os.path.join(pkg, fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def roofline(top, avg_s, p, f, r, launches_per_sweep, peak=None):
    """Roofline entry of the dominant kernel family: algorithmic FP32 flops
    of the rows it handles (2 s_i f^2 for X*^T X plus 2 s_i f for X*^T r, with
    s_i = floor(n_i r)), per launch: a sweep's flops over its measured
    launches of the family (cta_rows: one per run of rows with the same
    resident CTAs per SM, in each of three buckets per side)."""
    flops = 0.0
    for csr in (p.train_rows, p.train_cols):
        L = np.diff(csr.indptr)
        if top == "cta_rows":
            sel = (L > 32) & (L <= 1024)
        elif top == "warp_rows":
            sel = L <= 32
        elif top in ("split_gram", "split_hist"):
            sel = L > 1024
        else:
            sel = L > 32
        s = np.floor(L[sel].astype(np.float64) * r)
        if top == "solve_rows":
            flops += sel.sum() * (2.0 / 3.0 * f ** 3 + 2 * f * f)
        else:
            flops += float((2 * s * f * f + 2 * s * f).sum())
    per_launch = flops / launches_per_sweep
    achieved = per_launch / avg_s / 1e12
    traffic = None
    if top == TRAFFIC["kernel"] and kernel_sources_hash() == TRAFFIC["sources_sha256_16"]:
        traffic = TRAFFIC["bytes_per_sweep"] / launches_per_sweep
    if peak:
        pk, src = peak, "of measured: ALS_PROBE_FFMA (FP32 FMA throughput probe) in this run"
    else:
        pk, src = FP32_ALU_PEAK_TFLOPS, "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"
    return {"bound": "alu", "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
            "frac": achieved / pk, "traffic": traffic, "traffic_unit": "bytes per launch",
            "algorithmic_flops_per_launch": per_launch, "kernel": top,
            "avg_launch_ms": avg_s * 1e3, "peak_source": src}


def e2e_leg(p, w, r, M0, steps=3, sweeps=1):
    """Through the host-buffer C-ABI call (als_fit_host, `sweeps` sweeps per
    step): every step copies both sides' structure, M^(0) and the test set
    from pinned host memory and reads U and M back."""
    import torch
    from paper_2509_18024_gb300 import core_als

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        return t.numpy()

    rows = synth.CSR(p.train_rows.n_rows, p.train_rows.n_cols, pinned(p.train_rows.indptr),
                     pinned(p.train_rows.indices), pinned(p.train_rows.values))
    cols = synth.CSR(p.train_cols.n_rows, p.train_cols.n_cols, pinned(p.train_cols.indptr),
                     pinned(p.train_cols.indices), pinned(p.train_cols.values))
    test = (pinned(p.test_u), pinned(p.test_m), pinned(p.test_r))
    M0p = pinned(M0)
    eng = core_als.CoreALS(w["f"], w["lam"], r)
    eng.fit_host(rows, cols, M0p, sweeps, test=test)  # warm
    t0 = time.perf_counter()
    for _ in range(steps):
        eng.fit_host(rows, cols, M0p, sweeps, test=test)
    dt = time.perf_counter() - t0
    nnz, f = p.train_rows.nnz, w["f"]
    h2d = (p.n_u + 1) * 8 + (p.n_m + 1) * 8 + 2 * nnz * 8 + p.n_m * f * 4 + len(p.test_r) * 12
    d2h = (p.n_u + p.n_m) * f * 4
    return {"value": (p.n_u + p.n_m) * steps * sweeps / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h),
            "api": f"als_fit_host ({sweeps} sweep{'s' if sweeps > 1 else ''} per call, incl. validation)"}


PRECISIONS = {"fp32": 0, "tf32": 1, "bf16": 2, "fp32_tc": 3}


def variants(p, w, M0, rvals, steps=5):
    """Rows/s of other estimator settings on the same workload (device-timed)."""
    import torch
    from paper_2509_18024_gb300 import core_als
    Ru = core_als.DeviceCSR.from_host(p.train_rows)
    Ri = core_als.DeviceCSR.from_host(p.train_cols)
    out = {}
    for name, r, mode, prec, *kw in rvals:
        eng = core_als.CoreALS(w["f"], w["lam"], r, gram_mode=mode, precision=PRECISIONS[prec], **(kw[0] if kw else {}))
        M = torch.as_tensor(M0).cuda()
        U = torch.empty((p.n_u, w["f"]), dtype=torch.float32, device="cuda")
        for _ in range(2):
            eng.half_sweep(Ru, M, U)
            eng.half_sweep(Ri, U, M)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            eng.half_sweep(Ru, M, U)
            eng.half_sweep(Ri, U, M)
        b.record()
        torch.cuda.synchronize()
        out[name] = (p.n_u + p.n_m) * steps / (a.elapsed_time(b) / 1e3)
        eng.close()
    return out


def time_to_rmse(p, w, M0, settings, sweeps=15):
    """Algorithm 2 from the same M^(0) for each setting: the test RMSE after
    every sweep and the cumulative CUDA-event sweep time. The target is the
    first setting's final test RMSE x (1 + 1e-3); each setting reports the
    time of the first sweep that reaches it (None if it never does)."""
    import torch
    from paper_2509_18024_gb300 import core_als
    Ru = core_als.DeviceCSR.from_host(p.train_rows)
    Ri = core_als.DeviceCSR.from_host(p.train_cols)
    tu, tm, tr = (torch.as_tensor(a).cuda() for a in (p.test_u, p.test_m, p.test_r))
    curves = {}
    for name, r, mode, prec, *kw in settings:
        eng = core_als.CoreALS(w["f"], w["lam"], r, gram_mode=mode, precision=PRECISIONS[prec], **(kw[0] if kw else {}))
        eng.prepare(Ru)
        eng.prepare(Ri)
        M = torch.as_tensor(M0).cuda()
        U = torch.empty((p.n_u, w["f"]), dtype=torch.float32, device="cuda")
        cum, pts = 0.0, []
        for _ in range(sweeps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            eng.half_sweep(Ru, M, U)
            eng.half_sweep(Ri, U, M)
            b.record()
            torch.cuda.synchronize()
            cum += a.elapsed_time(b)
            pts.append((cum, eng.rmse(tu, tm, tr, U, M)))
        curves[name] = pts
        eng.close()
    first = settings[0][0]
    target = curves[first][-1][1] * (1 + 1e-3)
    res = {"target_rmse": target, "target_from": first, "sweeps": sweeps}
    for name, pts in curves.items():
        hit = next((t for t, e in pts if e <= target), None)
        res[name] = {"ms": hit, "final_rmse": pts[-1][1], "sweeps_to_target":
                     next((q + 1 for q, (t, e) in enumerate(pts) if e <= target), None)}
    return res


def large_leg(d, w, f, precision, steps, warmup, seed, sample_rows=10000, clocks=True, refine=None):
    """Sweep throughput on the 1M x 100k, 10^8-cell matrix (drawn on the
    device) at width f: ms per sweep (CUDA events, L2 flushed between
    sweeps), per-kernel times from one separately profiled sweep, and the
    error of one user half-sweep from M^(0) against the FP64 oracle on
    `sample_rows` sampled rows, with the oracle's own rate on that sample."""
    import torch
    import oracle
    from paper_2509_18024_gb300 import core_als
    lam = w["lam"]
    r = w["budget"]
    Ru = core_als.DeviceCSR(w["n_u"], w["n_m"], *d.rows)
    Ri = core_als.DeviceCSR(w["n_m"], w["n_u"], *d.cols)
    M0 = synth.init_factor(w["n_m"], f, 1000)
    kw = {} if refine is None else {"refine_steps": int(refine)}
    eng = core_als.CoreALS(f, lam, r, precision=PRECISIONS[precision], **kw)
    M = torch.as_tensor(M0).cuda()
    U = torch.empty((w["n_u"], f), dtype=torch.float32, device="cuda")
    eng.half_sweep(Ru, M, U)
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(w["n_u"], size=sample_rows, replace=False))
    indptr, indices, values = (t.cpu().numpy() for t in d.rows)
    t1 = time.perf_counter()
    Xo, _, _ = oracle.half_sweep(indptr, indices, values, M0.astype(np.float64), lam, r, oracle.GRAM_ASYM, rows=rows)
    t_or = time.perf_counter() - t1
    Xg = U.cpu().numpy()[rows].astype(np.float64)
    Xo = Xo[rows]
    err = float(np.linalg.norm(Xg - Xo) / np.linalg.norm(Xo))
    row_err = np.linalg.norm(Xg - Xo, axis=1) / np.maximum(np.linalg.norm(Xo, axis=1), 1e-300)
    L = np.diff(indptr)
    or_rate = w["n_u"] * 1.0 / (t_or * Ru.nnz / max(int(L[rows].sum()), 1))
    sse = torch.zeros(1, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        eng.half_sweep(Ru, M, U)
        eng.half_sweep(Ri, U, M)
        eng.sse_async(d.test_u, d.test_m, d.test_r, U, M, sse)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    launches0 = eng.launch_count
    clk = ClockSampler(0) if clocks else None
    if clk:
        clk.__enter__()
    for q in range(steps):
        flush.zero_()
        evs[q][0].record(stream)
        step()
        evs[q][1].record(stream)
    torch.cuda.synchronize()
    if clk:
        clk.__exit__(None, None, None)
    ms = sum(a.elapsed_time(b) for a, b in evs)
    launches = eng.launch_count - launches0
    eng.profile(True)
    flush.zero_()
    step()
    torch.cuda.synchronize()
    fam = {k: eng.kernel_time(k) for k in KERNEL_FAMILIES + ("refine_resid", "fp64_rows", "add_rows", "colmax")}
    fam = {k: v for k, v in fam.items() if v[1]}
    eng.profile(False)
    eng.close()
    total = sum(v[0] for v in fam.values()) or 1.0
    n_rows = w["n_u"] + w["n_m"]
    return {"n_f": f, "precision": precision, "refine_steps": "auto" if refine is None else int(refine),
            "ms_per_sweep": ms / steps,
            "row_solves_per_s": n_rows * steps / (ms / 1e3), "gpu_launches_per_sweep": launches / steps,
            "clocks": clk.summary() if clk else None,
            "kernel_ms_per_sweep": {k: v[0] for k, v in fam.items()},
            "kernel_share": {k: v[0] / total for k, v in fam.items()},
            "kernels_timing": "one separate profiled sweep, each launch alone on the stream",
            "error_vs_fp64_oracle": {"sample_rows": len(rows), "rel_fro": err, "row_rel_max": float(row_err.max()),
                                     "row_rel_p99": float(np.quantile(row_err, 0.99)),
                                     "what": "one user half-sweep from the same M^(0)"},
            "oracle_user_rows_per_s": or_rate, "oracle_cores": oracle.num_threads(),
            "test_rmse_after_timed_sweeps": float(np.sqrt(sse.item() / d.test_r.numel()))}


def draw_large(seed):
    import torch
    w = dict(synth.WORKLOADS["zipf_1m"])
    t0 = time.perf_counter()
    d = synth.zipf_ratings_device(w["n_u"], w["n_m"], w["f"], w["nnz"], w["zipf_s"], w["noise_sd"], seed)
    torch.cuda.synchronize()
    return d, w, time.perf_counter() - t0


def large_arm(args):
    """--workload zipf_1m: the 10^8-cell matrix at --nf (default 64) and
    --precision, as one JSON line."""
    d, w, gen_s = draw_large(args.seed)
    f = args.nf or 64
    if args.budget is not None:
        w["budget"] = args.budget
    res = large_leg(d, w, f, args.precision, args.steps, args.warmup, args.seed, refine=args.refine)
    out = {"metric": METRIC, "value": res["row_solves_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": res["ms_per_sweep"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": args.precision, "data": "synthetic (device-drawn Zipf)",
           "config": {"workload": f"zipf_1m: {w['n_u']} users x {w['n_m']} items, {w['nnz']} cells (Zipf "
                                  f"{w['zipf_s']}), n_f={f}, lambda={w['lam']}, r={w['budget']}, asymmetric Eq. core_ui",
                      "n_f": f, "precision": args.precision, "l2": "flushed between steps (256 MB write)",
                      "generation_s": round(gen_s, 1)},
           "gpu_launches": res["gpu_launches_per_sweep"] * args.steps, "clocks": res["clocks"],
           "kernels_ms_per_step": res["kernel_ms_per_sweep"], "kernels_timing": res["kernels_timing"],
           "error_vs_fp64_oracle": res["error_vs_fp64_oracle"],
           "cpu_baseline": {"value": res["oracle_user_rows_per_s"], "unit": "user row-solves/s",
                            "cores": res["oracle_cores"], "kind": "oracle",
                            "sample": "10000 random user rows, one half-sweep, extrapolated by observed entries"},
           "test_rmse_after_timed_sweeps": res["test_rmse_after_timed_sweeps"]}
    print(json.dumps(out), flush=True)


def simulation_leg(seed=1, sweeps=10, r=0.2):
    """The simulation design of Sec. 5.1 (3600 x 3600, n_f = 60, D1 factors
    with 0.6^|i-j| covariance, N(0,1) noise, 40 % of cells removed - R1):
    CORE (Algorithm 2), its fast variant and FULL ALS from the same M^(0),
    with ReMSE on the empirical set, P-ReMSE on the prediction set, and
    Hit@5 / NDCG@10 against the prediction-set items whose value is in the
    top 5 % (all computed by the library's kernels), and sweep times."""
    import torch
    from paper_2509_18024_gb300 import core_als
    p = synth.simulation("D1", synth.SIM_MISSING["R1"], seed=seed)
    Ru = core_als.DeviceCSR.from_host(p.train_rows)
    Ri = core_als.DeviceCSR.from_host(p.train_cols)
    rows = np.repeat(np.arange(p.n_u, dtype=np.int32), np.diff(p.train_rows.indptr))
    emp = tuple(torch.as_tensor(np.ascontiguousarray(a)).cuda()
                for a in (rows, p.train_rows.indices, p.train_rows.values))
    pred = tuple(torch.as_tensor(np.ascontiguousarray(a)).cuda() for a in (p.pred_u, p.pred_m, p.pred_r))
    rel = core_als.DeviceCSR.from_host(synth.relevant_items(p.n_u, p.n_m, p.pred_u, p.pred_m, p.pred_r,
                                                            synth.top_share_threshold(p.pred_r, 0.05)))
    M0 = torch.as_tensor(synth.init_factor(p.n_m, p.f, 77)).cuda()
    out = {"design": "Sec. 5.1: 3600 x 3600, n_f = 60, D1 N(0, 0.6^|i-j|) factors, N(0,1) noise, R1 (40 % removed)",
           "lambda": 0.01, "budget": r, "sweeps": sweeps}
    for name, kw in (("core", dict()), ("core_fast", dict(sketch="factor")), ("full", dict(gram_mode="full"))):
        eng = core_als.CoreALS(p.f, 0.01, 1.0 if name == "full" else r, **kw)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            U, M, rep = eng.fit(Ru, Ri, M0, 1)  # plans, workspace
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            U, M, rep = eng.fit(Ru, Ri, M0, sweeps)
            b.record()
        s.synchronize()
        hit, ndcg, n_eval = eng.ranking(Ru, rel, U, M, 5, 10)
        out[name] = {"ReMSE": eng.remse(*emp, U, M), "P-ReMSE": eng.remse(*pred, U, M), "Hit@5": hit,
                     "NDCG@10": ndcg, "users_evaluated": n_eval, "objective": rep["objective"],
                     "ms_per_sweep": a.elapsed_time(b) / sweeps}
        eng.close()
    return out


def peaks_leg():
    """Project-written roofline probes (als_probe), each one timed launch."""
    from paper_2509_18024_gb300 import core_als
    out = {}
    for kind, key in (("ffma", "fp32_ffma_tflops"), ("dfma", "fp64_dfma_tflops"), ("tc_bf16", "tc_bf16_tflops"),
                      ("tc_tf32", "tc_tf32_tflops"), ("l2_gather", "l2_gather_gbs"), ("hbm_copy", "hbm_copy_gbs")):
        try:
            out[key] = core_als.probe(kind)[0]
        except Exception as e:  # a probe that cannot run on this device
            out[key] = None
            out[key + "_error"] = str(e)
    return out


def warmstart_leg(budget=None, train_seeds=(101, 102, 103, 104, 105), held_seeds=(201, 202, 203, 204, 205),
                  precisions=(0, 1, 2), epochs=20):
    """The learned warm start on the 100k x 20k shape: user and item nets
    trained on the converged factors of the training seeds' matrices, judged
    on held-out seeds against plain FP32 ALS from the same M^(0). For each
    held-out matrix: sweeps and CUDA-event ms to the plain run's final test
    RMSE x (1 + 1e-3), for warm starts fitted in each precision (the warm
    runs' times include computing the warm start), the start the judging
    rule keeps (the one ahead after 5 sweeps) and the gain."""
    import torch
    from paper_2509_18024_gb300 import warmstart
    w = dict(synth.WORKLOADS["zipf_100k"])
    f, lam = w["f"], w["lam"]
    r = budget if budget is not None else w["budget"]
    sweeps = w["sweeps"]

    def draw(seed):
        return synth.zipf_ratings_device(w["n_u"], w["n_m"], w["f"], w["nnz"], w["zipf_s"], w["noise_sd"], seed)

    t0 = time.perf_counter()
    nets, hist = warmstart.train([draw(s) for s in train_seeds], f, lam, r, sweeps=sweeps, hidden=256, epochs=epochs,
                                 batch=4096)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    per_seed = []
    for s in held_seeds:
        prob = draw(s)
        M0 = synth.init_factor(w["n_m"], f, 5000 + s)
        res = warmstart.judge(nets, prob, f, lam, r, M0, sweeps, precisions=precisions)
        per_seed.append({"seed": s, "target_rmse": res["target"], "chosen": res["chosen"],
                         "judge_after": res["judge_after"], "gain": res["gain"],
                         "warm_start_ms": res["warm_start_ms"],
                         "sweeps_to_target": {k: v for k, v in res["sweeps_to_target"].items() if k != "warm"},
                         "ms_to_target": res["ms_to_target"],
                         "rmse_per_sweep": {k: [round(e, 5) for e in v] for k, v in res["curves"].items()
                                            if k != "warm"}})

    def med(key, sub):
        vals = [d[key][sub] for d in per_seed if d[key][sub] is not None]
        return float(statistics.median(vals)) if vals else None
    def med_gain(j, what):
        vals = [d["gain"]["to_plain_after"][j][what] for d in per_seed]
        vals = [v for v in vals if v is not None]
        return float(statistics.median(vals)) if vals else None
    runs = ("plain",) + tuple(f"warm_p{q}" for q in precisions)
    names = {"plain": "FP32 from random M^(0)", "warm_p0": "warm start, FP32",
             "warm_p1": "warm start, TF32 + 1 refinement", "warm_p2": "warm start, BF16 + 2 refinements"}
    return {"metric": "sweeps and ms to the plain FP32 run's final test RMSE (x 1.001)", "workload":
            f"zipf_100k shape (device-drawn), n_f={f}, lambda={lam}, r={r}, {sweeps} sweeps; nets "
            f"{f + 2}-256-256-{f} GELU, trained {epochs} epochs on {len(train_seeds)} seeds",
            "train_s": round(train_s, 1),
            "train_loss_first_last": {k: [v[0], v[-1]] for k, v in hist.items()},
            "median_sweeps": {k: med("sweeps_to_target", k) for k in runs},
            "median_ms": {k: med("ms_to_target", k) for k in runs},
            "warm_start_chosen": sum(d["chosen"] == "warm" for d in per_seed), "held_out_seeds": len(per_seed),
            "early_stopping": {str(j): {"to_rmse_plain_has_after_sweeps": j,
                                        "median_sweeps_saved": med_gain(j, "sweeps_saved"),
                                        "median_ms_saved": med_gain(j, "ms_saved")}
                               for j in per_seed[0]["gain"]["to_plain_after"]},
            "runs": {k: names[k] for k in runs}, "per_seed": per_seed}


def warmstart_arm(args):
    print(json.dumps(warmstart_leg(args.budget)), flush=True)


def batch_leg(seed=1, budget=None, precision="fp32", steps=5, warmup=2):
    """64 independent completion problems fitted as one batch (one sweep of
    all width groups replayed as a CUDA graph), against fitting them one by
    one. Problem q: t ~ U(0, 1), n_u = 500 * 100^t, n_m = 300 * (100/3)^t,
    density log-uniform in [0.5 %, 10 %] (capped at 4 * 10^6 cells), n_f
    uniform over {8, 16, 32, 64, 128}, Zipf(0.9) cells, ratings as the
    100k x 20k workload (rank-32 truth), drawn on the device; r = 0.25."""
    import torch
    from paper_2509_18024_gb300 import core_als
    rng = np.random.default_rng(seed)
    r = budget if budget is not None else 0.25
    prec = PRECISIONS[precision]
    specs, problems = [], []
    for q in range(64):
        t = rng.random()
        n_u, n_m = int(round(500 * 100 ** t)), int(round(300 * (100 / 3) ** t))
        dens = float(np.exp(rng.uniform(np.log(0.005), np.log(0.1))))
        nnz = max(1000, min(int(n_u * n_m * dens), 4_000_000))
        f = int(rng.choice([8, 16, 32, 64, 128]))
        d = synth.zipf_ratings_device(n_u, n_m, 32, nnz, 0.9, 0.5, 3000 + q)
        Ru = core_als.DeviceCSR(n_u, n_m, *d.rows)
        Ri = core_als.DeviceCSR(n_m, n_u, *d.cols)
        specs.append((n_u, n_m, nnz, f))
        problems.append((Ru, Ri, f, torch.empty((n_u, f), device="cuda"),
                         torch.as_tensor(synth.init_factor(n_m, f, 4000 + q)).cuda()))
    rows = sum(a + b for a, b, _, _ in specs)
    batch = core_als.CoreBatch(problems, 0.05, r, precision=prec)
    batch.fit(warmup).synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(batch.stream):
        a.record()
        batch.fit(steps)
        b.record()
    batch.synchronize()
    ms_batch = a.elapsed_time(b) / steps
    launches = batch.launches_per_sweep
    batch.close()
    # The same problems one by one (a handle per width, sweeps issued in turn).
    engines = {}
    for (Ru, Ri, f, U, M) in problems:
        if f not in engines:
            engines[f] = core_als.CoreALS(f, 0.05, r, precision=prec)
        engines[f].prepare(Ru)
        engines[f].prepare(Ri)
    for (Ru, Ri, f, U, M) in problems:
        engines[f].sweep(Ru, Ri, U, M)
    torch.cuda.synchronize()
    a.record()
    for _ in range(steps):
        for (Ru, Ri, f, U, M) in problems:
            engines[f].sweep(Ru, Ri, U, M)
    b.record()
    torch.cuda.synchronize()
    ms_seq = a.elapsed_time(b) / steps
    by_f = {}
    for n_u, n_m, nnz, f in specs:
        e = by_f.setdefault(f, [0, 0, 0])
        e[0] += 1
        e[1] += n_u + n_m
        e[2] += nnz
    out = {"metric": METRIC, "value": rows / (ms_batch / 1e3), "unit": UNIT, "n_gpus": 1, "steps": steps,
           "warmup": warmup, "ms_per_step": ms_batch, "higher_is_better": True, "dtype": precision,
           "data": "synthetic (device-drawn Zipf)",
           "config": {"workload": "batch64: 64 independent problems, 500x300 .. 50kx10k, n_f in {8,16,32,64,128}, "
                                  f"density 0.5-10 %, Zipf 0.9, r={r}", "problems": 64, "row_solves_per_sweep": rows,
                      "cells": int(sum(s[2] for s in specs)),
                      "by_n_f": {str(k): {"problems": v[0], "rows": v[1], "cells": v[2]} for k, v in sorted(by_f.items())}},
           "batched_graph": {"ms_per_sweep": ms_batch, "launches_per_sweep": launches},
           "one_by_one": {"ms_per_sweep": ms_seq, "row_solves_per_s": rows / (ms_seq / 1e3)},
           "speedup_of_batching": ms_seq / ms_batch}
    for e in engines.values():
        e.close()
    return out


def batch_arm(args):
    print(json.dumps(batch_leg(args.seed, args.budget, args.precision, args.steps, args.warmup)), flush=True)


def capture_arm(args):
    """Three half-sweeps of a small single-bucket case (a kernel capture
    takes the second launch with -s 1 -c 1)."""
    import torch
    from paper_2509_18024_gb300 import core_als
    f = args.nf or 32
    r = args.budget if args.budget is not None else 0.25
    csr, Y = synth.capture_case(args.capture_case, f)
    eng = core_als.CoreALS(f, 0.05, r, precision=PRECISIONS[args.precision])
    R = core_als.DeviceCSR.from_host(csr)
    Yd = torch.as_tensor(Y).cuda()
    X = torch.empty((csr.n_rows, f), device="cuda")
    for _ in range(3):
        eng.half_sweep(R, Yd, X)
    torch.cuda.synchronize()
    print(json.dumps({"capture_case": args.capture_case, "n_f": f, "budget": r, "precision": args.precision,
                      "rows": csr.n_rows, "nnz": csr.nnz}), flush=True)


def main():
    args = parse()
    if args.capture_case:
        capture_arm(args)
        return 0
    if args.workload == "warmstart":
        warmstart_arm(args)
        return 0
    if args.workload == "batch64":
        batch_arm(args)
        return 0
    if args.workload == "zipf_1m":
        large_arm(args)
        return 0
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus if args.gpus == 1 else 1)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    w = dict(synth.WORKLOADS[WORKLOAD])
    r = args.budget if args.budget is not None else w["budget"]
    if args.impl == "reference":
        if rank != 0:
            return 0
        p = synth.make_workload(WORKLOAD, seed=args.seed)
        M0 = synth.init_factor(p.n_m, p.f, 1000)
        reference_arm(args, p, w, M0, r)
        return 0

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    p = synth.make_workload(WORKLOAD, seed=args.seed)
    M0 = synth.init_factor(p.n_m, p.f, 1000)
    peaks = None
    if rank == 0 and not args.no_probes:
        import torch
        torch.cuda.set_device(local_rank)
        peaks = peaks_leg()
        args.ffma_peak = peaks.get("fp32_ffma_tflops")
    res = gpu_arm(args, p, w, M0, r, rank, world, local_rank)
    if rank == 0:
        out, eng, _, _ = res
        if peaks is not None:
            out["peaks_measured"] = peaks
            if os.path.exists(PEAKS_FILE):
                with open(PEAKS_FILE) as fh:
                    out["peaks_measured"]["driver_measured_peaks_file"] = json.load(fh)
        out["e2e"] = e2e_leg(p, w, r, M0)
        out["e2e_fit_15_sweeps"] = e2e_leg(p, w, r, M0, steps=2, sweeps=15)
        if not args.no_variants:
            out["variants_rows_per_s"] = variants(p, w, M0, [
                ("full_als_fp32", 1.0, "full", "fp32"), ("core_r0.10_fp32", 0.10, "asym", "fp32"),
                ("core_r0.50_fp32", 0.50, "asym", "fp32"), ("core_r0.25_fp32_tc", r, "asym", "fp32_tc"),
                ("core_r0.25_tf32", r, "asym", "tf32"), ("core_r0.25_bf16", r, "asym", "bf16"),
                ("full_als_bf16", 1.0, "full", "bf16"),
                ("core_fast_r0.25_fp32", r, "asym", "fp32", {"sketch": "factor"}),
                ("core_fast_r0.25_bf16", r, "asym", "bf16", {"sketch": "factor"}),
                ("core_fixed_s8_fp32", r, "asym", "fp32", {"fixed_keep": 8}),
                ("core_fixed_s32_fp32", r, "asym", "fp32", {"fixed_keep": 32})])
            out["time_to_rmse"] = time_to_rmse(p, w, M0, [
                ("core_fp32", r, "asym", "fp32"), ("core_tf32", r, "asym", "tf32"), ("core_bf16", r, "asym", "bf16"),
                ("core_fp32_tc", r, "asym", "fp32_tc"), ("full_fp32", 1.0, "full", "fp32"),
                ("core_fast_fp32", r, "asym", "fp32", {"sketch": "factor"}),
                ("core_fixed_s32_fp32", r, "asym", "fp32", {"fixed_keep": 32})])
        if world == 1 and not args.no_cpu_baseline:
            rate, done, t_sweep = oracle_sample(p, M0, w["lam"], r, 40000, 8000, 7)
            import oracle
            out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                                   "sample": f"{done} random rows (40000 user + 8000 item rows), one half-sweep "
                                             f"each, extrapolated to a full sweep by observed entries "
                                             f"(est. {t_sweep:.1f} s per sweep)"}
            # The same oracle on one core (a smaller sample of the same rows' kind).
            all_cores = oracle.num_threads()
            oracle.set_threads(1)
            try:
                rate1, done1, t1 = oracle_sample(p, M0, w["lam"], r, 4000, 800, 7)
            finally:
                oracle.set_threads(all_cores)
            out["cpu_baseline"]["one_core"] = {
                "value": rate1, "unit": UNIT, "cores": 1,
                "sample": f"{done1} random rows (4000 user + 800 item rows), extrapolated likewise "
                          f"(est. {t1:.1f} s per sweep)"}
            out["small_workload"] = small_leg(M0_seed=1000)
        if world == 1 and not args.no_sim:
            out["simulation_metrics"] = simulation_leg()
        if world == 1 and not args.no_batch:
            out["batch64"] = batch_leg(args.seed, None, "fp32", steps=3, warmup=1)
        if world == 1 and not args.no_warm:
            out["warm_start"] = warmstart_leg(train_seeds=(101, 102, 103), held_seeds=(201, 202),
                                              precisions=(0, 2), epochs=12)
        if world == 1 and not args.no_large:
            import torch
            eng.close()
            torch.cuda.empty_cache()
            d, wl, gen_s = draw_large(args.seed)
            out["zipf_1m_nf128"] = {"workload": f"zipf_1m: {wl['n_u']} users x {wl['n_m']} items, {wl['nnz']} cells "
                                                f"(Zipf {wl['zipf_s']}), n_f=128, lambda={wl['lam']}, "
                                                f"r={wl['budget']}, asymmetric Eq. core_ui; 2 timed sweeps each",
                                    "generation_s": round(gen_s, 1)}
            for prec in ("fp32", "bf16"):
                out["zipf_1m_nf128"][prec] = large_leg(d, wl, 128, prec, steps=2, warmup=1, seed=args.seed)
                torch.cuda.empty_cache()
            # n_f = 64: FP32 against BF16 with one refinement step (its error
            # against the FP64 oracle stays under the 1e-5 bar of FP32).
            out["zipf_1m_nf64"] = {"workload": out["zipf_1m_nf128"]["workload"].replace("n_f=128", "n_f=64")}
            for prec, ref in (("fp32", None), ("bf16", 1)):
                key = prec if ref is None else f"{prec}_refine{ref}"
                out["zipf_1m_nf64"][key] = large_leg(d, wl, 64, prec, steps=2, warmup=1, seed=args.seed, refine=ref)
                torch.cuda.empty_cache()
            del d
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
