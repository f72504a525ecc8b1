#!/usr/bin/env python
"""Benchmark of the QML hot path on one or more GB300s (one process per GPU).

Workload: TQU, HEALPix Nside 16 with the |b| < 20 deg cut (n = 5952 rows),
l = 2..47 (k = 6900 modes), six spectra, dense rank-200 noise, 100 simulated
maps.  One step = qml_fisher (Y build, C = Y Lambda Y^T + N, Cholesky,
X = L^-1 Y, W = X^T X, Fisher block sums, noise bias, eigendecomposition of F)
+ qml_estimate on the 100 maps (y, deconvolved / decorrelated / convolved Cl)
+ pix_loglike of one map at the fiducial spectra.  Metric: Fisher + Cl solves
per second over all ranks (weak scaling: every rank solves its own replica).

--impl reference times the CPU oracle (float64 numpy/scipy on the host
cores) on the same workload, one solve per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Fisher+Cl solves/s (TQU Nside16 l2-47, 100 sims)"
# DRAM bytes (read + write) of one W = X^T X launch of dgemm_kernel<1,0,4,4>
# at this workload, from one ncu capture of that kernel (set to None when the
# kernel changes until it is captured again)
DGEMM_SYRK_TRAFFIC = 8.550515e9 + 0.187149e9
DGEMM_SYRK_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                             "--set full capture of this launch")
# the same for the split kernel (ozaki_gemm_kernel<8, 2>, clusters of two) on
# W = X^T X at this workload; None when the kernel changes until recaptured
OZ_SYRK_TRAFFIC = 5.69e9 + 0.17715e9
OZ_SYRK_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one capture of "
                          "the kernel alone (slicing not included), banded work order")
UNIT = "solves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--nsims", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the split-precision forms")
    ap.add_argument("--no-fp64-qu32", action="store_true",
                    help="skip the float64 solves of the QU Nside 32 workload")
    ap.add_argument("--scan-items", type=int, default=4096,
                    help="items per pix_loglike_batch call of the split-Kt scan form")
    ap.add_argument("--emulator-full", action="store_true",
                    help="also run the emulator at TQU Nside 16 with 50k exact labels "
                         "(about ten minutes)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def workload_config(nsims):
    from paper_2605_21149_gb300 import synth
    wl = synth.workload(1)
    return wl, {"workload": f"{wl.name}: TQU HEALPix Nside 16, |b|<20 deg cut, n={wl.n} rows, "
                            f"l=2..47 (k={wl.k}), 6 spectra, dense rank-200 N, {nsims} sims",
                "n": wl.n, "k": wl.k, "nsims": nsims,
                "l2": "inputs larger than L2 (N 283 MB, Y 329 MB, W 381 MB per step)"}


# ------------------------------------------------------------- oracle ----
def oracle_solve(wl, Y, maps):
    from oracle import qml
    return qml.qml_for(wl, Y, maps=maps)


def oracle_inputs(wl, nsims):
    from oracle import harmonic, qml
    from paper_2605_21149_gb300 import synth
    g = synth.rng(1, synth.P_SIMS)
    alm = synth.draw_alm(wl.cl_fid, wl.lmin, wl.lmax, wl.comps, nsims, g)
    noise = synth.noise_draws(wl.G, nsims, g)
    Y = harmonic.build_Y_for(wl)
    return Y, qml.simulate(Y, alm, noise)


def aggregate(t_local, steps, world, device=None):
    """Whole-job rate over `world` replicas: every rank timed `steps` steps;
    the slowest rank's time counts (max over ranks, after a barrier)."""
    t = t_local
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([t_local], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dist.barrier()
        t = float(tt.item())
    return world * steps / t, t


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl, cfg = workload_config(args.nsims)
    Y, maps = oracle_inputs(wl, args.nsims)
    for _ in range(args.warmup):
        oracle_solve(wl, Y, maps)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_solve(wl, Y, maps)
    t = time.perf_counter() - t0
    v = args.steps / t
    cores = cpu_cores()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "one full Fisher + Cl solve per step (oracle, numpy/scipy "
                                       "float64 on the host cores)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- clocks ----
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.proc = None
        self.gpu_id = gpu_id

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return parse_clock_csv(out)


def parse_clock_csv(text):
    """Median SM clock, maximum SM clock and the throttle reasons seen in the
    nvidia-smi samples (ClockSampler.FIELDS, csv without header or units);
    lines that do not parse are skipped."""
    sm, mx, reasons = [], [], set()
    names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
    for ln in text.splitlines():
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 8:
            continue
        try:
            sm.append(float(f[0]))
            mx.append(float(f[1]))
        except ValueError:
            continue
        for nm, v in zip(names, f[4:8]):
            if v.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
            "samples": len(sm)}


# ---------------------------------------------------------------- ours ----
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {}


def measure_fp64_peak(torch, n=8192, reps=4):
    """cuBLAS DGEMM (torch.matmul float64) throughput: the float64 denominator."""
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    del a, b
    torch.cuda.empty_cache()
    return best


def summarize(value, forms):
    """Solves/s and lnL evals/s of every form against the plain float64 GPU
    path, with the relative errors against the oracle (or float64 path)."""
    if not forms:
        return {"tqu16_fp64_solves_s": value}

    def get(*keys):
        d = forms
        for k in keys:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d
    r = lambda x: None if x is None else float("%.4g" % x)
    out = {"tqu16_fp64_solves_s": r(value),
           "tqu16_split_solves_s": r(get("split_bf16", "value")),
           "tqu16_split_speedup": r(get("split_bf16", "speedup_vs_fp64")),
           "tqu16_rel_err_fp64": {k: r(v) for k, v in (get("rel_err_tqu16", "fp64") or {}).items()},
           "tqu16_rel_err_split": {k: r(v) for k, v in (get("rel_err_tqu16", "split_bf16") or {}).items()},
           "qu32_split_solves_s": r(get("qu_nside32", "split_bf16", "value")),
           "qu32_fp64_solves_s": r(get("qu_nside32", "fp64", "value")),
           "qu32_split_speedup": r(get("qu_nside32", "split_speedup_vs_fp64")),
           "qu32_rel_err_split_vs_fp64": {k: r(v) for k, v in
                                          (get("qu_nside32", "rel_err_split_vs_fp64") or {}).items()
                                          if k != "note"},
           "scan_split_kt_evals_s": r(get("lnl_batch", "split_kt", "value")),
           "scan_split_kt_items_per_call": get("lnl_batch", "split_kt", "items_per_call"),
           "scan_split_fp64kt_evals_s": r(get("lnl_batch", "split_fp64kt", "value")),
           "scan_fp64_evals_s": r(get("lnl_batch", "fp64", "value")),
           "mc1000_split_sims_s": r(get("mc_rhs_1000", "split_bf16", "value")),
           "mc1000_fp64_sims_s": r(get("mc_rhs_1000", "fp64", "value")),
           "split_gemm_bf16_frac": r(get("roofline_split", "frac")),
           "emu_points_s": r(get("emulator", "inference_points_per_s"))}
    return out


def rel_errors(F, est, lnl, ld, ref):
    """Errors of one GPU solve against the oracle (S20 metrics)."""
    import numpy as np
    F = F.cpu().numpy()
    Fr = ref["F"]
    sig = np.sqrt(np.diag(np.linalg.inv(Fr)))[:, None]
    cd, cdr = est["cl_deconv"].cpu().numpy(), ref["cl_deconv"]
    cc, ccr = est["cl_decorr"].cpu().numpy(), ref["cl_decorr"]
    lnl = float(lnl.cpu().numpy().ravel()[0])
    ld = float(ld.cpu().numpy().ravel()[0])
    return {"F": float(np.abs(F - Fr).max() / np.abs(Fr).max()),
            "cl_deconv": float((np.abs(cd - cdr) / np.maximum(np.abs(cdr), sig)).max()),
            "cl_decorr": float((np.abs(cc - ccr) / np.maximum(np.abs(ccr), 1.0)).max()),
            "lnL": abs(lnl - float(ref["lnL"][0])) / abs(float(ref["lnL"][0])),
            "logdet": abs(ld - float(ref["logdet"])) / abs(float(ref["logdet"]))}


def emulator_form(api, torch, td, full=False):
    """full=False: TQU Nside 8 (f_sky 0.7, l <= 15), 8192 exact labels;
    full=True: the TQU Nside 16 setup (|b| < 20 deg, l <= 47), 50k exact labels
    from the batched scan with split-precision Kt (about ten minutes)."""
    import numpy as np
    from paper_2605_21149_gb300 import synth
    if full:
        wl = synth.make_workload("emu TQU nside16", 16, 47, True, True, 20.0, synth.SPEC_NAMES,
                                 200, 41)
        prob = api.Problem.from_workload(wl, device=True, precision=1)
        ntrain = 50000
    else:
        wl = synth.make_workload("emu TQU nside8", 8, 15, True, True, synth.fsky_cut_deg(0.7),
                                 synth.SPEC_NAMES, 20, 40)
        prob = api.Problem.from_workload(wl, device=True)
        ntrain = 8192
    g = synth.rng(40, synth.P_EMU)
    alm = synth.draw_alm(synth.spectra(wl.lmax), wl.lmin, wl.lmax, wl.comps, 1, g)
    maps = api.synthesize(prob, td(alm), td(synth.noise_draws(wl.G, 1, g)))
    lo = np.array([0.042, 0.0, 0.7, 0.7])
    hi = np.array([0.078, 0.1, 1.3, 1.3])
    naudit, ninf = 1024, 1 << 20
    if full:
        api.tune_set("batch_split_kt", 1)
    # inference box 5 % wider than the training box, so that the hull check fires
    ilo, ihi = lo - 0.025 * (hi - lo), hi + 0.025 * (hi - lo)

    def exact(th):
        cl = np.stack([synth.spectra(wl.lmax, tau=t[0], r=t[1], a_ee=t[2], a_tt=t[3]) for t in th])
        cl_d = torch.as_tensor(cl, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lnl, _, _ = api.loglike_batch([(prob, maps)], np.zeros(len(th), dtype=np.int32), cl_d)
        torch.cuda.synchronize()
        return lnl[:, 0].cpu().numpy(), time.perf_counter() - t0

    th = lo + (hi - lo) * g.uniform(size=(ntrain, 4))
    y, t_lab = exact(th)
    emu = api.Emulator(lo, hi, seed=11)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    emu.train(th, y, epochs=100, batch=64, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    thi = torch.as_tensor(ilo + (ihi - ilo) * g.uniform(size=(ninf, 4)), device="cuda")
    # steady state of repeated calls: one untimed call of the same size sizes
    # the emulator's inference buffers, which it keeps between calls
    emu.predict(thi)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    _, fl = emu.predict(thi)
    ev1.record()
    ev1.synchronize()
    t_inf = ev0.elapsed_time(ev1) * 1e-3
    ta = ilo + (ihi - ilo) * g.uniform(size=(naudit, 4))
    pa, fa = emu.predict(ta)
    ya, _ = exact(ta)
    acc = np.asarray(fa) == 0
    err = np.abs(np.asarray(pa) - ya)
    emu.free()
    if full:
        api.tune_set("batch_split_kt", 0)
    wname = (f"TQU Nside 16 l=2..47 |b|<20 deg (n={wl.n}), split-precision labels"
             if full else f"TQU Nside 8 l=2..15 f_sky 0.7 (n={wl.n})")
    return {"workload": wname + ", theta=(tau, r, A_EE, A_TT), MLP 4x256 GELU, 2 heads",
            "labels": ntrain, "held_out": ntrain // 8, "label_evals_per_s": ntrain / t_lab,
            "train_s": t_train, "epochs": 100, "inference_points": ninf,
            "inference_box": "training box widened by 5 %",
            "inference_points_per_s": ninf / t_inf, "tol_abs_dlnL": 0.05,
            "fallback_rate": float((fl != 0).float().mean().item()),
            "audit": {"points": naudit, "accepted": float(acc.mean()),
                      "max_abs_dlnL_accepted": float(err[acc].max()) if acc.any() else None,
                      "median_abs_dlnL_accepted": float(np.median(err[acc])) if acc.any() else None}}


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2605_21149_gb300 import _native, api, build, synth
    build.build()
    lib = _native.load()

    wl, cfg = workload_config(args.nsims)
    cfg["parallelism"] = f"replicas x{world} (no data-path collective)"

    # ---- CPU baseline (rank 0, N = 1 only): the oracle as it stands; its
    # solve is kept as the reference of the forms' relative errors
    cpu = None
    oref = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import qml as oqml
        Y, omaps = oracle_inputs(wl, args.nsims)
        t0 = time.perf_counter()
        ref = oracle_solve(wl, Y, omaps)
        tc = time.perf_counter() - t0
        cpu = {"value": 1.0 / tc, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": "one full Fisher + Cl (100 sims) solve of this workload, "
                         f"{tc:.1f} s (numpy/scipy float64)"}
        lnl_ref, _, ld_ref = oqml.loglike(ref["C"], omaps[:, :1])
        oref = {"F": ref["F"], "cl_deconv": ref["cl_deconv"], "cl_decorr": ref["cl_decorr"],
                "y": ref["y"], "lnL": lnl_ref, "logdet": ld_ref, "maps": omaps}
        del Y, ref

    # ---- device inputs
    prob = api.Problem.from_workload(wl, device=True)
    g = synth.rng(1, synth.P_SIMS)
    alm = synth.draw_alm(wl.cl_fid, wl.lmin, wl.lmax, wl.comps, args.nsims, g)
    noise = synth.noise_draws(wl.G, args.nsims, g)
    td = lambda x: torch.as_tensor(x, device="cuda").t().contiguous().t()
    maps = api.synthesize(prob, td(alm), td(noise))
    cl_dev = torch.as_tensor(wl.cl_fid.reshape(-1), device="cuda")
    map1 = maps[:, :1]

    def step():
        F, plan = api.fisher(prob)
        plan.estimate(maps)
        api.loglike(prob, cl_dev, map1)
        plan.free()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    dev_uuid = str(getattr(torch.cuda.get_device_properties(local), "uuid", local))
    if dev_uuid and not dev_uuid.startswith("GPU-") and len(dev_uuid) > 8:
        dev_uuid = "GPU-" + dev_uuid
    sampler = ClockSampler(dev_uuid)
    sampler.start()
    time.sleep(0.3)
    c0 = lib.qml_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    c1 = lib.qml_launch_count()
    clocks = sampler.stop()
    value, t = aggregate(e0.elapsed_time(e1) * 1e-3, args.steps, world, device="cuda")

    # ---- lnL evals/s (single map, fiducial spectra) and the dominant kernel
    lnl_rate = None
    roof = None
    if rank == 0:
        reps = max(2, args.steps)
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record()
        for _ in range(reps):
            api.loglike(prob, cl_dev, map1)
        e3.record()
        e3.synchronize()
        lnl_rate = reps / (e2.elapsed_time(e3) * 1e-3)
        # dominant kernel: float64 tiled GEMM; timed on its largest launch of the
        # step (W = X^T X, lower triangle: k x k x n) with CUDA events on the
        # stream it runs on
        X = torch.randn(wl.k, wl.n, dtype=torch.float64, device="cuda").t()
        W = torch.empty(wl.k, wl.k, dtype=torch.float64, device="cuda").t()
        api.gemm(X, X, W, transA=True, lower=True)
        reps_g = 3
        e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e4.record()
        for _ in range(reps_g):
            api.gemm(X, X, W, transA=True, lower=True)
        e5.record()
        e5.synchronize()
        dur = e4.elapsed_time(e5) * 1e-3 / reps_g
        flops = float(wl.k) * wl.k * wl.n  # k(k+1)/2 outputs x 2n flops
        achieved = flops / dur / 1e12
        del X, W
        torch.cuda.empty_cache()
        fp64_peak = measure_fp64_peak(torch)
        roof = {"kernel": "dgemm_kernel<T,N> (W = X^T X lower, k=6900, n=5952)",
                "bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak,
                "peak_source": "cuBLAS DGEMM (torch.matmul float64 8192^3, best of 4) "
                               "measured in this run; MEASURED_PEAKS.json has no float64 entry",
                "traffic": DGEMM_SYRK_TRAFFIC, "traffic_source": DGEMM_SYRK_TRAFFIC_SOURCE,
                "flops_per_launch": flops, "ms_per_launch": dur * 1e3}

    # ---- split-precision form (bf16 digits on tcgen05, float64 recombination;
    # 1e-8 against the float64 oracle in tests/test_gpu_split_pipeline.py)
    forms = None
    if rank == 0 and not args.no_forms:
        forms = {}
        prob_s = api.Problem.from_workload(wl, device=True, precision=1)

        def step_s():
            F, plan = api.fisher(prob_s)
            plan.estimate(maps)
            api.loglike(prob_s, cl_dev, map1)
            plan.free()
        for _ in range(max(2, args.warmup)):
            step_s()
        torch.cuda.synchronize()
        e6, e7 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e6.record()
        for _ in range(args.steps):
            step_s()
        e7.record()
        e7.synchronize()
        ts = e6.elapsed_time(e7) * 1e-3
        forms["split_bf16"] = {"workload": cfg["workload"], "value": args.steps / ts, "unit": UNIT,
                               "ms_per_step": 1e3 * ts / args.steps,
                               "speedup_vs_fp64": (args.steps / ts) / (args.steps / (t / world)),
                               "tolerance": "1e-8 vs float64 oracle"}
        # the opt-in float-float 64-wide diagonal blocks of the split Cholesky
        # (tuning key split_diag_df; the default keeps them in float64)
        api.tune_set("split_diag_df", 1)
        try:
            step_s()
            torch.cuda.synchronize()
            e6.record()
            for _ in range(args.steps):
                step_s()
            e7.record()
            e7.synchronize()
        finally:
            api.tune_set("split_diag_df", 0)
        tdf = e6.elapsed_time(e7) * 1e-3
        forms["split_bf16"]["float_float_diagonal"] = {
            "value": args.steps / tdf, "unit": UNIT, "ms_per_step": 1e3 * tdf / args.steps,
            "note": "64-wide Cholesky diagonal blocks and their row solves in float-float "
                    "(split_diag_df = 1); the default factors them in float64"}
        # native multipole binning (Sect. 2.4), Delta l = 2: qml_fisher +
        # qml_estimate (100 maps) with and without bins on the split path
        try:
            edges = list(range(wl.lmin, wl.lmax + 2, 2))
            if edges[-1] != wl.lmax + 1:
                edges.append(wl.lmax + 1)
            prob_b = api.Problem.from_workload(wl, device=True, precision=1, bin_edges=edges)

            def fisher_estimate(pr):
                F, plan = api.fisher(pr)
                plan.estimate(maps)
                plan.free()
            tb = {}
            for name, pr in (("binned", prob_b), ("per_l", prob_s)):
                fisher_estimate(pr)
                torch.cuda.synchronize()
                e6.record()
                for _ in range(args.steps):
                    fisher_estimate(pr)
                e7.record()
                e7.synchronize()
                tb[name] = e6.elapsed_time(e7) / args.steps
            forms["binned_dl2"] = {
                "workload": cfg["workload"], "bins_per_spectrum": len(edges) - 1,
                "ms_fisher_estimate_binned": tb["binned"], "ms_fisher_estimate_per_l": tb["per_l"],
                "binning_overhead_ms": tb["binned"] - tb["per_l"],
                "note": "split precision; bins sum the per-l F, noise bias and y "
                        "(two small kernels) before the three normalisations"}
        except Exception as ex:  # report, do not lose the rest of the line
            forms["binned_dl2"] = {"error": f"{type(ex).__name__}: {ex}"}
        # relative errors of the float64 and split forms against the oracle's
        # solve of the same maps (the CPU-baseline leg), S20 metrics
        if oref is not None:
            om = td(oref["maps"])
            rel = {"reference": "oracle (numpy/scipy float64) on the same 100 maps; F: max|dF|/"
                                "max|F|, Cl: |dC| / max(|C|, sqrt((F^-1)_aa)), decorrelated: "
                                "|dC| / max(|C|, 1), lnL and ln|C|: relative"}
            for name, pr in (("fp64", prob), ("split_bf16", prob_s)):
                F_, pl_ = api.fisher(pr)
                e_ = pl_.estimate(om)
                l_, _, d_ = api.loglike(pr, cl_dev, om[:, :1])
                pl_.free()
                rel[name] = rel_errors(F_, e_, l_, d_, oref)
            forms["rel_err_tqu16"] = rel
        # the QU Nside 32 split-precision workload (n = 17152, k = 18424): 3
        # timed steps of each precision after one untimed step
        wl3 = synth.workload(2)
        p3s = api.Problem.from_workload(wl3, device=True, precision=1)
        g3 = synth.rng(2, synth.P_SIMS)
        alm3 = synth.draw_alm(wl3.cl_fid, wl3.lmin, wl3.lmax, wl3.comps, 2, g3)
        noise3 = synth.noise_draws(wl3.G, 2, g3)
        maps3 = api.synthesize(p3s, td(alm3), td(noise3))
        cl3 = torch.as_tensor(wl3.cl_fid.reshape(-1), device="cuda")

        def step3(pr):
            F, plan = api.fisher(pr)
            est = plan.estimate(maps3)
            _, _, ld = api.loglike(pr, cl3, maps3[:, :1])
            plan.free()
            return F, est, ld

        def timed3(pr, nrep):
            out = step3(pr)
            torch.cuda.synchronize()
            e8, e9 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e8.record()
            for _ in range(nrep):
                out = step3(pr)
            e9.record()
            e9.synchronize()
            return e8.elapsed_time(e9) * 1e-3 / nrep, out

        t3s, out_s = timed3(p3s, 3)
        f3 = {"workload": f"{wl3.name}: QU HEALPix Nside 32, f_sky 0.7 cut, n={wl3.n}, "
                          f"l=2..95 (k={wl3.k}), 3 spectra, rank-200 N, 2 maps",
              "split_bf16": {"value": 1.0 / t3s, "unit": UNIT, "ms_per_step": 1e3 * t3s,
                             "steps": 3}}
        if not args.no_fp64_qu32:
            p3d = api.Problem.from_workload(wl3, device=True, precision=0)
            t3d, out_d = timed3(p3d, 3)
            f3["fp64"] = {"value": 1.0 / t3d, "unit": UNIT, "ms_per_step": 1e3 * t3d, "steps": 3}
            f3["split_speedup_vs_fp64"] = t3d / t3s
            Fs, Fd = out_s[0].cpu().numpy(), out_d[0].cpu().numpy()
            sig = np.sqrt(np.diag(np.linalg.inv(Fd)))[:, None]
            cs, cd = out_s[1]["cl_deconv"].cpu().numpy(), out_d[1]["cl_deconv"].cpu().numpy()
            lds, ldd = float(out_s[2].cpu().numpy().ravel()[0]), float(out_d[2].cpu().numpy().ravel()[0])
            f3["rel_err_split_vs_fp64"] = {
                "F": float(np.abs(Fs - Fd).max() / np.abs(Fd).max()),
                "cl_deconv": float((np.abs(cs - cd) / np.maximum(np.abs(cd), sig)).max()),
                "logdet": abs(lds - ldd) / abs(ldd),
                "note": "against this GPU's float64 path on the same maps (the float64 path "
                        "matches the oracle to 1e-10 at TQU Nside 16; the split path matches "
                        "the oracle at this workload to 1e-8 in the tests)"}
            del p3d, out_d
        forms["qu_nside32"] = f3
        del p3s, maps3, out_s
        torch.cuda.empty_cache()
        # batched likelihood scan (the 64 x 64 (tau, r) grid, item i on mask
        # i mod 3 of the f_sky 0.5 / 0.7 / 0.9 TQU Nside 16 masks).  Three forms:
        # split-precision masks with the split inner factor Kt (tuning key
        # batch_split_kt = 1) on args.scan_items items per call (the whole grid:
        # 4096); split-precision masks with the default float64 Kt, and float64
        # throughout, on 256 items per call.  Each rate excludes the per-mask
        # setup: items/s = (N - 3) / (t(N items) - t(3 items)).
        bmasks, btaus, brs = synth.batch_workload(nside=16, lmax=47)
        bres = {"workload": "lnL scan: TQU Nside 16 l=2..47 (k=6900), masks f_sky 0.5/0.7/0.9 "
                            "(n=4800/6336/8256), 1 map per mask, items of the 64 x 64 (tau, r) grid"}

        def scan_masks(prec):
            out = []
            for j, wl_b in enumerate(bmasks):
                pb = api.Problem.from_workload(wl_b, device=True, precision=prec)
                gb = synth.rng(30 + j, synth.P_MAPS)
                ab = synth.draw_alm(wl_b.cl_fid, wl_b.lmin, wl_b.lmax, wl_b.comps, 1, gb)
                nzb = synth.noise_draws(wl_b.G, 1, gb)
                out.append((pb, api.synthesize(pb, td(ab), td(nzb))))
            return out

        def scan_items(nitems):
            sel = np.linspace(0, len(btaus) - 1, nitems).astype(int)
            return (sel % len(bmasks),
                    torch.as_tensor(synth.batch_item_spectra(47, btaus[sel], brs[sel]),
                                    device="cuda"))

        def timed_scan(bprobs, nitems):
            im3, cl3_ = scan_items(3)
            im, cl_ = scan_items(nitems)
            api.loglike_batch(bprobs, im3, cl3_)
            torch.cuda.synchronize()
            ts = []
            for im_, c_ in ((im3, cl3_), (im, cl_)):
                e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0_.record()
                api.loglike_batch(bprobs, im_, c_)
                e1_.record()
                e1_.synchronize()
                ts.append(e0_.elapsed_time(e1_) * 1e-3)
            rate = (nitems - 3) / (ts[1] - ts[0])
            return {"value": rate, "unit": "lnL evals/s", "items_per_call": nitems,
                    "ms_per_call": 1e3 * ts[1], "mask_setup_ms": 1e3 * (ts[0] - 3 / rate)}

        kdim = bmasks[0].k
        kt_flops = kdim ** 3 / 3.0
        bsplit = scan_masks(1)
        api.tune_set("batch_split_kt", 1)
        try:
            # schedule autotuner (worker streams x graph replay) on 32 items
            im32, cl32 = scan_items(32)
            rates = api.autotune_batch(bsplit, im32, cl32)
            bres["autotune"] = {"candidates": {f"streams={k[0]},graphs={k[1]}": v
                                               for k, v in rates.items()},
                                "chosen": {"batch_streams": api.tune_get("batch_streams"),
                                           "batch_graphs": api.tune_get("batch_graphs")},
                                "tuned_gemm_shapes": api.tune_table().count("dgemm:")}
            bres["split_kt"] = timed_scan(bsplit, args.scan_items)
            bres["split_kt"]["note"] = ("split masks and split trailing updates of each item's "
                                        "Kt (batch_split_kt = 1); float64 diagonal blocks and ln|Kt|")
        finally:
            api.tune_set("batch_split_kt", 0)
        bres["split_fp64kt"] = timed_scan(bsplit, 256)
        bres["split_fp64kt"]["note"] = ("split masks (N factor, M = U^T U), each item's Kt "
                                        "factored in native float64 (the default)")
        del bsplit
        torch.cuda.empty_cache()
        bfp = scan_masks(0)
        bres["fp64"] = timed_scan(bfp, 256)
        del bfp
        torch.cuda.empty_cache()
        for key in ("split_kt", "split_fp64kt", "fp64"):
            # the item's dominant work, the Kt Cholesky, as float64-equivalent flops
            bres[key]["kt_factor_fp64_equiv_tflops"] = bres[key]["value"] * kt_flops / 1e12
        bres["split_kt_speedup_vs_fp64"] = bres["split_kt"]["value"] / bres["fp64"]["value"]
        bres["split_fp64kt_speedup_vs_fp64"] = bres["split_fp64kt"]["value"] / bres["fp64"]["value"]
        forms["lnl_batch"] = bres
        # Monte Carlo right-hand sides: 1000 simulated maps through one plan
        # (TQU Nside 16), float64 and split precision
        nmc = 1000
        gmc = synth.rng(1, synth.P_SIMS)
        mc_maps = api.synthesize(prob, td(synth.draw_alm(wl.cl_fid, wl.lmin, wl.lmax, wl.comps, nmc, gmc)),
                                 td(synth.noise_draws(wl.G, nmc, gmc)))
        mres = {"workload": "TQU Nside 16 l=2..47, 1000 simulated maps per qml_estimate call "
                            "(plan from one qml_fisher)"}
        for prec, name in ((0, "fp64"), (1, "split_bf16")):
            pm = api.Problem.from_workload(wl, device=True, precision=prec)
            _, plan_mc = api.fisher(pm)
            plan_mc.estimate(mc_maps)  # warm-up at the timed shape (tile tuning happens here)
            torch.cuda.synchronize()
            em0, em1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            em0.record()
            plan_mc.estimate(mc_maps)
            em1.record()
            em1.synchronize()
            tmc = em0.elapsed_time(em1) * 1e-3
            mres[name] = {"value": nmc / tmc, "unit": "sims/s", "ms_per_call": 1e3 * tmc}
            plan_mc.free()
        forms["mc_rhs_1000"] = mres
        del mc_maps
        torch.cuda.empty_cache()
        # harmonic (SMW) basis against the pixel basis on the same workload,
        # qml_fisher + qml_estimate (100 maps); float64 and split precision
        def fisher_estimate_ms(pr, mp, reps=2):
            F_, pl_ = api.fisher(pr)
            pl_.estimate(mp)
            pl_.free()
            torch.cuda.synchronize()
            e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0_.record()
            for _ in range(reps):
                F_, pl_ = api.fisher(pr)
                pl_.estimate(mp)
                pl_.free()
            e1_.record()
            e1_.synchronize()
            return e0_.elapsed_time(e1_) / reps

        hres = {"workload": cfg["workload"],
                "note": "qml_fisher + qml_estimate (100 maps); the two bases agree to 1e-11 on F"}
        for prec, pname in ((0, "fp64"), (1, "split_bf16")):
            for basis, bname in ((0, "pixel"), (1, "harmonic")):
                pr = api.Problem.from_workload(wl, device=True, precision=prec, basis=basis)
                hres[f"{bname}_{pname}_ms"] = fisher_estimate_ms(pr, maps)
        forms["harmonic_basis"] = hres
        torch.cuda.empty_cache()
        # multipole switching: TQU Nside 16 estimated on l = 2..47 with the
        # signal band to l_max^sig = 4 Nside = 64 (k_sig = 12663), split precision
        wls = synth.make_workload("TQU nside16 lsig64", 16, 64, True, True, 20.0,
                                  synth.SPEC_NAMES, 200, 21)
        gs_ = synth.rng(21, synth.P_SIMS)
        psig = api.Problem.from_workload(wls, device=True, precision=1)
        maps_s = api.synthesize(psig, td(synth.draw_alm(wls.cl_fid, 2, 64, wls.comps, 100, gs_)),
                                td(synth.noise_draws(wls.G, 100, gs_)))
        sres = {"workload": "TQU Nside 16, window l = 2..47, signal band l = 2..64, 100 maps"}
        for basis, bname in ((0, "pixel"), (1, "harmonic")):
            pr = api.Problem.from_workload(wls, device=True, precision=1, window=(2, 47),
                                           basis=basis)
            sres[f"{bname}_split_ms"] = fisher_estimate_ms(pr, maps_s)
        forms["switching_lsig64"] = sres
        del psig, maps_s
        torch.cuda.empty_cache()
        # cross-QML (Eq. q_cross): two noise realisations of the TQU Nside 16
        # setup, 100 map pairs, split precision (two qml_fisher + qml_cross)
        wl2 = synth.make_workload("TQU nside16 noise 2", 16, 47, True, True, 20.0,
                                  synth.SPEC_NAMES, 200, 51)
        p1x = api.Problem.from_workload(wl, device=True, precision=1)
        p2x = api.Problem.from_workload(wl2, device=True, precision=1)
        maps2 = api.synthesize(p2x, td(alm), td(synth.noise_draws(wl2.G, args.nsims, g)))

        def cross_once():
            _, q1 = api.fisher(p1x)
            _, q2 = api.fisher(p2x)
            api.cross(q1, q2, maps, maps2)
            q1.free()
            q2.free()
        cross_once()
        torch.cuda.synchronize()
        e0x, e1x = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0x.record()
        cross_once()
        e1x.record()
        e1x.synchronize()
        forms["cross_qml"] = {"workload": "TQU Nside 16 l=2..47, two noise realisations, "
                                          f"{args.nsims} map pairs, split precision",
                              "ms_two_fishers_plus_cross": e0x.elapsed_time(e1x)}
        del p1x, p2x, maps2
        torch.cuda.empty_cache()
        # the Sect. 4 validation experiments (paper_2605_21149_gb300.validate):
        # mean-chi^2 r scan (31 points, 1000 maps at r = 0) and the Fisher vs
        # scatter test over five sky fractions (1000 maps each), QU Nside 16,
        # l = 2..32
        from paper_2605_21149_gb300 import validate
        wlr = synth.make_workload("QU nside16 l32 cut10", 16, 32, False, True, 10.0,
                                  ("EE", "BB", "EB"), 10, 81)
        t0v = time.perf_counter()
        rs = validate.mean_chi2_rscan(wlr, np.linspace(0.0, 0.01, 31), r_true=0.0, nsims=1000)
        t_rs = time.perf_counter() - t0v
        t0v = time.perf_counter()
        sw = validate.fsky_sweep(16, 32, (0.0, 10.0, 18.0, 30.0, 40.0), nsims=1000)
        t_sw = time.perf_counter() - t0v
        forms["validation"] = {
            "rscan": {"workload": "QU Nside 16 l=2..32 |b|<10 deg cut, r in [0, 0.01] x 31, "
                                  "1000 maps at r = 0",
                      "s": t_rs, "r_peak": rs["r_peak"], "upper68": rs["upper68"],
                      "upper95": rs["upper95"], "sigma1": rs["sigma1"]},
            "fsky_sweep": {"workload": "QU Nside 16 l=2..32, cuts 0/10/18/30/40 deg, 1000 maps",
                           "s": t_sw,
                           "fsky": [round(r["fsky"], 3) for r in sw],
                           "max_abs_ratio_minus_1": [float(np.abs(r["ratio"] - 1).max())
                                                     for r in sw],
                           "bound_5_std_errors": 5.0 / np.sqrt(2 * 1000)}}
        # lnL emulator: exact labels from the batched scan (TQU Nside 8,
        # f_sky 0.7, l <= 15), training of the two-head MLP, then inference with
        # the fallback flags over 2^20 points and an audit of accepted points
        forms["emulator"] = emulator_form(api, torch, td)
        if args.emulator_full:
            forms["emulator_tqu_nside16_50k"] = emulator_form(api, torch, td, full=True)
        # the split kernel against the measured bf16 tensor peak: W = X^T X
        # (k=6900, n=5952), 36 digit products of 2 k(k+1)/2 n flops each
        X = torch.randn(wl.k, wl.n, dtype=torch.float64, device="cuda").t()
        W = torch.empty(wl.k, wl.k, dtype=torch.float64, device="cuda").t()
        api.gemm(X, X, W, transA=True, lower=True, precision=1)
        e12, e13 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e12.record()
        for _ in range(3):
            api.gemm(X, X, W, transA=True, lower=True, precision=1)
        e13.record()
        e13.synchronize()
        dur_s = e12.elapsed_time(e13) * 1e-3 / 3
        pk = peaks()
        bf16_peak = pk.get("bf16_tflops", 1900.0)
        tensor_flops = 36 * float(wl.k) * wl.k * wl.n
        forms["roofline_split"] = {
            "kernel": "split GEMM (slicing + ozaki_gemm_kernel), W = X^T X lower, k=6900, n=5952",
            "bound": "tensor", "achieved": tensor_flops / dur_s / 1e12, "peak": bf16_peak,
            "unit": "TFLOP/s", "frac": tensor_flops / dur_s / 1e12 / bf16_peak,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst) of measured",
            "fp64_equivalent_tflops": float(wl.k) * wl.k * wl.n / dur_s / 1e12,
            "ms_per_launch": dur_s * 1e3,
            "traffic": OZ_SYRK_TRAFFIC, "traffic_source": OZ_SYRK_TRAFFIC_SOURCE}
        del X, W
        torch.cuda.empty_cache()

    # ---- end to end through the same entry points with pinned host buffers
    e2e = None
    if rank == 0 and not args.no_e2e:
        def pinned(a):
            # pinned host memory, column-major like every matrix of the C ABI
            # (a row-major array would be copied into pageable memory by the
            # binding first)
            t_ = torch.empty(a.shape[::-1], dtype=torch.float64, pin_memory=True)
            f = t_.numpy().T
            f[...] = a
            return f
        hN = pinned(wl.N())
        hp = api.Problem(wl.lmin, wl.lmax, theta_T=pinned(wl.theta_T), phi_T=pinned(wl.phi_T),
                         theta_P=pinned(wl.theta_P), phi_P=pinned(wl.phi_P),
                         transfer_T=pinned(wl.transfer_T), transfer_P=pinned(wl.transfer_P),
                         spec=wl.spec, cl_fid=pinned(wl.cl_fid.reshape(-1)), N=hN)
        assert hp._p.N == hN.ctypes.data, "N must reach the library without a copy"
        hmaps = np.asfortranarray(maps.cpu().numpy())
        hm = torch.empty((args.nsims, wl.n), dtype=torch.float64, pin_memory=True).numpy().T
        hm[...] = hmaps
        h1 = np.asfortranarray(hm[:, :1])
        hcl = pinned(wl.cl_fid.reshape(-1))

        def hstep():
            F, plan = api.fisher(hp)
            est = plan.estimate(hm)
            api.loglike(hp, hcl, h1)
            plan.free()
            return est
        hstep()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            hstep()
        te = time.perf_counter() - t0
        nb = 8
        geo = (2 * wl.npix_T + 2 * wl.npix_P + 2 * (wl.lmax + 1) + 6 * (wl.lmax + 1)) * nb
        h2d = 2 * (geo + wl.n * wl.n * nb) + wl.n * args.nsims * nb + wl.n * nb + 6 * (wl.lmax + 1) * nb
        na = len(wl.spec) * wl.nl
        d2h = na * na * nb + (4 * na * args.nsims + na) * nb + 3 * nb
        e2e = {"value": args.steps / te, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h),
               "note": "same C-ABI calls with pinned host buffers; copies inside the timed region"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "config": cfg,
                "lnl_evals_per_s": lnl_rate, "roofline": roof, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": int(c1 - c0), "clocks": clocks, "forms": forms}
        # the metric's headline figures in one short object, last on the line
        line["summary"] = summarize(value, forms)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
