"""Single-call cases for profiler captures (ncu), on the TQU Nside 16 workload.

    python profile_cases.py syrk     # W = X^T X, k=6900, n=5952
    python profile_cases.py syrk_split  # the same, split precision
    python profile_cases.py trail_split
        # split Cholesky trailing update: C (6400 x 6400, lower) -= P P^T, K = 512
    python profile_cases.py ybuild   # Y, 5952 x 6900
    python profile_cases.py fisher   # one full qml_fisher
    python profile_cases.py step --precision 1
        # one bench step: qml_fisher + qml_estimate (100 maps) + pix_loglike
    python profile_cases.py emu_predict [--points N]
        # emulator inference: a 4 x 256 emulator trained for two epochs on
        # 8192 points of a 4-D test function predicts N points (2^18)

Each case runs its call `--reps` times (default 2) after one untimed call and
prints the CUDA-event time per call.
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def main():
    import torch

    from paper_2605_21149_gb300 import api, build, synth

    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=("syrk", "syrk_split", "trail_split", "ybuild", "fisher", "step",
                                     "emu_predict"))
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--points", type=int, default=1 << 18, help="emu_predict: points per call")
    ap.add_argument("--tune", action="append", default=[],
                    help="key=value entry of the library's tuning table (repeatable)")
    args = ap.parse_args()
    build.build()
    for kv in args.tune:
        key, value = kv.split("=", 1)
        api.tune_set(key, int(value))
    wl = synth.workload(1)
    prob = api.Problem.from_workload(wl, precision=args.precision)
    if args.case in ("syrk", "syrk_split"):
        X = torch.randn(wl.k, wl.n, dtype=torch.float64, device="cuda").t()
        W = torch.empty(wl.k, wl.k, dtype=torch.float64, device="cuda").t()
        prec = 1 if args.case == "syrk_split" else 0
        fn = lambda: api.gemm(X, X, W, transA=True, lower=True, precision=prec)
    elif args.case == "trail_split":
        P = torch.randn(512, 6400, dtype=torch.float64, device="cuda").t()
        T = torch.zeros(6400, 6400, dtype=torch.float64, device="cuda").t()
        fn = lambda: api.gemm(P, P, T, transB=True, lower=True, alpha=-1.0, beta=1.0, precision=1)
    elif args.case == "emu_predict":
        import numpy as np
        rng = np.random.default_rng(1)
        th = rng.uniform(-1, 1, size=(8192, 4))
        y = (-0.5 * (th ** 2 * np.array([30.0, 10.0, 5.0, 2.0])).sum(axis=1)
             + np.sin(2 * th[:, 0]) * th[:, 1])
        emu = api.Emulator(-np.ones(4), np.ones(4), seed=7)
        emu.train(th, y, epochs=2, batch=64)
        thi = torch.as_tensor(rng.uniform(-1.05, 1.05, size=(args.points, 4)), device="cuda")
        fn = lambda: emu.predict(thi)
    elif args.case == "ybuild":
        fn = lambda: api.ybuild(prob)
    elif args.case == "fisher":
        fn = lambda: api.fisher(prob, keep_plan=False)
    else:
        g = synth.rng(1, synth.P_SIMS)
        alm = synth.draw_alm(wl.cl_fid, wl.lmin, wl.lmax, wl.comps, 100, g)
        noise = synth.noise_draws(wl.G, 100, g)
        td = lambda x: torch.as_tensor(x, device="cuda").t().contiguous().t()
        maps = api.synthesize(prob, td(alm), td(noise))
        cl = torch.as_tensor(wl.cl_fid.reshape(-1), device="cuda")

        def fn():
            F, plan = api.fisher(prob)
            plan.estimate(maps)
            api.loglike(prob, cl, maps[:, :1])
            plan.free()
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        fn()
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    print(f"{args.case}: {ms:.3f} ms per call")
    if args.case == "emu_predict":
        print(f"emu_predict: {args.points / (ms * 1e-3):.4g} points/s")


if __name__ == "__main__":
    main()
