"""Single-call cases for profiler captures (ncu), on the TQU Nside 16 workload.

    python -m paper_2605_21149_gb300.profile_cases syrk     # W = X^T X, k=6900, n=5952
    python -m paper_2605_21149_gb300.profile_cases syrk_split  # the same, split precision
    python -m paper_2605_21149_gb300.profile_cases ybuild   # Y, 5952 x 6900
    python -m paper_2605_21149_gb300.profile_cases fisher   # one full qml_fisher

Each case runs its call `--reps` times (default 2) after one untimed call and
prints the CUDA-event time per call.
"""
from __future__ import annotations

import argparse


def main():
    import torch

    from . import api, build, synth

    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=("syrk", "syrk_split", "ybuild", "fisher"))
    ap.add_argument("--reps", type=int, default=2)
    args = ap.parse_args()
    build.build()
    wl = synth.workload(1)
    prob = api.Problem.from_workload(wl)
    if args.case in ("syrk", "syrk_split"):
        X = torch.randn(wl.k, wl.n, dtype=torch.float64, device="cuda").t()
        W = torch.empty(wl.k, wl.k, dtype=torch.float64, device="cuda").t()
        prec = 1 if args.case == "syrk_split" else 0
        fn = lambda: api.gemm(X, X, W, transA=True, lower=True, precision=prec)
    elif args.case == "ybuild":
        fn = lambda: api.ybuild(prob)
    else:
        fn = lambda: api.fisher(prob, keep_plan=False)
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        fn()
    e1.record()
    e1.synchronize()
    print(f"{args.case}: {e0.elapsed_time(e1) / args.reps:.3f} ms per call")


if __name__ == "__main__":
    main()
