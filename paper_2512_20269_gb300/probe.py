"""Runs one library operation once, for profilers (ncu) and quick checks.

    python -m paper_2512_20269_gb300.probe --op precond --d 3 --n 256 --p 4 --precision fp64
    python -m paper_2512_20269_gb300.probe --op stiffness --n 256 --p 4
    python -m paper_2512_20269_gb300.probe --op solve --n 64 --p 4 --autotune
    python -m paper_2512_20269_gb300.probe --op precond --n 256 --p 4 --warp

Builds the plan (optionally autotuned, or with the warp-FFT transform pass
on every eligible direction), draws the N(0,1) right-hand side of
seed 1 on the host, and runs the operation once on cuda:0 through the C ABI.
Prints the plan's launch geometry.
"""

from __future__ import annotations

import argparse
import sys


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["precond", "stiffness", "solve"], default="precond")
    ap.add_argument("--d", type=int, default=3)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--coef", choices=["const", "sin"], default="const")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--warp", action="store_true", help="warp-FFT pass on every eligible direction")
    a = ap.parse_args(argv)

    import torch

    from . import IFFDPlan, inputs
    plan = IFFDPlan(a.d, a.n, a.p, precision=a.precision, coef=a.coef, true_residual=False)
    if a.autotune:
        plan.autotune()
    if a.warp:
        from . import IFFDError
        for k in range(a.d):
            try:
                plan.set_geometry(k, warp=True)
            except IFFDError:
                pass  # not eligible: block kernel
    f = torch.from_numpy(inputs.rhs(plan.shape, "normal", 1)).cuda()
    if a.op == "precond":
        plan.apply_preconditioner(f)
    elif a.op == "stiffness":
        plan.apply_stiffness(f)
    else:
        _, info = plan.pcg_solve(f)
        print("iters", info["iters"], "rel_res", info["rel_res"])
    torch.cuda.synchronize()
    print("ok", a.op, "N", plan.N, [plan.tiles(k) for k in range(a.d)])
    return 0


if __name__ == "__main__":
    sys.exit(main())
