"""Runs one library operation once, for profilers (ncu) and quick checks.

    python -m paper_2512_20269_gb300.probe --op precond --d 3 --n 256 --p 4 --precision fp64
    python -m paper_2512_20269_gb300.probe --op stiffness --n 256 --p 4
    python -m paper_2512_20269_gb300.probe --op solve --n 64 --p 4 --autotune
    python -m paper_2512_20269_gb300.probe --op precond --n 256 --p 4 --warp
    python -m paper_2512_20269_gb300.probe --op general --n 64 --p 4

Builds the plan (optionally autotuned, or with the warp-FFT transform pass
on every eligible direction), draws the N(0,1) right-hand side of
seed 1 on the host, and runs the operation once on cuda:0 through the C ABI.
`general` applies the general-coefficient stiffness with the scalar
a = 1 + sin(2 pi (x + 2y + 3z)) cos(pi x y) / 2 at the Gauss points (z = 0 in
2D). Prints the plan's launch geometry.
"""

from __future__ import annotations

import argparse
import sys


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["precond", "stiffness", "solve", "general"], default="precond")
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
    elif a.op == "general":
        import math
        xs = [torch.from_numpy(plan.quad_points(k)[0]).cuda() for k in range(a.d)]
        g = torch.meshgrid(*reversed(xs), indexing="ij")[::-1]
        X, Y = g[0], g[1]
        Z = g[2] if a.d == 3 else torch.zeros_like(X)
        coef = (1.0 + 0.5 * torch.sin(2 * math.pi * (X + 2 * Y + 3 * Z)) * torch.cos(math.pi * X * Y))[None]
        plan.apply_stiffness_general(coef.contiguous(), f)
    else:
        _, info = plan.pcg_solve(f)
        print("iters", info["iters"], "rel_res", info["rel_res"])
    torch.cuda.synchronize()
    print("ok", a.op, "N", plan.N, [plan.tiles(k) for k in range(a.d)])
    return 0


if __name__ == "__main__":
    sys.exit(main())
