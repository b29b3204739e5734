#!/usr/bin/env python3
"""Benchmark of the IFFD-preconditioned PCG solve on one GB300 per rank.

One step = one full PCG solve (zero start, relative residual 1e-8) of the 3D
Dirichlet Poisson problem with n = 256 elements per direction and degree p = 4
(258^3 = 17,173,512 DoFs, right-hand side N(0,1) from seed 1), FP64 IFFD
preconditioner, through the C ABI: every step of the path (preconditioner
passes, stiffness sweeps, PCG updates, reductions) runs in the library's
kernels. Printed metric: DoFs solved per second (whole job).

Also measured in the same run (outside the timed K steps): the same solve with
the exact Fast Diagonalization preconditioner (the comparator) and with the
FP32-transform IFFD preconditioner; per-kernel device time from CUDA events
recorded by the library on the launching stream during the timed region; SM
clocks sampled by nvidia-smi during the timed region; an end-to-end number
with host buffers; the GPU's FP64 and FP32 FMA rates (measured by the
library's calibration kernel, the roofline denominators of the arithmetic-
bound kernels); and the CPU oracle's own full PCG solve of the same problem.

Multi-GPU: problems are independent, so N ranks solve N independent copies
(replicas, weak scaling, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --probe precond|stiffness|solve|general [--n 256 --p 4 ...]   (one operation, for ncu)
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PCG-solved DoF/s at rel. res 1e-8, IGA-FFD vs exact FD on 1 GB300; % HBM peak"
UNIT = "DoF/s"
_CSRC = "paper_2512_20269_gb300/csrc/"
# source files whose kernels a traffic record (profiles/ncu_traffic.txt) covers
SRC_FILES = {"precond": [_CSRC + f for f in ("precond.cu", "precond_block.cuh", "device_common.cuh")],
             "precond_df": [_CSRC + f for f in ("precond_warp.cuh", "precond_dev.cuh", "dfloat.cuh", "device_common.cuh")],
             "stiff": [_CSRC + f for f in ("stiffness.cu", "stiff_dev.cuh", "device_common.cuh")],
             "pcg": [_CSRC + f for f in ("pcg.cu", "pcg_dev.cuh", "device_common.cuh")]}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


def algorithmic(kind: str, d: int, n: int, p: int, n_out: int, N: int, precision: str):
    """Algorithmic work of one launch of a kernel kind: (amount, unit, bound).

    Per-DoF figures: transform pass 2.5 log2(n) + 2 n_out flops (FFT-type DST +
    remainder projections); the fused pass does two of them plus the eigenvalue
    sum and division (3 flops). Stiffness in the symmetric-Toeplitz form of the
    interior rows (pair sums u_{i-k} + u_{i+k} shared by M and K): first sweep
    M u and K u from one set of pair sums, 5p + 2 flops, plus 2 for the fused
    direction update p = z + beta p; middle sweep M T1, K T1 (shared pairs) and
    M T2 plus the sum, 8p + 4; last sweep K T1 + M T2, 6p + 3, plus 2 for the
    fused dot product. The backward pass along x also forms the PCG dot product
    (r, z) of its output (2 flops per DoF), so the backward kind, averaged over
    its d - 1 directions, adds 2 / (d - 1). PCG update 48 B/DoF."""
    per_pass = 2.5 * math.log2(n) + 2 * n_out
    if kind.startswith("precond"):
        if precision == "df":
            # double-float passes (FP64 accuracy on the FP32 pipe): each pass
            # reads and writes 8 B per DoF (FP64 or a float pair); the last
            # backward pass also reads r for the fused dot product (averaged
            # over the d - 1 backward directions). They are bound by FP32
            # instruction issue (ncu), far from HBM; reported against HBM.
            byt = {"precond_fwd": 16.0, "precond_fused": 16.0, "precond_bwd": 16.0 + 8.0 / (d - 1)}[kind]
            return byt * N, "B", "hbm"
        if precision == "fp32":
            # FP32 intermediates: the first FWD pass reads FP64 and writes FP32
            # (12 B/DoF), the last BWD pass the reverse (12), the others read
            # and write FP32 (8); per launch kind averaged over its directions
            edge = (12.0 + 8.0 * (d - 2)) / (d - 1)
            byt = {"precond_fwd": edge, "precond_fused": 8.0, "precond_bwd": edge}[kind]
            return byt * N, "B", "hbm"
        if kind == "precond_fused":
            fl = (2 * per_pass + 3) * N
        elif kind == "precond_bwd":
            fl = (per_pass + 2.0 / (d - 1)) * N
        else:
            fl = per_pass * N
        return fl, "flop", "alu"
    if kind.startswith("stiff"):
        per = {"stiff_first": 5 * p + 4, "stiff_mid": 8 * p + 4, "stiff_last": 6 * p + 5}[kind]
        return per * N, "flop", "alu"
    if kind == "pcg_update":
        return 48.0 * N, "B", "hbm"
    if kind == "fd_pass":
        return 2 * 2 * n * N, "flop", "alu"
    return None, None, None


def file_sha(rel) -> str:
    """sha256[:16] of one file, or of the concatenation of a list of files."""
    h = hashlib.sha256()
    try:
        for r in ([rel] if isinstance(rel, str) else rel):
            with open(os.path.join(ROOT, r), "rb") as fh:
                h.update(fh.read())
    except Exception:
        return ""
    return h.hexdigest()[:16]


def ncu_traffic(kind: str):
    """DRAM bytes per launch of `kind` (for transform passes `kind/arith`, the
    pass arithmetic) from the committed ncu summary, only if the kernel sources
    still have the hash recorded with the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and not line.startswith("#") and parts[0] == kind:
            src, sha, val = parts[1], parts[2], float(parts[3])
            if file_sha(SRC_FILES.get(src, src)) == sha:
                return val
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = os.path.join("/tmp", f"iffd_clocks_{os.getpid()}.csv")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(gpu_index), "-lms", "50"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.remove(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def cpu_oracle_solve(w):
    """The oracle (CPU, float64, numpy/scipy) solving the same problem the GPU
    solves: its own textbook PCG with its own IFFD preconditioner, zero start,
    to the same relative residual 1e-8. The 1D setup (splitting and eigendata,
    also excluded on the GPU) and the right-hand side are prepared before the
    clock starts; the timed region is the whole PCG solve."""
    import scipy.sparse

    from oracle import operators, splitting
    from paper_2512_20269_gb300 import inputs

    s = splitting.axis_split(w.n, w.p, (0, 1))
    splits = [s] * w.d
    MK = [(scipy.sparse.csr_matrix(s.M), scipy.sparse.csr_matrix(s.K))] * w.d
    f = inputs.workload_rhs(w)
    t0 = time.perf_counter()
    u, iters, hist = operators.pcg(f, lambda v: operators.stiffness_apply(v, MK),
                                   lambda v: operators.iffd_apply(v, splits), rtol=1e-8)
    sec = time.perf_counter() - t0
    return {"value": w.N / sec, "unit": UNIT, "cores": _cores(), "kind": "oracle",
            "sample": (f"full solve: the oracle's PCG (numpy/scipy FP64, IFFD preconditioner by dense Q~ per "
                       f"direction) on the whole {w.name} problem ({w.N} DoFs), zero start to relative residual "
                       f"1e-8, {iters} iterations, {sec:.2f} s; 1D setup excluded as on the GPU; BLAS threads = "
                       f"all cores"),
            "iters": int(iters), "rel_res": float(hist[-1]), "seconds": sec}


def cpu_subcase_errors(sub, u_gpu: dict):
    """Error of the GPU solves of the 64^3 subcase (n = 64, p = 4, 66^3 DoFs,
    N(0,1) seed 1) against the oracle's exact solution A^{-1} f (its exact Fast
    Diagonalization with dense generalized eigenvectors, which is A^{-1} on the
    cube), and the oracle's own PCG iteration count there. u_gpu: {variant:
    (u as numpy, iterations)}."""
    import scipy.sparse

    from oracle import operators, splitting
    from paper_2512_20269_gb300 import inputs

    s = splitting.axis_split(sub.n, sub.p, (0, 1))
    f = inputs.workload_rhs(sub)
    Q, lam = operators.exact_fd_eig(s.M, s.K)
    u_ex = operators.exact_fd_apply(f, [(Q, lam)] * sub.d)
    MK = [(scipy.sparse.csr_matrix(s.M), scipy.sparse.csr_matrix(s.K))] * sub.d
    _, it_or, _ = operators.pcg(f, lambda v: operators.stiffness_apply(v, MK),
                                lambda v: operators.iffd_apply(v, [s] * sub.d), rtol=1e-8)
    nrm = float(np.linalg.norm(u_ex))
    out = {"workload": sub.name, "N": sub.N, "oracle_pcg_iters": int(it_or),
           "reference": "oracle exact-FD solve A^-1 f (dense generalized eigenvectors)"}
    for name, (u, it) in u_gpu.items():
        out[name] = {"iters": int(it), "rel_err_vs_oracle": float(np.linalg.norm(u - u_ex) / nrm),
                     "max_rel_err_vs_oracle": float(np.abs(u - u_ex).max() / np.abs(u_ex).max())}
    return out


def run_reference(args, rank: int, world: int):
    """Reference arm: the oracle as it stands, on the host cores. Each step is
    one full oracle PCG solve of the 258^3 problem (cpu_oracle_solve)."""
    from paper_2512_20269_gb300 import inputs
    if rank != 0:
        return 0
    w = inputs.CUBE_N256_P4
    for _ in range(args.warmup):
        cpu_oracle_solve(w)
    secs = []
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = cpu_oracle_solve(w)
        secs.append(last["seconds"])
    wall = time.perf_counter() - t0
    total = sum(secs)
    value = w.N * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w),
            "cpu_baseline": dict(last, value=value),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    line["cpu_baseline"].pop("seconds", None)
    print(json.dumps(line), flush=True)
    return 0


def reduce_max_ms(ms: float, dist, device: str) -> float:
    """Max of the per-rank timed-region durations (the slowest replica bounds
    the job). `dist` is torch.distributed (or None for one rank)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(dofs_per_solve: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job DoF/s of `world` independent replicas that each solved
    `steps` problems of `dofs_per_solve` DoFs within `max_ms` milliseconds."""
    return dofs_per_solve * steps * world / (max_ms / 1e3)


def workload_config(w):
    return {"workload": w.name, "d": w.d, "n": w.n, "p": w.p, "N": w.N, "rhs": f"{w.dist} seed {w.seed}",
            "precond": "IFFD", "precision": "fp64", "rtol": 1e-8, "boundary": "Dirichlet on all faces",
            "l2": "no flush: 137 MB vectors, ~1 GB working set > 126 MB L2",
            "timing": "timed solves as the library runs repeated solves (iteration chunks replayed from "
                      "captured CUDA graphs); per-kernel times from the same solves replayed right after with "
                      "a CUDA event pair around every launch"}


def _timed(fn, reps: int, warm: int):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    out = None
    for _ in range(reps):
        out = fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps, out


def run_other_workload(args, rank: int, world: int, local: int) -> int:
    """Secondary workloads (one JSON line each, same metric); not the headline."""
    import torch

    from paper_2512_20269_gb300 import IFFDEngine, IFFDPlan, _lib, inputs
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2512_20269_gb300 import build
        build.build()
    torch.cuda.set_device(local)
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": world, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic", "steps": args.steps, "warmup": args.warmup}
    if args.workload in ("square", "varcoef"):
        w = inputs.SQUARE_N64_P3 if args.workload == "square" else inputs.CUBE_N384_P8
        coef = "const" if args.workload == "square" else "sin"
        f = torch.from_numpy(inputs.workload_rhs(w)).cuda()
        res = {}
        for prec, pc in (("fp64", "iffd"), ("fp32", "iffd"), ("exact_fd", "exact_fd")):
            pr = "fp64" if prec == "exact_fd" else prec
            plan = IFFDPlan(w.d, w.n, w.p, precision=pr, precond=pc, coef=coef, true_residual=False).autotune()
            u = plan.empty()
            reps = args.steps if pc == "iffd" else min(args.steps, 2)
            ms, (_, info) = _timed(lambda: plan.pcg_solve(f, u), reps, 1 if pc != "iffd" else max(args.warmup, 1))
            chk = IFFDPlan(w.d, w.n, w.p, precision=pr, precond=pc, coef=coef, true_residual=True).autotune()
            _, ic = chk.pcg_solve(f)
            res[prec] = {"value": w.N / (ms / 1e3), "ms_per_solve": ms, "iters": info["iters"],
                         "true_rel_res": ic["true_rel_res"]}
            del plan, chk
            torch.cuda.empty_cache()
        line.update({"value": res["fp64"]["value"], "ms_per_step": res["fp64"]["ms_per_solve"], "dtype": "f64",
                     "config": {"workload": w.name, "d": w.d, "n": w.n, "p": w.p, "N": w.N,
                                "coefficient": "1 + 0.5 prod sin(2 pi x_k)" if coef == "sin" else "1",
                                "rhs": f"{w.dist} seed {w.seed}"},
                     "variants": {"fp32_transform": res["fp32"], "exact_fd": res["exact_fd"]},
                     "fp64": res["fp64"]})
    elif args.workload == "batched":
        probs = inputs.batched_problems()
        systems = []
        for k, (d, n, p, nrhs) in enumerate(probs):
            for j in range(nrhs):
                N = (n + p - 2) ** d
                systems.append((d, n, p, inputs.device_rhs(N, 3_000_003 * (k + 1) + j)))
        total = sum(f.numel() for *_, f in systems)
        budget = 64 << 30
        outs = [torch.empty_like(f) for *_, f in systems]

        eng = IFFDEngine(budget, precision="fp32", autotune=not args.no_autotune, persistent=args.persistent)

        def solve_all():
            k0 = eng.stats()["kernel_launches"]
            for (d, n, p, f), u in zip(systems, outs):
                assert eng.submit(d, n, p, f, u) is not None
            done = eng.run_to_completion(iterations_per_step=4)
            return done, eng.stats()["kernel_launches"] - k0

        for _ in range(max(args.warmup, 1)):
            solve_all()  # the first call also builds and caches every (n, p) plan
        torch.cuda.synchronize()
        reps = max(1, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(reps):
            done, kl = solve_all()
        torch.cuda.synchronize()
        sec = (time.perf_counter() - t0) / reps
        eng.close()
        iters = [info["iters"] for _, info in done]
        line.update({"value": total / sec, "ms_per_step": sec * 1e3, "dtype": "f64",
                     "config": {"workload": "batched_512_cubes", "problems": len(probs), "systems": len(systems),
                                "dofs": int(total), "n": list(inputs.BATCH_N), "p": list(inputs.BATCH_P),
                                "precond": "IFFD, FP32 transforms", "pcg": "fp64", "seed": 3,
                                "autotune": not args.no_autotune, "persistent": args.persistent},
                     "iters_min_max_mean": [min(iters), max(iters), float(np.mean(iters))],
                     "gpu_launches": kl,
                     "launch_mode": ("one persistent launch per engine step over a device work queue (block "
                                     "transform kernels)" if args.persistent else
                                     "captured graph of batched launches per iteration"),
                     "timing": "wall clock around submit + engine steps to completion; plans cached, arena "
                               "allocated once (setup excluded)"})
    else:
        from paper_2512_20269_gb300.serving import Server
        # the configured 2000 req/s, or a lower rate (--serve-rate) at which one
        # GPU keeps up, to show latency in normal operation
        reqs = inputs.serving_requests(rate=args.serve_rate, duration=60.0 if args.serve_rate >= 2000 else
                                       max(args.serve_seconds, 1.0))
        cap = args.serve_cap_dofs if args.serve_cap_dofs > 0 else None
        srv = Server(budget_bytes=150 * (1 << 30), precision="fp32", iterations_per_step=args.serve_iters,
                     max_inflight_dofs=cap)
        # at a sustainable rate the run also drains the requests still in flight
        st = srv.run(reqs, max_wall_s=args.serve_seconds if args.serve_rate >= 2000 else args.serve_seconds + 30.0)
        line.update({"value": st["dof_per_s"], "ms_per_step": None, "dtype": "f64",
                     "config": {"workload": f"serving_poisson_{args.serve_rate:g}rps", "rate_rps": args.serve_rate,
                                "arrival_window_s": 60 if args.serve_rate >= 2000 else max(args.serve_seconds, 1.0),
                                "run_wall_s": args.serve_seconds, "budget_bytes": 150 * (1 << 30),
                                "precond": "IFFD, FP32 transforms", "seed": 4, "max_inflight_dofs": cap,
                                "iterations_per_step": args.serve_iters},
                     "serving": st})
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_probe(args) -> int:
    """One library operation on cuda:0 through the C ABI, for profilers (ncu):
    the plan of (d, n, p) (optionally autotuned, or with the warp-FFT pass on
    every eligible direction), the N(0,1) right-hand side of seed 1, and one
    preconditioner apply, stiffness apply, PCG solve, or general-coefficient
    stiffness apply (scalar a = 1 + sin(2 pi (x + 2y + 3z)) cos(pi x y) / 2 at
    the Gauss points). Prints the launch geometry; not a benchmark."""
    import torch

    from paper_2512_20269_gb300 import IFFDError, IFFDPlan, _lib, inputs
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2512_20269_gb300 import build
        build.build()
    plan = IFFDPlan(args.d, args.n, args.p, precision=args.precision, coef=args.coef, true_residual=False)
    if args.autotune:
        plan.autotune()
    if args.warp:
        for k in range(args.d):
            try:
                plan.set_geometry(k, warp=True)
            except IFFDError:
                pass  # not eligible: block kernel
    f = torch.from_numpy(inputs.rhs(plan.shape, "normal", 1)).cuda()
    torch.cuda.synchronize()
    # profiler range: `ncu --profile-from-start off` captures only the operation
    torch.cuda.profiler.start()
    for _ in range(max(1, args.probe_reps)):
        if args.probe == "precond":
            plan.apply_preconditioner(f)
        elif args.probe == "stiffness":
            plan.apply_stiffness(f)
        elif args.probe == "general":
            xs = [torch.from_numpy(plan.quad_points(k)[0]).cuda() for k in range(args.d)]
            g = torch.meshgrid(*reversed(xs), indexing="ij")[::-1]
            X, Y = g[0], g[1]
            Z = g[2] if args.d == 3 else torch.zeros_like(X)
            coef = (1.0 + 0.5 * torch.sin(2 * math.pi * (X + 2 * Y + 3 * Z)) * torch.cos(math.pi * X * Y))[None]
            plan.apply_stiffness_general(coef.contiguous(), f)
        else:
            _, info = plan.pcg_solve(f)
            print("iters", info["iters"], "rel_res", info["rel_res"])
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print("ok", args.probe, "N", plan.N, [plan.tiles(k) for k in range(args.d)])
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--workload", default="cube", choices=["cube", "square", "varcoef", "batched", "serving"],
                    help="cube (default, the headline line): 258^3 p=4; square: 65^2 p=3; varcoef: 390^3 p=8 "
                         "variable coefficient; batched: 512 uneven 3D problems; serving: Poisson request stream")
    ap.add_argument("--serve-seconds", type=float, default=30.0)
    ap.add_argument("--no-autotune", action="store_true", help="batched: default launch geometry")
    ap.add_argument("--persistent", action="store_true",
                    help="batched: each engine step as one persistent launch over a device work queue")
    ap.add_argument("--serve-iters", type=int, default=2, help="serving: PCG iterations per engine step")
    ap.add_argument("--serve-rate", type=float, default=2000.0,
                    help="serving: arrival rate (req/s); below 2000 the arrival window equals --serve-seconds")
    ap.add_argument("--serve-cap-dofs", type=int, default=0,
                    help="serving: cap on the DoFs in flight (0 = HBM budget only)")
    ap.add_argument("--probe", choices=["precond", "stiffness", "solve", "general"], default=None,
                    help="run one library operation once (for ncu) instead of the benchmark")
    ap.add_argument("--d", type=int, default=3, help="--probe: dimension")
    ap.add_argument("--n", type=int, default=256, help="--probe: elements per direction")
    ap.add_argument("--p", type=int, default=4, help="--probe: degree")
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp64", help="--probe: transform precision")
    ap.add_argument("--coef", choices=["const", "sin"], default="const", help="--probe: coefficient")
    ap.add_argument("--autotune", action="store_true", help="--probe: autotune the plan first")
    ap.add_argument("--warp", action="store_true", help="--probe: warp-FFT pass on every eligible direction")
    ap.add_argument("--probe-reps", type=int, default=1, help="--probe: repetitions of the operation")
    args = ap.parse_args()
    if args.probe:
        return run_probe(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload != "cube":
        return run_other_workload(args, rank, world, local)

    import numpy as np
    import torch

    from paper_2512_20269_gb300 import IFFDPlan, _lib, inputs

    if not os.path.exists(_lib.LIB_PATH):
        from paper_2512_20269_gb300 import build
        build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    w = inputs.CUBE_N256_P4
    # roofline denominators of the arithmetic-bound kernels, measured on this
    # GPU by the library's FMA-chain calibration kernel (not timed)
    from paper_2512_20269_gb300 import measure_peak
    pk64 = measure_peak("fp64")
    pk32 = measure_peak("fp32")
    pk32x2 = measure_peak("fp32x2")
    fp64_peak = pk64["tflops"]
    peak_src = (f"measured: iffd_measure_peak FP64 FMA chains on {pk64['sm_count']} SMs (cudaDeviceGetAttribute), "
                f"best of 3 CUDA-event-timed launches")
    # setup (excluded from timing): plan, then the launch-geometry autotuner
    plan = IFFDPlan(w.d, w.n, w.p, precision="fp64", precond="iffd", true_residual=False).autotune()
    f_host = torch.from_numpy(inputs.workload_rhs(w))
    f = f_host.cuda()
    u = plan.empty()
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        _, info = plan.pcg_solve(f, u)
    iters = info["iters"]

    # ---------------- timed region: K solves, inputs resident in HBM
    launches0 = plan.launch_count()
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        _, info = plan.pcg_solve(f, u)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    gpu_launches = plan.launch_count() - launches0
    # per-kernel device times: the same solves again, right after, with a CUDA
    # event pair around every launch on the launching stream (the library's
    # profiler; its launches are direct, not from the captured graphs)
    plan.profile_reset()
    plan.profile_enable(True)
    for _ in range(args.steps):
        plan.pcg_solve(f, u)
    torch.cuda.synchronize()
    plan.profile_enable(False)
    prof = plan.profile_read()
    ms = reduce_max_ms(ms, dist, "cuda")
    value = replica_throughput(w.N, args.steps, world, ms)

    # ---------------- per-kernel roofline (dominant kernel by device time)
    n_out = w.p - 2 if w.p % 2 == 0 else w.p - 1
    total_k = sum(v[1] for v in prof.values()) or 1.0
    rooflines = {}
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    # Launches that did work: iterations are enqueued in chunks (the first as
    # long as the plan's previous solve, then 4); launches enqueued past
    # convergence return at their first instruction, so per-launch rates use
    # the launches of the executed iterations only.
    # preconditioner applies that did work: the initial one and one per
    # iteration except the last (its residual met the tolerance, so its apply
    # exits at once)
    applies = args.steps * iters
    eff = {"precond_fwd": applies * (w.d - 1), "precond_fused": applies, "precond_bwd": applies * (w.d - 1),
           "stiff_first": args.steps * iters, "stiff_mid": args.steps * iters, "stiff_last": args.steps * iters,
           "pcg_update": args.steps * iters}
    arith = "df" if all(plan.tiles(a).get("double_float") for a in range(w.d)) else "fp64"
    for kind, (cnt, kms) in prof.items():
        if cnt == 0:
            continue
        amount, unit, bound = algorithmic(kind, w.d, w.n, w.p, n_out, w.N, arith)
        entry = {"launches": cnt, "ms": kms, "share": kms / total_k}
        if amount is not None:
            n_eff = min(cnt, eff.get(kind, cnt))
            entry["launches_with_work"] = n_eff
            avg_s = kms / n_eff / 1e3
            if unit == "flop":
                ach = amount / avg_s / 1e12
                entry.update({"bound": bound, "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                              "frac": ach / fp64_peak, "alg_per_launch": amount})
            else:
                ach = amount / avg_s / 1e9
                entry.update({"bound": bound, "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                              "frac": ach / hbm_peak, "alg_per_launch": amount})
        tk = ncu_traffic(f"{kind}/{arith}" if kind.startswith("precond") else kind)
        if tk is not None:
            entry["traffic"] = tk
        rooflines[kind] = entry
    dom = max((k for k in rooflines if "bound" in rooflines[k]), key=lambda k: rooflines[k]["ms"])
    d = rooflines[dom]
    roofline = {"bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"], "unit": d["unit"],
                "frac": d["frac"], "traffic": d.get("traffic"), "kernel": dom,
                "peak_source": (peak_src if d["bound"] == "alu" else "MEASURED_PEAKS.json hbm_gbs (measured copy)")}

    # ---------------- end to end: pinned host f -> device, solve, u -> host.
    # Every step copies its f in and its u out; the copies run on two more
    # streams (one per direction, so that the two copy engines work at once),
    # double-buffered, so that step k+1's input and step k-1's output move
    # while step k solves: the timed region is the first input copy, the K
    # solves and the last output copy.
    f_pin = f_host.pin_memory()
    u_pin = [torch.empty_like(f_pin).pin_memory() for _ in range(2)]
    f_dev = [torch.empty_like(f) for _ in range(2)]
    u_dev2 = [plan.empty() for _ in range(2)]
    copy_in, copy_out = torch.cuda.Stream(), torch.cuda.Stream()
    h2d = [torch.cuda.Event() for _ in range(2)]
    d2h = [torch.cuda.Event() for _ in range(2)]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for k in range(max(args.warmup, 4)):  # untimed: both buffer pairs seen (the solve graphs captured)
        b = k & 1
        f_dev[b].copy_(f_pin)
        plan.pcg_solve(f_dev[b], u_dev2[b], stream=stream)
        u_pin[b].copy_(u_dev2[b])
    torch.cuda.synchronize()
    e0.record(stream)
    copy_in.wait_event(e0)
    with torch.cuda.stream(copy_in):
        f_dev[0].copy_(f_pin, non_blocking=True)
        h2d[0].record(copy_in)
    for k in range(args.steps):
        b = k & 1
        if k + 1 < args.steps:  # the next step's input (its buffer's last solve has returned)
            with torch.cuda.stream(copy_in):
                f_dev[b ^ 1].copy_(f_pin, non_blocking=True)
                h2d[b ^ 1].record(copy_in)
        stream.wait_event(h2d[b])
        if k >= 2:
            stream.wait_event(d2h[b])  # u_dev2[b] copied out (step k-2)
        plan.pcg_solve(f_dev[b], u_dev2[b], stream=stream)  # returns when the solve is done
        solved = torch.cuda.Event()
        solved.record(stream)
        copy_out.wait_event(solved)
        with torch.cuda.stream(copy_out):
            u_pin[b].copy_(u_dev2[b], non_blocking=True)
            d2h[b].record(copy_out)
    e1.record(copy_out)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1)
    u_dev = u_dev2[(args.steps - 1) & 1]
    assert torch.equal(u_pin[(args.steps - 1) & 1], u_dev.cpu())
    e2e = {"value": w.N * args.steps * world / (ms_e2e / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(f_pin.numel() * 8), "d2h_bytes_per_step": int(u_pin[0].numel() * 8),
           "copies": "pinned host, one stream per direction, overlapping the neighbouring steps' solves"}

    # ---------------- accuracy of the timed solve's iterate (true residual)
    plan_chk = IFFDPlan(w.d, w.n, w.p, precision="fp64", precond="iffd", true_residual=True).autotune()
    _, info_chk = plan_chk.pcg_solve(f, u_dev)
    del plan_chk

    variants = {}
    if not args.no_variants:
        for name, prec, pc, reps in (("fp32_transform", "fp32", "iffd", args.steps), ("exact_fd", "fp64", "exact_fd", 2),
                                     ("fp64_pipe_transforms", "fp64", "iffd", args.steps)):
            pv = IFFDPlan(w.d, w.n, w.p, precision=prec, precond=pc, true_residual=False)
            if name == "fp64_pipe_transforms":  # FP64 arithmetic on the FP64 pipe instead of double-float
                for a in range(w.d):
                    pv.set_geometry(a, pipelined=False)
            pv.autotune()
            pv.pcg_solve(f, u_dev)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                _, iv = pv.pcg_solve(f, u_dev)
            b.record(stream)
            torch.cuda.synchronize()
            vms = a.elapsed_time(b) / reps
            pchk = IFFDPlan(w.d, w.n, w.p, precision=prec, precond=pc, true_residual=True)
            if name == "fp64_pipe_transforms":
                for a in range(w.d):
                    pchk.set_geometry(a, pipelined=False)
            pchk.autotune()
            _, ichk = pchk.pcg_solve(f, u_dev)
            variants[name] = {"value": w.N / (vms / 1e3), "unit": UNIT, "ms_per_solve": vms, "iters": iv["iters"],
                              "true_rel_res": ichk["true_rel_res"]}
            del pv, pchk

    # ---------------- general coefficient (-div(a grad u), a non-separable) on a
    # 130^3 grid, p = 4: the operator at the tensor Gauss points and PCG with the
    # IFFD preconditioner of the constant-coefficient operator. The application
    # is bound by the FP64 pipe: its sum-factorised sweeps cost, per output
    # value, 2 flops per matrix entry (an FMA), i.e. (3D, p1 = p + 1 entries per
    # Gauss point row, q / m = n p1 / m entries per basis-function row)
    #   x: 2 x q0 m1 m2 outputs x p1;  y: 3 x q0 q1 m2 x p1;
    #   z (fused): per Gauss point 3 p1 (gradient) + 3 p1 (transpose) FMAs and
    #     5 multiplies for w a g (w, w a, 3 products; 2D: 2 p1 + 2 p1 and 4);
    #   y^T: 3 x q0 m1 m2 x q1 p1 / m1;  x^T: 2 x m0 m1 m2 x q0 p1 / m0.
    # Algorithmic bytes: u and Au (16 per DoF) and a at every Gauss point (8).
    if not args.no_variants:
        pg = IFFDPlan(w.d, 128, w.p, precision="fp64", true_residual=True)
        xs = [torch.from_numpy(pg.quad_points(k)[0]).cuda() for k in range(w.d)]
        if w.d == 3:
            Zg, Yg, Xg = torch.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
        else:
            Yg, Xg = torch.meshgrid(xs[1], xs[0], indexing="ij")
            Zg = torch.zeros_like(Xg)
        coef = (1.0 + 0.5 * torch.sin(2 * math.pi * (Xg + 2 * Yg + 3 * Zg)) * torch.cos(math.pi * Xg * Yg))
        coef = coef[None].contiguous()
        del Xg, Yg, Zg
        fg = torch.from_numpy(inputs.rhs(pg.shape, "uniform", seed=3)).cuda()
        ug = pg.empty()
        for _ in range(2):
            pg.apply_stiffness_general(coef, fg, ug)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(5):
            pg.apply_stiffness_general(coef, fg, ug)
        b.record(stream)
        torch.cuda.synchronize()
        gms = a.elapsed_time(b) / 5
        pg.pcg_solve_general(coef, fg, ug)
        torch.cuda.synchronize()
        a.record(stream)
        _, ig = pg.pcg_solve_general(coef, fg, ug)
        b.record(stream)
        torch.cuda.synchronize()
        sms = a.elapsed_time(b)
        gbytes = 16.0 * pg.N + 8.0 * coef.numel()
        p1 = w.p + 1
        qd = [pg.quad_points(k)[0].size for k in range(w.d)]
        md = list(pg.m)
        if w.d == 3:
            q0, q1, q2 = qd
            m0, m1, m2 = md
            gflop = (2 * (2 * q0 * m1 * m2 * p1 + 3 * q0 * q1 * m2 * p1 + 3 * q0 * m1 * m2 * q1 * p1 / m1
                          + 2 * m0 * m1 * m2 * q0 * p1 / m0) + q0 * q1 * q2 * (12 * p1 + 5)) / 1e9
        else:
            q0, q1 = qd
            m0, m1 = md
            gflop = (2 * (2 * q0 * m1 * p1 + 2 * m0 * m1 * q0 * p1 / m0) + q0 * q1 * (8 * p1 + 4)) / 1e9
        variants["general_coef"] = {
            "config": {"workload": f"cube n=128 p={w.p}, a = 1 + sin(2 pi (x + 2y + 3z)) cos(pi x y) / 2",
                       "dofs": pg.N, "gauss_points": int(coef.numel())},
            "apply_ms": gms, "apply_alg_bytes": gbytes, "apply_hbm_frac": gbytes / (gms / 1e3) / 1e9 / hbm_peak,
            "apply_gflop": gflop, "apply_fp64_tflops": gflop / gms, "apply_fp64_frac": gflop / gms / fp64_peak,
            "ms_per_solve": sms, "value": pg.N / (sms / 1e3), "unit": UNIT, "iters": ig["iters"],
            "true_rel_res": ig["true_rel_res"]}
        del pg, coef, fg, ug, xs
        torch.cuda.empty_cache()

    # ---------------- preconditioner applies per second (inputs resident)
    # algorithmic bytes per DoF of one apply: FP64, 16 per pass and 24 for the
    # fused pass (it also reads 1/sum(lambda)); FP32 transforms, 12 for the
    # first and last pass and 8 for the others
    apply_stats = {}
    if not args.no_variants:
        for name, prec in (("fp64", "fp64"), ("fp32_transform", "fp32"), ("fp32_unpaired", "fp32"),
                           ("fp64_pipe", "fp64")):
            pa = IFFDPlan(w.d, w.n, w.p, precision=prec, true_residual=False)
            if name == "fp64_pipe":
                for a in range(w.d):
                    pa.set_geometry(a, pipelined=False)
            pa.autotune()
            if name == "fp32_unpaired":  # the warp-FFT pass with one sequence per lane group
                for a in range(w.d):
                    if pa.tiles(a)["warp"]:
                        pa.set_geometry(a, warp=True)
            zz = pa.empty()
            for _ in range(3):
                pa.apply_preconditioner(f, zz)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            reps = 20
            a.record(stream)
            for _ in range(reps):
                pa.apply_preconditioner(f, zz)
            b.record(stream)
            torch.cuda.synchronize()
            ams = a.elapsed_time(b) / reps
            df_mode = prec == "fp64" and all(pa.tiles(a).get("double_float") for a in range(w.d))
            if prec == "fp32":
                bpd = 24.0 + 8.0 * (2 * w.d - 3)
            else:  # FP64: 16 B per pass; the FP64-pipe fused pass also reads 1/sum(lambda)
                bpd = 16.0 * (2 * w.d - 1) + (0.0 if df_mode else 8.0)
            gbs = bpd * w.N / (ams / 1e3) / 1e9
            apply_stats[name] = {"ms": ams, "applies_per_s": 1e3 / ams, "alg_bytes_per_dof": bpd,
                                 "arithmetic": "double-float" if (prec == "fp64" and df_mode) else prec,
                                 "achieved_gbs": gbs, "hbm_frac": gbs / hbm_peak,
                                 "tiles": [pa.tiles(k) for k in range(w.d)]}
            del pa, zz

    # ---------------- the 64^3 subcase (n = 64, p = 4): FP64 and FP32-transform
    # solves on the GPU, compared with the oracle's exact solution below
    sub = inputs.CUBE_N64_P4
    sub_u = {}
    fs = torch.from_numpy(inputs.workload_rhs(sub)).cuda()
    for name, prec in (("fp64", "fp64"), ("fp32_transform", "fp32")):
        ps = IFFDPlan(sub.d, sub.n, sub.p, precision=prec, true_residual=False)
        us, isub = ps.pcg_solve(fs)
        sub_u[name] = (us.cpu().numpy(), isub["iters"])
        del ps
    del fs

    cpu = None
    subcase = None
    if rank == 0 and not args.no_cpu_baseline:
        # cpu_baseline leg: the oracle's own full solve of the headline problem,
        # and the oracle's exact solution of the subcase
        try:
            cpu = cpu_oracle_solve(w)
            cpu.pop("seconds", None)
        except Exception as exc:  # report, never fail the bench line
            cpu = {"value": None, "unit": UNIT, "cores": _cores(), "kind": "oracle", "sample": f"failed: {exc}"}
        try:
            subcase = cpu_subcase_errors(sub, sub_u)
        except Exception as exc:
            subcase = {"failed": str(exc)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(w),
                "iters": iters, "true_rel_res": info_chk["true_rel_res"], "roofline": roofline,
                "geometry": "iffd_autotune (tiles and radix sequences tuned in setup, excluded from timing)",
                "tiles": [plan.tiles(a) for a in range(w.d)],
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(gpu_launches), "clocks": clk,
                "variants": variants, "precond_apply": apply_stats, "kernels": rooflines,
                "hbm_frac_of_solve": None, "subcase_64": subcase,
                "peaks": {"fp64_fma_tflops": fp64_peak, "fp32_fma_tflops": pk32["tflops"],
                          "fp32x2_fma_tflops": pk32x2["tflops"],
                          "sm_count": pk64["sm_count"], "hbm_gbs": hbm_peak}}
        # fraction of HBM peak of the whole solve at the method's algorithmic traffic
        # (176 B/DoF per PCG iteration: 96 preconditioner + 32 stiffness with the
        # direction update + 48 for the x, r update; 96 for the initial apply)
        line["hbm_frac_of_solve"] = (176.0 * w.N * iters + 96.0 * w.N) / (ms / args.steps / 1e3) / 1e9 / hbm_peak
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
