"""GPU parity: every CUDA path through the C ABI against the CPU oracle on the
same seeded inputs.

Tolerances:
* FP64 preconditioner apply and exact FD: max |z - z_oracle| <= 1e-12 max |z_oracle|;
* FP32-transform preconditioner: 1e-5 (relative 2-norm);
* stiffness: 1e-13 max-norm relative;
* PCG: recurrence and true relative residual <= rtol (1e-8, true residual with
  a 1e-9 rounding allowance), iteration count within +-1 of the oracle's PCG.
"""

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import (oracle_exact_fd, oracle_pcg, oracle_precond, oracle_split, oracle_stiffness, rel_max_err,
                        require_gpu)

pytestmark = pytest.mark.gpu

# (d, n, p): several tiles and a ragged tail along every direction; odd and even
# p (DST-I / DST-II-III), odd n (odd-length DST), radices 2, 3, 4, 5, 7, 8.
SHAPES = [
    (2, 64, 3), (2, 20, 2), (2, 17, 5), (2, 45, 4), (2, 35, 6), (2, 7, 1), (2, 9, 8),
    (3, 16, 4), (3, 12, 3), (3, 21, 6), (3, 24, 8), (3, 14, 7), (3, 10, 2), (3, 25, 5),
]


def _to_gpu(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("d,n,p", SHAPES)
def test_preconditioner_fp64_parity(d, n, p):
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(d, n, p)
    r = inputs.rhs(plan.shape, "normal", seed=10 + n + p)
    z = plan.apply_preconditioner(_to_gpu(torch, r)).cpu().numpy()
    zo = oracle_precond(r, n, p)
    assert rel_max_err(z, zo) <= 1e-12
    assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)


@pytest.mark.parametrize("d,n,p", SHAPES[:4] + SHAPES[7:11])
def test_preconditioner_fp32_transform_error(d, n, p):
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(d, n, p, precision="fp32")
    r = inputs.rhs(plan.shape, "uniform", seed=20 + n + p)
    z = plan.apply_preconditioner(_to_gpu(torch, r)).cpu().numpy()
    zo = oracle_precond(r, n, p)
    assert np.linalg.norm(z - zo) <= 1e-5 * np.linalg.norm(zo)


@pytest.mark.parametrize("d,n,p", SHAPES)
def test_stiffness_parity(d, n, p):
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(d, n, p)
    u = inputs.rhs(plan.shape, "normal", seed=30 + n + p)
    Au = plan.apply_stiffness(_to_gpu(torch, u)).cpu().numpy()
    Ao = oracle_stiffness(u, n, p)
    assert rel_max_err(Au, Ao) <= 1e-13


@pytest.mark.parametrize("d,n,p", [(2, 20, 3), (2, 17, 4), (3, 12, 3), (3, 14, 4), (3, 10, 5)])
def test_exact_fd_parity(d, n, p):
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(d, n, p, precond="exact_fd")
    r = inputs.rhs(plan.shape, "normal", seed=40 + n)
    z = plan.apply_preconditioner(_to_gpu(torch, r)).cpu().numpy()
    zo = oracle_exact_fd(r, n, p)
    assert rel_max_err(z, zo) <= 1e-12


@pytest.mark.parametrize("d,n,p", [(2, 64, 3), (2, 30, 2), (3, 16, 4), (3, 12, 5), (3, 20, 8), (2, 40, 6)])
def test_pcg_fp64_against_oracle(d, n, p):
    """The GPU PCG stops where the oracle's PCG does and its iterate solves
    A^ u = f to the stated relative residual (checked with the oracle's A^)."""
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(d, n, p)
    f = inputs.rhs(plan.shape, "uniform", seed=50 + n + p)
    u, info = plan.pcg_solve(_to_gpu(torch, f))
    u = u.cpu().numpy()
    _, it_o, hist = oracle_pcg(f, n, p)
    assert info["status"] == 0
    assert abs(info["iters"] - it_o) <= 1, (info, it_o)
    assert info["rel_res"] <= 1e-8
    true_rel = np.linalg.norm(f - oracle_stiffness(u, n, p)) / np.linalg.norm(f)
    assert true_rel <= 1.1e-8
    assert abs(true_rel - info["true_rel_res"]) <= 1e-9
    if p == 2:
        assert info["iters"] == 1  # IFFD is exact when S^reg = S (end of Section 4)


def test_pcg_exact_fd_is_direct():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(3, 14, 4, precond="exact_fd")
    f = inputs.rhs(plan.shape, "normal", seed=3)
    _, info = plan.pcg_solve(_to_gpu(torch, f))
    assert info["iters"] == 1 and info["true_rel_res"] <= 1e-12


def test_pcg_fp32_transform_iterations():
    """FP32 transforms with FP64 PCG: same accuracy, at most 2 more iterations."""
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    w = inputs.CUBE_N64_P4
    f = _to_gpu(torch, inputs.workload_rhs(w))
    _, i64 = IFFDPlan(3, w.n, w.p).pcg_solve(f)
    _, i32 = IFFDPlan(3, w.n, w.p, precision="fp32").pcg_solve(f)
    assert i64["true_rel_res"] <= 1.1e-8 and i32["true_rel_res"] <= 1.1e-8
    assert i32["iters"] <= i64["iters"] + 2


def test_pcg_deterministic():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(3, 18, 4)
    f = _to_gpu(torch, inputs.rhs(plan.shape, "normal", seed=9))
    u1, i1 = plan.pcg_solve(f)
    u2, i2 = plan.pcg_solve(f)
    assert i1 == i2
    assert torch.equal(u1, u2)


@pytest.mark.parametrize("n", [128, 256])
def test_table_square_iterations(n):
    """Table "tab:square": 2D Dirichlet, p = 2..7 -> 1/7/6/6/6/6 (+-1)."""
    import json
    import os
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table_square_iterations.json")))
    ref = g["iterations"][g["n"].index(n)]
    for p, it_ref in zip(g["p"], ref):
        plan = IFFDPlan(2, n, p)
        f = _to_gpu(torch, inputs.rhs(plan.shape, "uniform", seed=100 + p))
        _, info = plan.pcg_solve(f)
        assert abs(info["iters"] - it_ref) <= 1, (p, info)
        assert info["true_rel_res"] <= 1.1e-8


def test_argument_errors():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan, IFFDError, _lib
    plan = IFFDPlan(2, 16, 3)
    r = torch.zeros(plan.shape, dtype=torch.float64, device="cuda")
    lib = _lib.load()
    rc = lib.iffd_apply_preconditioner(plan._h, r.data_ptr(), r.data_ptr(), plan._ws_ptr, None)
    assert rc == 1
    rc = lib.iffd_apply_preconditioner(plan._h, r.data_ptr(), plan.empty().data_ptr(), plan._ws_ptr + 8, None)
    assert rc == 4
    with pytest.raises(IFFDError):
        IFFDPlan(3, 4, 5)
    # zero right-hand side: converged at iteration 0, u = 0
    u, info = plan.pcg_solve(r)
    assert info["iters"] == 0 and float(u.abs().max()) == 0.0


@pytest.mark.parametrize("d,n,p", [(2, 64, 3), (3, 13, 3), (2, 33, 4)])
def test_ragged_tiles_and_padding(d, n, p):
    """Pencils share complex FFTs in pairs and the last tile of every direction
    is padded. A right-hand side supported only on the last x position (so its
    whole response passes through those ragged tiles) must still match the
    oracle to 1e-12, as must the full right-hand side."""
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(d, n, p)
    r = inputs.rhs(plan.shape, "normal", seed=77)
    z = plan.apply_preconditioner(_to_gpu(torch, r)).cpu().numpy()
    assert rel_max_err(z, oracle_precond(r, n, p)) <= 1e-12
    r2 = np.zeros_like(r)
    r2[..., -1] = r[..., -1]
    z2 = plan.apply_preconditioner(_to_gpu(torch, r2)).cpu().numpy()
    assert rel_max_err(z2, oracle_precond(r2, n, p)) <= 1e-12


# Transform lengths with a large prime factor run as Bluestein's chirp
# convolution: L = 298 (2 * 149), 134 (2 * 67), 61, 37 (3D), 58 (2 * 29, 3D).
BLUESTEIN_SHAPES = [(2, 149, 5), (2, 134, 6), (2, 61, 4), (3, 37, 4), (3, 29, 5)]


@pytest.mark.parametrize("d,n,p", BLUESTEIN_SHAPES)
def test_bluestein_preconditioner_parity(d, n, p):
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan, host_transform
    assert host_transform(n, p, "fp64")["bluestein"] and host_transform(n, p, "fp32")["bluestein"]
    plan = IFFDPlan(d, n, p)
    r = inputs.rhs(plan.shape, "normal", seed=60 + n + p)
    rg = _to_gpu(torch, r)
    zo = oracle_precond(r, n, p)
    z = plan.apply_preconditioner(rg).cpu().numpy()
    assert rel_max_err(z, zo) <= 1e-12
    assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)
    z32 = IFFDPlan(d, n, p, precision="fp32").apply_preconditioner(rg).cpu().numpy()
    assert np.linalg.norm(z32 - zo) <= 1e-5 * np.linalg.norm(zo)


def test_bluestein_long_fp32_and_pcg():
    """A 2D DST-I of length 556 (L = 1114 = 2 * 557, F = 2304): FP32 transforms
    within 1e-5 of the oracle, and a PCG solve through Bluestein passes reaches
    the relative residual in the oracle's iteration count (+-1)."""
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan, host_transform
    n, p = 557, 3
    assert host_transform(n, p, "fp32")["bluestein"]
    plan = IFFDPlan(2, n, p, precision="fp32")
    r = inputs.rhs(plan.shape, "uniform", seed=61)
    zo = oracle_precond(r, n, p)
    z = plan.apply_preconditioner(_to_gpu(torch, r)).cpu().numpy()
    assert np.linalg.norm(z - zo) <= 1e-5 * np.linalg.norm(zo)
    n, p = 149, 5
    plan = IFFDPlan(2, n, p)
    f = inputs.rhs(plan.shape, "uniform", seed=62)
    u, info = plan.pcg_solve(_to_gpu(torch, f))
    _, it_o, _ = oracle_pcg(f, n, p)
    assert info["status"] == 0 and abs(info["iters"] - it_o) <= 1
    true_rel = np.linalg.norm(f - oracle_stiffness(u.cpu().numpy(), n, p)) / np.linalg.norm(f)
    assert true_rel <= 1.1e-8
