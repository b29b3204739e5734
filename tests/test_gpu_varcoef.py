"""GPU parity of the variable-coefficient path: -div(a grad u) with
a = 1 + 0.5 sin(2 pi x1) sin(2 pi x2) [sin(2 pi x3)], stiffness by the tensor
(p+1)-point Gauss rule (exactly the rank-2 Kronecker form, pinned in the oracle
tests against direct Galerkin assembly), constant-coefficient IFFD as the
preconditioner."""

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import (oracle_precond, oracle_varcoef_sampled, oracle_varcoef_stiffness, rel_max_err,
                        require_gpu)

pytestmark = pytest.mark.gpu


def _gpu(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("d,n,p", [(2, 20, 3), (2, 17, 6), (3, 12, 4), (3, 10, 8), (3, 14, 5), (3, 9, 2)])
def test_varcoef_stiffness_parity(d, n, p):
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(d, n, p, coef="sin", coef_amp=0.5)
    u = inputs.rhs(plan.shape, "normal", seed=60 + n + p)
    Au = plan.apply_stiffness(_gpu(torch, u)).cpu().numpy()
    assert rel_max_err(Au, oracle_varcoef_stiffness(u, n, p)) <= 1e-13


@pytest.mark.parametrize("d,n,p", [(2, 40, 4), (3, 16, 8), (3, 20, 3)])
def test_varcoef_pcg_against_oracle(d, n, p):
    torch = require_gpu()
    from oracle import operators
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(d, n, p, coef="sin", coef_amp=0.5)
    f = inputs.rhs(plan.shape, "uniform", seed=70 + n)
    u, info = plan.pcg_solve(_gpu(torch, f))
    u = u.cpu().numpy()
    _, it_o, _ = operators.pcg(f, lambda v: oracle_varcoef_stiffness(v, n, p), lambda r: oracle_precond(r, n, p))
    assert info["status"] == 0
    assert abs(info["iters"] - it_o) <= 1, (info, it_o)
    true_rel = np.linalg.norm(f - oracle_varcoef_stiffness(u, n, p)) / np.linalg.norm(f)
    assert true_rel <= 1.1e-8
    # the preconditioner stays the constant-coefficient IFFD (A != A^ here)
    assert info["iters"] > 2


def test_varcoef_fp32_transform_iterations():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    f = _gpu(torch, inputs.rhs((26, 26, 26), "uniform", seed=2))
    _, i64 = IFFDPlan(3, 24, 4, coef="sin").pcg_solve(f)
    _, i32 = IFFDPlan(3, 24, 4, coef="sin", precision="fp32").pcg_solve(f)
    assert i64["true_rel_res"] <= 1.1e-8 and i32["true_rel_res"] <= 1.1e-8
    assert i32["iters"] <= i64["iters"] + 2


def test_noalloc_rejects_varcoef_plans():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan, _lib
    plan = IFFDPlan(3, 12, 3, coef="sin")
    u = plan.empty().zero_()
    rc = _lib.load().iffd_apply_stiffness_noalloc(plan._h, u.data_ptr(), plan.empty().data_ptr(), None)
    assert rc == 2


@pytest.mark.slow
def test_cube_n384_p8_varcoef_full():
    """390^3 = 59,319,000 DoFs: sampled stiffness outputs (interior, faces,
    edges, corners) against the oracle's local Kronecker sums; PCG to 1e-8."""
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    w = inputs.CUBE_N384_P8
    plan = IFFDPlan(w.d, w.n, w.p, coef="sin", coef_amp=0.5)
    f = inputs.workload_rhs(w)
    fg = _gpu(torch, f)
    Au = plan.apply_stiffness(fg)
    m = w.m
    rng = np.random.default_rng(5)
    pts = [(0, 0, 0), (m - 1, m - 1, m - 1), (0, m // 2, m - 1), (3, 7, 200), (m - 5, 1, 2)]
    pts += [tuple(int(x) for x in rng.integers(0, m, 3)) for _ in range(40)]
    got = np.array([float(Au[k, j, i]) for (k, j, i) in pts])
    ref = oracle_varcoef_sampled(f, w.n, w.p, pts)
    scale = float(Au.abs().max())
    assert np.abs(got - ref).max() <= 1e-13 * scale
    del Au
    u, info = plan.pcg_solve(fg)
    assert info["status"] == 0 and info["true_rel_res"] <= 1.1e-8
