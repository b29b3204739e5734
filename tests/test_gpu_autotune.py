"""GPU tests of the launch-geometry autotuner (iffd_autotune): a tuned plan still
matches the oracle, picks a geometry from the candidate set, and plans of the
same size class (stand-alone or inside the engine) get the same geometry and
bitwise the same results."""

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import oracle_precond, oracle_stiffness, oracle_varcoef_stiffness, rel_max_err, require_gpu

pytestmark = pytest.mark.gpu


def _gpu(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# 102^3 and 111^3 are large enough to be tuned (a pass needs 4 x 152 tiles);
# the 2D Bluestein case keeps the default geometry.
@pytest.mark.parametrize("d,n,p,prec", [(3, 100, 4, "fp64"), (2, 149, 5, "fp64"), (3, 110, 3, "fp32")])
def test_tuned_plan_matches_oracle_and_is_cached(d, n, p, prec):
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(d, n, p, precision=prec).autotune()
    for a in range(d):
        t = plan.tiles(a)
        assert t["pencils_transform"] in (2, 4, 8, 16, 32) and t["pencils_stiffness"] in (2, 4, 8, 16, 32)
        assert t["radices"] and all(r > 1 for r in t["radices"])
    r = inputs.rhs(plan.shape, "normal", seed=70 + n)
    rg = _gpu(torch, r)
    z = plan.apply_preconditioner(rg).cpu().numpy()
    zo = oracle_precond(r, n, p)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.linalg.norm(z - zo) <= tol * np.linalg.norm(zo)
    assert rel_max_err(plan.apply_stiffness(rg).cpu().numpy(), oracle_stiffness(r, n, p)) <= 1e-13
    u, info = plan.pcg_solve(rg)
    assert info["status"] == 0 and info["true_rel_res"] <= 1.1e-8
    # a second plan of the same class takes the cached geometry: same tiles,
    # bitwise the same preconditioner and solution
    plan2 = IFFDPlan(d, n, p, precision=prec).autotune()
    assert [plan2.tiles(a) for a in range(d)] == [plan.tiles(a) for a in range(d)]
    assert torch.equal(plan2.apply_preconditioner(rg), plan.apply_preconditioner(rg))
    u2, info2 = plan2.pcg_solve(rg)
    assert info2["iters"] == info["iters"] and torch.equal(u2, u)


def test_tuned_varcoef_stiffness():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    n, p = 20, 4
    plan = IFFDPlan(3, n, p, coef="sin").autotune()
    u = inputs.rhs(plan.shape, "normal", seed=71)
    Au = plan.apply_stiffness(_gpu(torch, u)).cpu().numpy()
    assert rel_max_err(Au, oracle_varcoef_stiffness(u, n, p)) <= 1e-13


def test_engine_autotune_equals_tuned_plan():
    """With autotune the engine tunes each class at its first request; every
    result equals the stand-alone solve of a tuned plan bitwise."""
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDEngine, IFFDPlan
    mix = [(2, 30, 4), (3, 100, 4), (3, 26, 5), (2, 61, 4), (3, 100, 4)]
    eng = IFFDEngine(2 << 30, precision="fp32", autotune=True)
    reqs = {}
    for k, (d, n, p) in enumerate(mix):
        m = n + p - 2
        f = _gpu(torch, inputs.rhs((m,) * d, "normal", seed=400 + k))
        u = torch.empty_like(f)
        reqs[eng.submit(d, n, p, f, u)] = (d, n, p, f, u)
    done = dict(eng.run_to_completion(iterations_per_step=2))
    for rid, (d, n, p, f, u) in reqs.items():
        plan = IFFDPlan(d, n, p, precision="fp32", true_residual=False).autotune()
        ua, ia = plan.pcg_solve(f)
        assert done[rid]["iters"] == ia["iters"]
        assert torch.equal(u, ua), (d, n, p)
