"""GPU tests of the persistent pipelined transform kernel (each CTA loads its
next tile with asynchronous copies while it transforms the current one): it
must give bitwise the results of the plain kernel (same arithmetic, same
partial sums) and therefore match the oracle."""

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import oracle_precond, require_gpu

pytestmark = pytest.mark.gpu


def _gpu(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# DST-I, DST-II/III, Bluestein, mixed boundaries (generic transform); tiles of
# 2..32 pencils; tile counts from a few to many per CTA
CASES = [
    (3, 40, 4, None, "fp64", 8), (3, 33, 3, None, "fp64", 2), (2, 149, 5, None, "fp64", 4),
    (3, 24, 4, ((1, 0), (0, 1), (0, 0)), "fp64", 16), (3, 40, 4, None, "fp32", 16), (2, 64, 3, None, "fp32", 32),
    (3, 64, 6, None, "fp32", 8),
]


def _dset(pair):
    return tuple(k for k, v in zip((0, 1), pair) if v)


@pytest.mark.parametrize("d,n,p,dirichlet,prec,pp", CASES)
def test_pipelined_pass_equals_plain_and_oracle(d, n, p, dirichlet, prec, pp):
    torch = require_gpu()
    from oracle import operators, splitting
    from paper_2512_20269_gb300 import IFFDPlan
    plain = IFFDPlan(d, n, p, precision=prec, dirichlet=dirichlet)
    pipe = IFFDPlan(d, n, p, precision=prec, dirichlet=dirichlet)
    for a in range(d):
        plain.set_geometry(a, pencils_transform=pp, pipelined=False)
        pipe.set_geometry(a, pencils_transform=pp, pipelined=True)
        assert pipe.tiles(a)["pipelined"] and not plain.tiles(a)["pipelined"]
    r = inputs.rhs(plain.shape, "normal", seed=700 + n + p)
    rg = _gpu(torch, r)
    z0 = plain.apply_preconditioner(rg)
    z1 = pipe.apply_preconditioner(rg)
    assert torch.equal(z0, z1)
    D = dirichlet or [(1, 1)] * d
    zo = operators.iffd_apply(r, [splitting.axis_split(n, p, _dset(pair)) for pair in D])
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.linalg.norm(z1.cpu().numpy() - zo) <= tol * np.linalg.norm(zo)
    u0, i0 = plain.pcg_solve(rg)
    u1, i1 = pipe.pcg_solve(rg)
    assert i0["iters"] == i1["iters"] and torch.equal(u0, u1)
    assert i1["true_rel_res"] <= 1.1e-8


def test_set_geometry_errors():
    require_gpu()
    from paper_2512_20269_gb300 import IFFDError, IFFDPlan
    plan = IFFDPlan(3, 16, 4)
    with pytest.raises(IFFDError):
        plan.set_geometry(0, pencils_transform=3)
    with pytest.raises(IFFDError):
        plan.set_geometry(5, pencils_transform=8)
    plan.set_geometry(1, pencils_transform=16, pencils_stiffness=4, pipelined=True)
    t = plan.tiles(1)
    assert (t["pencils_transform"], t["pencils_stiffness"], t["pipelined"]) == (16, 4, True)
