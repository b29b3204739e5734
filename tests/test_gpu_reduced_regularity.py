"""GPU parity with repeated interior knots (reduced regularity, Remark
"reduced_regularity" of Section 4): the regular space and its transform are
unchanged, V_reg gets a dense block around every repeated knot, S^out grows by
one function per extra knot copy, and the stiffness sweeps use general band
rows. Compared element by element with the oracle (its V_reg by L2 projection,
its V_out from the null space of V_reg^T) on the same seeded inputs."""

import functools

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import rel_max_err, require_gpu

pytestmark = pytest.mark.gpu


def _dset(pair):
    return tuple(k for k, v in zip((0, 1), pair) if v)


def _key(rep):
    return tuple(sorted((rep or {}).items()))


@functools.lru_cache(maxsize=None)
def _split(n, p, pair, rep):
    from oracle import splitting
    return splitting.axis_split(n, p, _dset(pair), rep=dict(rep))


@functools.lru_cache(maxsize=None)
def _sin_mk(n, p, pair, rep):
    import scipy.sparse
    from oracle import splines
    Ms, Ks = splines.mass_stiffness(n, p, _dset(pair), weight=lambda x: np.sin(2 * np.pi * x), rep=dict(rep))
    return scipy.sparse.csr_matrix(Ms), scipy.sparse.csr_matrix(Ks)


def _splits(ns, p, dirichlet, knots):
    return [_split(n, p, tuple(D), _key(k)) for n, D, k in zip(ns, dirichlet, knots)]


def _mk(ns, p, dirichlet, knots):
    import scipy.sparse
    return [(scipy.sparse.csr_matrix(s.M), scipy.sparse.csr_matrix(s.K)) for s in _splits(ns, p, dirichlet, knots)]


def _gpu(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# (d, n per direction, p, Dirichlet flags, repeated knots per direction):
# interior knots, several knots on one axis, knots next to an end (their
# block joins the edge block), the largest multiplicity p - 1, natural ends,
# directions without repeats, a Bluestein length (n = 37), and tiny n where
# V_reg is one dense block
CASES = [
    (2, (24, 24), 3, ((1, 1), (1, 1)), ({12: 2}, None)),
    (2, (20, 22), 4, ((1, 1), (1, 0)), ({5: 1, 14: 3}, {11: 2})),
    (2, (30, 18), 2, ((0, 1), (1, 1)), ({15: 1}, {1: 1})),
    (2, (16, 37), 5, ((1, 1), (0, 1)), ({2: 4}, {18: 2, 30: 1})),
    (2, (26, 20), 8, ((1, 1), (1, 1)), ({13: 7}, None)),
    (3, (12, 13, 14), 3, ((1, 1), (1, 1), (1, 1)), ({6: 1}, {4: 2, 9: 1}, None)),
    (3, (14, 12, 12), 4, ((1, 0), (0, 1), (1, 1)), ({7: 3}, None, {11: 1})),
    (3, (10, 9, 9), 6, ((1, 1), (1, 1), (1, 1)), ({5: 5}, None, None)),
    (2, (5, 9), 4, ((1, 1), (1, 1)), (None, {4: 2})),
    (3, (64, 48, 40), 4, ((1, 1), (1, 1), (1, 1)), ({32: 1}, {10: 2, 30: 3}, {20: 3})),
    (2, (200, 160), 3, ((1, 1), (1, 0)), ({100: 2}, {40: 1, 120: 1})),
]


@pytest.mark.parametrize("d,ns,p,dirichlet,knots", CASES)
def test_reduced_regularity_preconditioner_and_stiffness_parity(d, ns, p, dirichlet, knots):
    torch = require_gpu()
    from oracle import operators
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(d, list(ns), p, dirichlet=dirichlet, knots=list(knots))
    sp = _splits(ns, p, dirichlet, knots)
    assert tuple(plan.m) == tuple(s.m for s in sp)
    r = inputs.rhs(plan.shape, "normal", seed=300 + sum(ns) + p)
    rg = _gpu(torch, r)
    zo = operators.iffd_apply(r, sp)
    z = plan.apply_preconditioner(rg).cpu().numpy()
    assert rel_max_err(z, zo) <= 1e-12
    assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)
    Ao = operators.stiffness_apply(r, _mk(ns, p, dirichlet, knots))
    assert rel_max_err(plan.apply_stiffness(rg).cpu().numpy(), Ao) <= 1e-13
    z32 = IFFDPlan(d, list(ns), p, precision="fp32", dirichlet=dirichlet, knots=list(knots))
    z32 = z32.apply_preconditioner(rg).cpu().numpy()
    assert np.linalg.norm(z32 - zo) <= 1e-5 * np.linalg.norm(zo)


@pytest.mark.parametrize("d,ns,p,dirichlet,knots", [CASES[1], CASES[5], CASES[6]])
def test_reduced_regularity_pcg_matches_oracle(d, ns, p, dirichlet, knots):
    """PCG with the IFFD preconditioner on the reduced-regularity space: same
    iteration count as the oracle's PCG (+-1) on the same right-hand side, true
    relative residual <= 1.1e-8 against the oracle's operator."""
    torch = require_gpu()
    from oracle import operators
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(d, list(ns), p, dirichlet=dirichlet, knots=list(knots))
    f = inputs.rhs(plan.shape, "uniform", seed=41 + p)
    u, info = plan.pcg_solve(_gpu(torch, f))
    assert info["status"] == 0 and info["true_rel_res"] <= 1.1e-8
    sp = _splits(ns, p, dirichlet, knots)
    mk = _mk(ns, p, dirichlet, knots)
    _, it_o, _ = operators.pcg(f, lambda v: operators.stiffness_apply(v, mk),
                               lambda r: operators.iffd_apply(r, sp), rtol=1e-8)
    assert abs(info["iters"] - it_o) <= 1
    true_rel = np.linalg.norm(f - operators.stiffness_apply(u.cpu().numpy(), mk)) / np.linalg.norm(f)
    assert true_rel <= 1.1e-8


@pytest.mark.parametrize("d,ns,p,dirichlet,knots", [CASES[0], CASES[6]])
def test_reduced_regularity_exact_fd_varcoef_pipelined(d, ns, p, dirichlet, knots):
    torch = require_gpu()
    from oracle import operators
    from paper_2512_20269_gb300 import IFFDPlan
    r = inputs.rhs(tuple(reversed([s.m for s in _splits(ns, p, dirichlet, knots)])), "normal", seed=77 + p)
    rg = _gpu(torch, r)
    sp = _splits(ns, p, dirichlet, knots)
    fd = IFFDPlan(d, list(ns), p, precond="exact_fd", dirichlet=dirichlet, knots=list(knots))
    zo = operators.exact_fd_apply(r, [operators.exact_fd_eig(s.M, s.K) for s in sp])
    assert rel_max_err(fd.apply_preconditioner(rg).cpu().numpy(), zo) <= 1e-12
    vc = IFFDPlan(d, list(ns), p, coef="sin", dirichlet=dirichlet, knots=list(knots))
    mks = [_sin_mk(n, p, tuple(D), _key(k)) for n, D, k in zip(ns, dirichlet, knots)]
    Ao = operators.varcoef_stiffness_apply(r, _mk(ns, p, dirichlet, knots), mks, 0.5)
    assert rel_max_err(vc.apply_stiffness(rg).cpu().numpy(), Ao) <= 1e-13
    plain = IFFDPlan(d, list(ns), p, dirichlet=dirichlet, knots=list(knots))
    pipe = IFFDPlan(d, list(ns), p, dirichlet=dirichlet, knots=list(knots))
    for a in range(d):
        plain.set_geometry(a, pencils_transform=4, pipelined=False)
        pipe.set_geometry(a, pencils_transform=4, pipelined=True)
    assert torch.equal(plain.apply_preconditioner(rg), pipe.apply_preconditioner(rg))


def test_reduced_regularity_setup_errors():
    require_gpu()
    from paper_2512_20269_gb300 import IFFDError, IFFDPlan
    with pytest.raises(IFFDError):
        IFFDPlan(2, 16, 4, knots=[{16: 1}, None])
    with pytest.raises(IFFDError):
        IFFDPlan(2, 16, 4, knots=[{8: 4}, None])
    with pytest.raises(ValueError):
        IFFDPlan(2, 16, 4, knots=[{8: 1}])
    with pytest.raises(IFFDError):  # n_out above 16
        IFFDPlan(2, 40, 4, knots=[{5: 3, 10: 3, 15: 3, 20: 3, 25: 3, 30: 3}, None])
