"""GPU parity of the general-coefficient stiffness (-div(C(x) grad u) with C
sampled at the tensor Gauss points, Section 2's Galerkin form; Section 7's
pulled-back geometry has this form) and of PCG on it with the IFFD
preconditioner of the constant-coefficient operator. Compared element by
element with the oracle (oracle.general) on the same seeded inputs."""

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


def _gpu(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _dset(pair):
    return tuple(k for k, v in zip((0, 1), pair) if v)


def _axes(ns, p, dirichlet, knots):
    from oracle import general
    return [general.quad_axis(n, p, _dset(D), rep=k) for n, D, k in zip(ns, dirichlet, knots)]


def _coef(axes, kind):
    """Coefficient fields on the tensor Gauss grid (shape (ncomp, nq_d, .., nq_1)):
    a non-separable scalar, or a symmetric positive definite tensor whose
    principal axes turn with x (the form a curved geometry map gives)."""
    d = len(axes)
    X = np.meshgrid(*[ax[0] for ax in reversed(axes)], indexing="ij")[::-1]  # X[0] = x_1 (fastest)
    if kind == "scalar":
        s = sum((k + 1) * X[k] for k in range(d))
        return (1.0 + 0.5 * np.sin(2 * np.pi * s) * np.cos(np.pi * X[0] * X[1]))[None]
    if d == 2:
        th = np.pi * X[0] * X[1] + 0.3
        kap = 0.25 + X[1]
        c, s = np.cos(th), np.sin(th)
        return np.stack([c * c + kap * s * s, (1 - kap) * s * c, s * s + kap * c * c])
    v = [0.8 * np.sin(2 * np.pi * X[0] + X[2]), 0.7 * np.cos(2 * np.pi * X[1] * X[0]), 0.6 * np.sin(np.pi * X[2])]
    a = 1.0 + 0.3 * X[0] * X[1] * X[2]
    comps = [(i, j) for i in range(3) for j in range(i, 3)]
    return np.stack([(a if i == j else 0.0) + 0.5 * v[i] * v[j] for i, j in comps])


CASES = [
    (2, (24, 17), 3, ((1, 1), (1, 0)), (None, None), "scalar"),
    (2, (20, 22), 4, ((1, 1), (1, 1)), ({7: 2}, None), "tensor"),
    (2, (31, 9), 2, ((0, 1), (1, 1)), (None, None), "tensor"),
    (3, (10, 8, 12), 2, ((1, 1), (1, 1), (1, 1)), (None, None, None), "scalar"),
    (3, (9, 11, 7), 4, ((1, 1), (1, 0), (0, 1)), (None, {5: 1}, None), "tensor"),
    (3, (12, 6, 8), 3, ((1, 1), (1, 1), (1, 1)), (None, None, None), "tensor"),
]


@pytest.mark.parametrize("d,ns,p,dirichlet,knots,kind", CASES)
def test_general_stiffness_matches_oracle(d, ns, p, dirichlet, knots, kind):
    torch = require_gpu()
    from oracle import general
    from paper_2512_20269_gb300 import IFFDPlan
    kw = {} if all(k is None for k in knots) else {"knots": list(knots)}
    plan = IFFDPlan(d, list(ns), p, dirichlet=dirichlet, **kw)
    axes = _axes(ns, p, dirichlet, knots)
    for a in range(d):
        x, w = plan.quad_points(a)
        assert np.max(np.abs(x - axes[a][0])) <= 1e-15 and np.max(np.abs(w - axes[a][1])) <= 1e-15
    C = _coef(axes, kind)
    assert plan.quad_shape == C.shape[1:]
    u = inputs.rhs(plan.shape, "normal", seed=500 + sum(ns) + p)
    ref = general.general_stiffness_apply(u, axes, C)
    got = plan.apply_stiffness_general(_gpu(torch, C), _gpu(torch, u)).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_unit_coefficient_equals_constant_stiffness_at_size():
    """a = 1 (and C = I as a tensor) reproduces the constant-coefficient
    stiffness sweeps on a 66^3 grid with p = 4 (exact Gauss integration)."""
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(3, 64, 4)
    u = _gpu(torch, inputs.rhs(plan.shape, "normal", seed=8))
    Au = plan.apply_stiffness(u)
    q = plan.quad_shape
    one = torch.ones((1,) + q, dtype=torch.float64, device="cuda")
    eye = torch.zeros((6,) + q, dtype=torch.float64, device="cuda")
    eye[0] = eye[3] = eye[5] = 1.0
    scale = float(Au.abs().max())
    assert float((plan.apply_stiffness_general(one, u) - Au).abs().max()) <= 1e-12 * scale
    assert float((plan.apply_stiffness_general(eye, u) - Au).abs().max()) <= 1e-12 * scale


@pytest.mark.parametrize("case", [CASES[1], CASES[3], CASES[4]])
def test_general_pcg_matches_oracle(case):
    """PCG with the IFFD preconditioner of A^ on A_C u = f: same iteration
    count as the oracle's PCG (+-1), true relative residual <= 1.1e-8 against
    the oracle's operator."""
    d, ns, p, dirichlet, knots, kind = case
    torch = require_gpu()
    from oracle import general, operators, splitting
    from paper_2512_20269_gb300 import IFFDPlan
    kw = {} if all(k is None for k in knots) else {"knots": list(knots)}
    plan = IFFDPlan(d, list(ns), p, dirichlet=dirichlet, **kw)
    axes = _axes(ns, p, dirichlet, knots)
    C = _coef(axes, kind)
    f = inputs.rhs(plan.shape, "uniform", seed=61 + p)
    u, info = plan.pcg_solve_general(_gpu(torch, C), _gpu(torch, f))
    assert info["status"] == 0 and info["true_rel_res"] <= 1.1e-8
    sp = [splitting.axis_split(n, p, _dset(D), rep=k) for n, D, k in zip(ns, dirichlet, knots)]
    _, it_o, _ = operators.pcg(f, lambda v: general.general_stiffness_apply(v, axes, C),
                               lambda r: operators.iffd_apply(r, sp), rtol=1e-8)
    assert abs(info["iters"] - it_o) <= 1
    res = f - general.general_stiffness_apply(u.cpu().numpy(), axes, C)
    assert np.linalg.norm(res) <= 1.1e-8 * np.linalg.norm(f)


def test_general_pcg_at_size_and_unit_coefficient():
    """At 66^3, p = 4: with a = 1 the general solve takes the iterations of the
    constant-coefficient solve; with the non-separable tensor field (eigenvalues
    in [1, 2.1]) it still converges, within a few more iterations."""
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(3, 64, 4)
    f = _gpu(torch, inputs.rhs(plan.shape, "uniform", seed=9))
    _, i0 = plan.pcg_solve(f)
    one = torch.ones((1,) + plan.quad_shape, dtype=torch.float64, device="cuda")
    u1, i1 = plan.pcg_solve_general(one, f)
    assert i1["status"] == 0 and abs(i1["iters"] - i0["iters"]) <= 1 and i1["true_rel_res"] <= 1.1e-8
    axes = [(plan.quad_points(a)[0], None) for a in range(3)]
    C = _gpu(torch, _coef(axes, "tensor"))
    u2, i2 = plan.pcg_solve_general(C, f)
    assert i2["status"] == 0 and i2["true_rel_res"] <= 1.1e-8 and i2["iters"] <= 4 * i0["iters"] + 10
    # the solution satisfies the general operator
    r = f - plan.apply_stiffness_general(C, u2)
    assert float(torch.linalg.norm(r) / torch.linalg.norm(f)) <= 1.1e-8


def test_general_argument_errors():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDError, IFFDPlan
    plan = IFFDPlan(2, 12, 3)
    q = plan.quad_shape
    u = torch.zeros(plan.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):  # not ncomp x quad_shape values
        plan.apply_stiffness_general(torch.ones((5,) + q[1:], dtype=torch.float64, device="cuda"), u)
    with pytest.raises(IFFDError):  # ncomp = 2 in 2D
        plan.apply_stiffness_general(torch.ones((2,) + q, dtype=torch.float64, device="cuda"), u)
    with pytest.raises(IFFDError):  # u and Au alias
        plan.apply_stiffness_general(torch.ones((1,) + q, dtype=torch.float64, device="cuda"), u, u)
