"""Pins of the general-coefficient stiffness oracle (oracle.general): what fixes
it independently of itself.

* a = 1 gives the Kronecker stiffness of eq. "system_matrix" (built from the
  banded 1D M and K, another assembly path);
* a = 1 + s_1 s_2 s_3 / 2 gives the separable variable-coefficient operator
  (1D matrices weighted by s);
* a constant diagonal C gives sum_k c_kk (M x .. K_k .. x M);
* an off-diagonal constant C is fixed by a closed-form integral of two
  polynomials the spline space reproduces;
* A is symmetric, and positive definite with Dirichlet ends, for a random
  symmetric positive definite field C(x);
* for non-separable scalar and tensor fields on a tiny 2D grid, A equals a
  brute-force element-by-element Galerkin assembly (tensor-product B-splines
  and their gradients evaluated point by point, no Kronecker factorisation);
* the quadrature data: weights sum to 1, values form a partition of unity,
  derivatives sum to 0;
* and mistakes planted in the oracle (values and derivatives swapped,
  directions reversed, a wrong or dropped tensor component, transposed
  weights) each break one of these pins.
"""

import numpy as np
import pytest

from oracle import general, operators, splines


def _axes(ns, p, dsets, reps=None):
    reps = reps or [None] * len(ns)
    return [general.quad_axis(n, p, D, rep=r) for n, D, r in zip(ns, dsets, reps)]


def _mk(ns, p, dsets, reps=None, weight=None):
    reps = reps or [None] * len(ns)
    return [splines.mass_stiffness(n, p, D, weight=weight, rep=r) for n, D, r in zip(ns, dsets, reps)]


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


CASES = [((5, 7), 2, [(0, 1), (0,)], None), ((6, 4, 5), 3, [(0, 1), (1,), (0, 1)], None),
         ((8, 5), 4, [(0, 1), (0, 1)], [{4: 2}, None]), ((4, 5, 6), 2, [(), (0, 1), (0,)], None)]


@pytest.mark.parametrize("ns,p,dsets,reps", CASES)
def test_unit_coefficient_is_the_kronecker_stiffness(ns, p, dsets, reps):
    axes = _axes(ns, p, dsets, reps)
    mk = _mk(ns, p, dsets, reps)
    u = _rand(tuple(M.shape[0] for M, _ in reversed(mk)), 1)
    C = np.ones((1,) + tuple(ax[0].size for ax in reversed(axes)))
    ref = operators.stiffness_apply(u, mk)
    assert np.max(np.abs(general.general_stiffness_apply(u, axes, C) - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_separable_sine_coefficient_is_the_varcoef_operator():
    ns, p, dsets = (6, 5, 7), 3, [(0, 1)] * 3
    axes = _axes(ns, p, dsets)
    s = [np.sin(2 * np.pi * ax[0]) for ax in axes]
    a = 1.0 + 0.5 * np.multiply.outer(s[2], np.multiply.outer(s[1], s[0]))
    u = _rand(tuple(ax[2].shape[1] for ax in reversed(axes)), 2)
    mk = _mk(ns, p, dsets)
    mks = _mk(ns, p, dsets, weight=lambda x: np.sin(2 * np.pi * x))
    ref = operators.varcoef_stiffness_apply(u, mk, mks, 0.5)
    got = general.general_stiffness_apply(u, axes, a[None])
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_constant_diagonal_tensor():
    ns, p, dsets = (5, 6, 4), 2, [(0, 1), (0,), (1,)]
    axes = _axes(ns, p, dsets)
    mk = _mk(ns, p, dsets)
    c = (0.7, 1.9, 3.1)
    shape_q = tuple(ax[0].size for ax in reversed(axes))
    C = np.zeros((6,) + shape_q)
    C[0], C[3], C[5] = c  # (11, 12, 13, 22, 23, 33)
    u = _rand(tuple(M.shape[0] for M, _ in reversed(mk)), 3)
    ref = np.zeros_like(u)
    for k in range(3):
        ref += c[k] * operators.kron_apply([mk[j][1] if j == k else mk[j][0] for j in range(3)], u)
    assert np.max(np.abs(general.general_stiffness_apply(u, axes, C) - ref)) <= 1e-12 * np.max(np.abs(ref))


def _project(ax, fn):
    """Coefficients of fn in the full spline space (exact when fn is in it):
    the L2 projection with the Gauss rule, which integrates these products exactly."""
    x, w, B, _ = ax
    M = B.T @ (w[:, None] * B)
    return np.linalg.solve(M, B.T @ (w * fn(x)))


@pytest.mark.parametrize("n,p", [(4, 2), (5, 3), (3, 4)])
def test_off_diagonal_closed_form(n, p):
    """Natural ends, u = x^2 y and v = x y^2 (both in the space for p >= 2),
    constant C = [[c11, c12], [c12, c22]]: v^T A u = int grad v . C grad u
    = c11 / 4 + 5 c12 / 9 + c22 / 4."""
    ax = general.quad_axis(n, p, ())
    c11, c12, c22 = 1.3, -0.4, 0.8
    shape_q = (ax[0].size, ax[0].size)
    C = np.stack([np.full(shape_q, c11), np.full(shape_q, c12), np.full(shape_q, c22)])
    one, lin, sq = _project(ax, lambda t: np.ones_like(t)), _project(ax, lambda t: t), _project(ax, lambda t: t * t)
    del one
    u = np.multiply.outer(lin, sq)  # shape (y, x): u = x^2 y
    v = np.multiply.outer(sq, lin)  # v = x y^2
    val = float(np.sum(v * general.general_stiffness_apply(u, [ax, ax], C)))
    assert abs(val - (c11 / 4 + 5 * c12 / 9 + c22 / 4)) <= 1e-12


def test_random_spd_field_gives_spd_matrix():
    ns, p, dsets = (3, 4, 3), 2, [(0, 1), (0,), (0, 1)]
    axes = _axes(ns, p, dsets)
    shape_q = tuple(ax[0].size for ax in reversed(axes))
    rng = np.random.default_rng(4)
    L = rng.standard_normal((3, 3) + shape_q) * 0.3
    Cf = np.einsum("ik...,jk...->ij...", L, L) + np.eye(3).reshape(3, 3, 1, 1, 1)
    C = np.stack([Cf[i, j] for i in range(3) for j in range(i, 3)])
    A = general.general_stiffness_dense(axes, C)
    assert np.max(np.abs(A - A.T)) <= 1e-13 * np.max(np.abs(A))
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0.0


@pytest.mark.parametrize("n,p,rep", [(6, 3, None), (7, 4, {3: 2})])
def test_quadrature_data(n, p, rep):
    x, w, B, D = general.quad_axis(n, p, (), rep=rep)
    assert x.size == n * (p + 1) and np.all(np.diff(x) > 0)
    assert abs(w.sum() - 1.0) <= 1e-14
    assert np.max(np.abs(B.sum(axis=1) - 1.0)) <= 1e-13
    assert np.max(np.abs(D.sum(axis=1))) <= 1e-11



def _pin_errors():
    """The pins above as numbers (each must be ~0 for a correct oracle)."""
    errs = {}
    ns, p, dsets = (5, 7), 2, [(0, 1), (0,)]
    axes = _axes(ns, p, dsets)
    mk = _mk(ns, p, dsets)
    u = _rand(tuple(M.shape[0] for M, _ in reversed(mk)), 1)
    C = np.ones((1,) + tuple(ax[0].size for ax in reversed(axes)))
    ref = operators.stiffness_apply(u, mk)
    errs["unit"] = np.max(np.abs(general.general_stiffness_apply(u, axes, C) - ref)) / np.max(np.abs(ref))
    ns, p, dsets = (5, 6, 4), 2, [(0, 1), (0,), (1,)]
    axes = _axes(ns, p, dsets)
    mk = _mk(ns, p, dsets)
    c = (0.7, 1.9, 3.1)
    C = np.zeros((6,) + tuple(ax[0].size for ax in reversed(axes)))
    C[0], C[3], C[5] = c
    u = _rand(tuple(M.shape[0] for M, _ in reversed(mk)), 3)
    ref = sum(c[k] * operators.kron_apply([mk[j][1] if j == k else mk[j][0] for j in range(3)], u) for k in range(3))
    errs["diag"] = np.max(np.abs(general.general_stiffness_apply(u, axes, C) - ref)) / np.max(np.abs(ref))
    ax = general.quad_axis(4, 2, ())
    shape_q = (ax[0].size, ax[0].size)
    C = np.stack([np.full(shape_q, 1.3), np.full(shape_q, -0.4), np.full(shape_q, 0.8)])
    lin, sq = _project(ax, lambda t: t), _project(ax, lambda t: t * t)
    val = float(np.sum(np.multiply.outer(sq, lin) * general.general_stiffness_apply(np.multiply.outer(lin, sq),
                                                                                    [ax, ax], C)))
    errs["offdiag"] = abs(val - (1.3 / 4 + 5 * -0.4 / 9 + 0.8 / 4))
    return errs


def test_pins_catch_planted_mistakes(monkeypatch):
    """Plausible mistakes planted in the oracle (on the CPU) each break at
    least one pin: the pins fix the derivative placement, the direction
    order, the component order of the tensor, and the weight layout."""
    assert max(_pin_errors().values()) <= 1e-12
    real_kron = general.kron_apply
    real_component = general.component
    real_weights = general.weights
    real_quad = general.quad_axis

    def swapped_bd(n, p, dirichlet=(0, 1), rep=None):  # derivatives in place of values and back
        x, w, B, D = real_quad(n, p, dirichlet, rep)
        return x, w, D, B

    def reversed_directions(mats, u):  # direction k's matrix applied along another direction
        return real_kron(mats[::-1], u)

    def wrong_component(C, d, k, l):  # C12 read from the C22 slot
        if C.shape[0] > 1 and {k, l} == {0, 1}:
            return real_component(C, d, 1, 1)
        return real_component(C, d, k, l)

    def dropped_offdiag(C, d, k, l):  # off-diagonal terms dropped
        return real_component(C, d, k, l) if k == l else 0.0

    def transposed_weights(axes):  # direction 1's weights on the slowest axis
        return np.transpose(real_weights(axes))

    for name, attr, fake in (("swap", "quad_axis", swapped_bd), ("direction", "kron_apply", reversed_directions),
                             ("component", "component", wrong_component),
                             ("offdiag", "component", dropped_offdiag), ("weights", "weights", transposed_weights)):
        with monkeypatch.context() as m:
            m.setattr(general, attr, fake)
            try:
                errs = _pin_errors()
                worst = max(errs.values())
            except ValueError:  # shapes no longer match: the mistake is caught too
                worst = np.inf
            assert worst > 1e-6, name


@pytest.mark.parametrize("kind", ["scalar", "tensor"])
def test_non_separable_coefficient_by_element_assembly(kind):
    """Brute force on a tiny 2D grid: A_ij = sum over elements and tensor Gauss
    points of w grad B_i . C grad B_j, with the tensor-product B-splines and
    their gradients evaluated point by point (no Kronecker factorisation),
    for a non-separable C, equals the oracle's matrix."""
    ns, p, dsets = (3, 4), 2, [(0, 1), (0,)]
    knots = [splines.open_knots(n, p) for n in ns]
    keep = [splines.kept_indices(n, p, D) for n, D in zip(ns, dsets)]
    m = [len(k) for k in keep]
    pos = [{int(g): i for i, g in enumerate(k)} for k in keep]

    def coef(x, y):
        if kind == "scalar":
            return np.array([[1.0 + x * y * y + np.sin(x + 2 * y), 0.0], [0.0, 0.0]])
        a, b = 1.2 + np.cos(3 * x * y), 0.9 + x * x
        c = 0.3 * np.sin(x + y)
        return np.array([[a, c], [c, b]])

    A = np.zeros((m[0] * m[1], m[0] * m[1]))
    for ex in range(ns[0]):
        xg, wx = splines.gauss_rule(p + 1, ex / ns[0], (ex + 1) / ns[0])
        Bx, Dx = splines.bspline_derivs(knots[0], p, ex, xg, 0), splines.bspline_derivs(knots[0], p, ex, xg, 1)
        sx = splines._element_span(knots[0], ex, ns[0]) - p
        for ey in range(ns[1]):
            yg, wy = splines.gauss_rule(p + 1, ey / ns[1], (ey + 1) / ns[1])
            By, Dy = splines.bspline_derivs(knots[1], p, ey, yg, 0), splines.bspline_derivs(knots[1], p, ey, yg, 1)
            sy = splines._element_span(knots[1], ey, ns[1]) - p
            for gx in range(p + 1):
                for gy in range(p + 1):
                    C = coef(xg[gx], yg[gy])
                    if kind == "scalar":
                        C = C[0, 0] * np.eye(2)
                    funcs = []
                    for ix in range(p + 1):
                        for iy in range(p + 1):
                            gi, gj = sx + ix, sy + iy
                            if gi in pos[0] and gj in pos[1]:
                                grad = np.array([Dx[gx, ix] * By[gy, iy], Bx[gx, ix] * Dy[gy, iy]])
                                funcs.append((pos[0][gi] + m[0] * pos[1][gj], grad))
                    for r, gr in funcs:
                        for c, gc in funcs:
                            A[r, c] += wx[gx] * wy[gy] * gr @ C @ gc
    axes = _axes(ns, p, dsets)
    X = np.meshgrid(axes[1][0], axes[0][0], indexing="ij")  # (y, x) grids
    Y, Xx = X[0], X[1]
    if kind == "scalar":
        Cq = (1.0 + Xx * Y * Y + np.sin(Xx + 2 * Y))[None]
    else:
        Cq = np.stack([1.2 + np.cos(3 * Xx * Y), 0.3 * np.sin(Xx + Y), 0.9 + Xx * Xx])
    got = general.general_stiffness_dense(axes, Cq)
    assert np.max(np.abs(got - A)) <= 1e-12 * np.max(np.abs(A))
