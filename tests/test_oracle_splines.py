"""Pins of the oracle's univariate B-spline layer (Section 2) against facts the
paper or textbook mathematics fix independently of the oracle's code."""

import numpy as np
import pytest

from oracle import splines


def eulerian(n: int) -> np.ndarray:
    """Eulerian numbers A(n, k), k = 0..n-1, from their recurrence
    A(n, k) = (k+1) A(n-1, k) + (n-k) A(n-1, k-1). The centred cardinal
    B-spline of odd degree n takes the values A(n, k)/n! at the integers
    (a classical identity, independent of the B-spline recurrence)."""
    A = [1]
    for nn in range(2, n + 1):
        prev = A + [0]
        A = [(k + 1) * prev[k] + (nn - k) * (prev[k - 1] if k > 0 else 0) for k in range(nn)]
    return np.array(A, dtype=np.float64)


@pytest.mark.parametrize("deg", [1, 3, 5, 7, 9, 15, 17])
def test_cardinal_odd_degree_equals_eulerian_numbers(deg):
    from math import factorial
    half = (deg + 1) // 2
    ks = np.arange(-half + 1, half, dtype=np.float64)
    vals = splines.cardinal_bspline(deg, ks)
    ref = eulerian(deg)
    # A(deg, k) for k = 0..deg-1 are the values at -(deg-1)/2 .. (deg-1)/2
    np.testing.assert_allclose(vals, ref / factorial(deg), rtol=0, atol=1e-15)


def test_cardinal_small_degrees_p15():
    """P15: B~_3(0)=2/3, B~_3(+-1)=1/6, B~_2(0)=3/4, B~_2(+-1)=1/8; integer
    samples sum to 1 (partition of unity of the integer translates)."""
    np.testing.assert_allclose(splines.cardinal_bspline(3, [0.0, 1.0, -1.0]), [2 / 3, 1 / 6, 1 / 6], atol=1e-16)
    np.testing.assert_allclose(splines.cardinal_bspline(2, [0.0, 1.0, -1.0]), [3 / 4, 1 / 8, 1 / 8], atol=1e-16)
    for q in range(0, 12):
        ks = np.arange(-q - 1, q + 2, dtype=np.float64)
        assert abs(splines.cardinal_bspline(q, ks).sum() - 1.0) < 1e-14
        x = np.linspace(-3, 3, 37) + 0.123
        tot = sum(splines.cardinal_bspline(q, x - k) for k in range(-q - 4, q + 5))
        np.testing.assert_allclose(tot, 1.0, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 8])
def test_partition_of_unity_and_derivatives(p):
    """Cox-de Boor values sum to 1 (Section 2); derivatives agree with a
    central difference of the values and sum to 0."""
    n = 7
    knots = splines.open_knots(n, p)
    assert knots.size == n + 2 * p + 1
    for e in [0, 3, n - 1]:
        x = np.linspace(e / n, (e + 1) / n, 9)[1:-1]
        B = splines.bspline_derivs(knots, p, e, x, 0)
        np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-14)
        assert (B >= -1e-15).all()
        eps = 1e-6
        dB = splines.bspline_derivs(knots, p, e, x, 1)
        fd = (splines.bspline_derivs(knots, p, e, x + eps, 0) - splines.bspline_derivs(knots, p, e, x - eps, 0)) / (2 * eps)
        np.testing.assert_allclose(dB, fd, atol=1e-6 * max(1.0, np.abs(dB).max()))
        np.testing.assert_allclose(dB.sum(axis=1), 0.0, atol=1e-10)
        if p >= 2:
            d2 = splines.bspline_derivs(knots, p, e, x, 2)
            fd2 = (splines.bspline_derivs(knots, p, e, x + eps, 1) - splines.bspline_derivs(knots, p, e, x - eps, 1)) / (2 * eps)
            np.testing.assert_allclose(d2, fd2, atol=1e-5 * max(1.0, np.abs(d2).max()))


def test_linear_hat_matrices_textbook():
    """p = 1: hat functions; M = h/6 tridiag(1,4,1), K = 1/h tridiag(-1,2,-1)
    on the Dirichlet space (the classical P1 finite-element matrices)."""
    n = 9
    h = 1.0 / n
    M, K = splines.mass_stiffness(n, 1, (0, 1))
    m = n - 1
    Mref = h / 6 * (4 * np.eye(m) + np.eye(m, k=1) + np.eye(m, k=-1))
    Kref = 1 / h * (2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1))
    np.testing.assert_allclose(M, Mref, atol=1e-15)
    np.testing.assert_allclose(K, Kref, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
def test_mass_stiffness_p1_p2(p):
    """P1: before Dirichlet removal the mass matrix sums to 1 and K annihilates
    constants. P2: symmetric, half-bandwidth p, M SPD, K SPD on S_{p,h,{0,1}}.
    Interior rows of M are h * B~_{2p+1}(k) (autocorrelation of the cardinal
    B-spline, checked against the Eulerian numbers)."""
    from math import factorial
    n = 3 * p + 4
    Mf, Kf = splines.assemble_full(n, p)
    assert abs(Mf.sum() - 1.0) < 1e-13
    assert np.abs(Kf @ np.ones(n + p)).max() < 1e-10 * np.abs(Kf).max()
    M, K = splines.mass_stiffness(n, p, (0, 1))
    assert M.shape == (n + p - 2, n + p - 2)
    for A in (M, K):
        np.testing.assert_allclose(A, A.T, atol=1e-15 * np.abs(A).max())
        i, j = np.nonzero(np.abs(A) > 0)
        assert np.abs(i - j).max() == p
    assert np.linalg.eigvalsh(M).min() > 0
    assert np.linalg.eigvalsh(K).min() > 0
    # an interior row of the full matrix: B_r with r = p + 1 .. n - 2 has full support
    r = p + (n - 2 * p) // 2
    row = Mf[r, r - p:r + p + 1] * n
    ref = eulerian(2 * p + 1) / factorial(2 * p + 1)
    np.testing.assert_allclose(row, ref, atol=1e-12)


def test_weighted_matrices_reduce_to_plain():
    """A constant weight a = 2 doubles M and K (the weighted assembly path)."""
    M, K = splines.mass_stiffness(11, 4, (0, 1))
    Mw, Kw = splines.mass_stiffness(11, 4, (0, 1), weight=lambda x: 2.0 + 0 * x)
    np.testing.assert_allclose(Mw, 2 * M, atol=1e-15)
    np.testing.assert_allclose(Kw, 2 * K, atol=1e-11)
