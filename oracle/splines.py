"""Univariate B-spline discretisation (Section 2) -- oracle, test infrastructure only.

Everything is float64 and written for clarity, not speed.

* ``open_knots``          -- the p-open uniform knot vector of Section 2.
* ``bspline_table``       -- Cox-de Boor recursion (Section 2), with the rule that
                             a summand whose denominator vanishes is dropped.
* ``bspline_derivs``      -- k-th derivatives through the standard derivative
                             recursion d/dx B_{q,i} = q (B_{q-1,i}/(xi_{i+q}-xi_i)
                             - B_{q-1,i+1}/(xi_{i+q+1}-xi_{i+1})), same dropping rule.
* ``gauss_rule``          -- (p+1)-point Gauss-Legendre rule on an element
                             (library nodes; exact for the degree-2p products of M).
* ``assemble_full``       -- M_ij = int B_i B_j, K_ij = int B_i' B_j' over [0,1]
                             (Section 3, the 1D factors of eq. "system_matrix"),
                             optionally with a weight a(x) under the integral.
* ``kept_indices`` /
  ``mass_stiffness``      -- removal of the B-splines that do not vanish on the
                             Dirichlet set (end of Section 2): m = n + p - |D|.
* ``cardinal_bspline``    -- the symmetric cardinal B-spline of Lemma 3,
                             eq. "cardinal", evaluated by its recurrence.
"""

from __future__ import annotations

from fractions import Fraction

import numpy as np


def open_knots(n: int, p: int, rep=None) -> np.ndarray:
    """p-open knot vector on the uniform grid z_k = k/n (Section 2):
    p+1 copies of 0, the interior breakpoints 1/n..(n-1)/n, p+1 copies of 1.
    ``rep`` = {k: extra} repeats the interior breakpoint k/n extra more times
    (reduced regularity C^{p-1-extra} there, Remark "reduced_regularity")."""
    rep = rep or {}
    interior = []
    for k in range(1, n):
        interior += [k / n] * (1 + int(rep.get(k, 0)))
    return np.array([0.0] * (p + 1) + interior + [1.0] * (p + 1), dtype=np.float64)


def n_basis(n: int, p: int, rep=None) -> int:
    """Number of B-splines of S_{p,h} with the repeated knots ``rep``."""
    return n + p + sum(int(v) for v in (rep or {}).values())


def _element_span(knots: np.ndarray, e: int, n: int) -> int:
    """Index s with xi_s = z_e < xi_{s+1} = z_{e+1} for element e (0-based):
    the last knot equal to z_e."""
    return int(np.searchsorted(knots, e / n, side="right")) - 1


def bspline_table(knots: np.ndarray, q: int, e: int, x: np.ndarray, p: int, n: int | None = None) -> dict:
    """Cox-de Boor recursion up to degree q on element e of a degree-p knot vector.

    Returns {i: B_{q,i}(x)} for the B-splines of degree q that can be nonzero on
    element e. The degree-0 function of the element's span is 1 on the whole
    closed element (so end points are evaluated with the element's polynomial
    piece). Summands with a vanishing denominator are dropped (Section 2).
    """
    x = np.asarray(x, dtype=np.float64)
    n = _n_elements(knots, p) if n is None else n
    s = _element_span(knots, e, n)
    vals = {s: np.ones_like(x)}
    for d in range(1, q + 1):
        new = {}
        for i in range(s - d, s + 1):
            acc = np.zeros_like(x)
            den1 = knots[i + d] - knots[i]
            if i in vals and den1 != 0.0:
                acc = acc + (x - knots[i]) / den1 * vals[i]
            den2 = knots[i + d + 1] - knots[i + 1]
            if (i + 1) in vals and den2 != 0.0:
                acc = acc + (knots[i + d + 1] - x) / den2 * vals[i + 1]
            new[i] = acc
        vals = new
    return vals


def _n_elements(knots: np.ndarray, p: int) -> int:
    """Number of (uniform) elements of a knot vector built by open_knots."""
    return len(np.unique(knots)) - 1


def bspline_derivs(knots: np.ndarray, p: int, e: int, x: np.ndarray, k: int) -> np.ndarray:
    """k-th derivative of the p+1 B-splines nonzero on element e, at points x
    of the element: B_{p,s-p}, ..., B_{p,s} with s the element's span (s = p + e
    without repeated knots).

    Returns an array of shape (len(x), p+1); column j is B_{p,s-p+j}^{(k)}.
    For k > p all derivatives vanish.
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.zeros((x.size, p + 1))
    if k > p:
        return out
    n = _n_elements(knots, p)
    s = _element_span(knots, e, n)
    cur = bspline_table(knots, p - k, e, x, p, n)  # degree p-k values
    for d in range(p - k + 1, p + 1):
        new = {}
        for i in range(s - d, s + 1):
            acc = np.zeros_like(x)
            den1 = knots[i + d] - knots[i]
            if i in cur and den1 != 0.0:
                acc = acc + d * cur[i] / den1
            den2 = knots[i + d + 1] - knots[i + 1]
            if (i + 1) in cur and den2 != 0.0:
                acc = acc - d * cur[i + 1] / den2
            new[i] = acc
        cur = new
    for j in range(p + 1):
        out[:, j] = cur.get(s - p + j, np.zeros_like(x))
    return out


def gauss_rule(npts: int, a: float, b: float):
    """Gauss-Legendre nodes and weights on [a, b] (library nodes on [-1, 1])."""
    t, w = np.polynomial.legendre.leggauss(npts)
    return 0.5 * (b - a) * t + 0.5 * (a + b), 0.5 * (b - a) * w


def assemble_full(n: int, p: int, weight=None, nq: int | None = None, rep=None):
    """Full mass and stiffness matrices of S_{p,h} (n + p B-splines, plus one
    per repeated knot of ``rep``).

    M_ij = int_0^1 a(x) B_i(x) B_j(x) dx,  K_ij = int_0^1 a(x) B_i'(x) B_j'(x) dx,
    with a = 1 unless ``weight`` is given, integrated element by element with
    an nq-point Gauss rule (nq = p+1 by default).
    """
    knots = open_knots(n, p, rep)
    nq = p + 1 if nq is None else nq
    size = n_basis(n, p, rep)
    M = np.zeros((size, size))
    K = np.zeros((size, size))
    for e in range(n):
        xg, wg = gauss_rule(nq, e / n, (e + 1) / n)
        if weight is not None:
            wg = wg * weight(xg)
        B = bspline_derivs(knots, p, e, xg, 0)
        dB = bspline_derivs(knots, p, e, xg, 1)
        s0 = _element_span(knots, e, n) - p
        M[s0:s0 + p + 1, s0:s0 + p + 1] += B.T @ (wg[:, None] * B)
        K[s0:s0 + p + 1, s0:s0 + p + 1] += dB.T @ (wg[:, None] * dB)
    return M, K


def kept_indices(n: int, p: int, dirichlet=(0, 1), rep=None) -> np.ndarray:
    """Indices of the B-splines kept in S_{p,h,D}: the first is dropped when 0
    is in D and the last when 1 is in D (the only ones that do not vanish there)."""
    size = n_basis(n, p, rep)
    idx = list(range(size))
    if 1 in dirichlet:
        idx.remove(size - 1)
    if 0 in dirichlet:
        idx.remove(0)
    return np.array(idx, dtype=np.int64)


def mass_stiffness(n: int, p: int, dirichlet=(0, 1), weight=None, rep=None):
    """M and K of S_{p,h,D} (size m = n + p - |D|, plus the repeated knots)."""
    M, K = assemble_full(n, p, weight, rep=rep)
    keep = kept_indices(n, p, dirichlet, rep)
    return M[np.ix_(keep, keep)], K[np.ix_(keep, keep)]


def cardinal_bspline(p: int, x) -> np.ndarray:
    """Symmetric cardinal B-spline of degree p (Lemma 3, eq. "cardinal").

    B~_0 is the indicator of [-1/2, 1/2); for q >= 1
    B~_q(x) = (q+1+2x)/(2q) B~_{q-1}(x+1/2) + (q+1-2x)/(2q) B~_{q-1}(x-1/2).
    The recursion is evaluated with memoisation on the (degree, shift) pairs.
    """
    x = np.asarray(x, dtype=np.float64)
    memo: dict = {}

    def rec(q: int, shift: Fraction) -> np.ndarray:
        key = (q, shift)
        if key in memo:
            return memo[key]
        y = x + float(shift)
        if q == 0:
            val = ((y >= -0.5) & (y < 0.5)).astype(np.float64)
        else:
            val = ((q + 1 + 2 * y) / (2 * q)) * rec(q - 1, shift + Fraction(1, 2)) \
                + ((q + 1 - 2 * y) / (2 * q)) * rec(q - 1, shift - Fraction(1, 2))
        memo[key] = val
        return val

    return rec(p, Fraction(0))
