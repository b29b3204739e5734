"""Stiffness with a general (non-separable, possibly anisotropic) diffusion
coefficient, sampled at the Gauss points -- oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Model problem of Section 2 with the coefficient moved inside the integral,
-div(C(x) grad u) = f on [0,1]^d: the Galerkin matrix on S_{p,h,D} is
A_ij = int grad B_i . C grad B_j dx. On a geometry F the pulled-back problem
on the parameter domain has exactly this form with C = det(DF) DF^{-1} DF^{-T}
(Section 7), so a symmetric C(x) sampled at the quadrature points stands for
both a variable coefficient and a map. The IFFD preconditioner stays the one of
the parametric Laplacian (A^ of eq. "system_matrix"), and PCG with it solves
A u = f.

Plain definition, with the tensor (p+1)-point Gauss rule of every element (the
rule of Section 2): let B_k and D_k be the values and the first derivatives of
the kept B-splines of direction k at the n (p+1) Gauss points of that
direction (a matrix with n (p+1) rows and m_k columns), w_k the Gauss weights,
and G_k = E_d x ... x E_1 with E_j = D_j for j = k and B_j otherwise (the
k-th partial derivative at every tensor Gauss point). Then

    A = sum_{k,l} G_k^T diag(w C_kl) G_l,   w = w_d x ... x w_1.

Coefficient arrays have shape (ncomp, nq_d, ..., nq_1) (x_1 fastest, as the
data): ncomp = 1 is a scalar a(x) (C = a I); otherwise the upper triangle of
the symmetric C row by row: (11, 12, 22) in 2D, (11, 12, 13, 22, 23, 33) in 3D.
"""

from __future__ import annotations

import numpy as np

from . import splines
from .operators import kron_apply


def quad_axis(n: int, p: int, dirichlet=(0, 1), rep=None):
    """Gauss points x, weights w, and the matrices B (values) and D (first
    derivatives) of the kept B-splines of S_{p,h,D} at those points; element
    e owns rows e (p+1) .. e (p+1) + p."""
    knots = splines.open_knots(n, p, rep)
    size = splines.n_basis(n, p, rep)
    keep = splines.kept_indices(n, p, dirichlet, rep)
    nq = n * (p + 1)
    B = np.zeros((nq, size))
    D = np.zeros((nq, size))
    xs, ws = [], []
    for e in range(n):
        xg, wg = splines.gauss_rule(p + 1, e / n, (e + 1) / n)
        s0 = splines._element_span(knots, e, n) - p
        rows = slice(e * (p + 1), (e + 1) * (p + 1))
        B[rows, s0:s0 + p + 1] = splines.bspline_derivs(knots, p, e, xg, 0)
        D[rows, s0:s0 + p + 1] = splines.bspline_derivs(knots, p, e, xg, 1)
        xs.append(xg)
        ws.append(wg)
    return np.concatenate(xs), np.concatenate(ws), B[:, keep], D[:, keep]


def component(C: np.ndarray, d: int, k: int, l: int):
    """C_kl (0-based directions) from the packed coefficient array."""
    if C.shape[0] == 1:
        return C[0] if k == l else 0.0
    a, b = min(k, l), max(k, l)
    idx = [(i, j) for i in range(d) for j in range(i, d)].index((a, b))
    return C[idx]


def weights(axes) -> np.ndarray:
    """w_d x ... x w_1 as an array of shape (nq_d, ..., nq_1)."""
    w = np.ones(())
    for ax in axes:  # direction 1 first: it becomes the last (fastest) axis
        w = np.multiply.outer(ax[1], w)
    return w


def general_stiffness_apply(u: np.ndarray, axes, C: np.ndarray) -> np.ndarray:
    """A u for the definition above. axes = [quad_axis(...) of direction 1, ...,
    of direction d]; C has shape (ncomp, nq_d, ..., nq_1)."""
    d = u.ndim
    G = [kron_apply([axes[j][3] if j == k else axes[j][2] for j in range(d)], u) for k in range(d)]
    w = weights(axes)
    out = np.zeros_like(u)
    for k in range(d):
        h = np.zeros_like(G[0])
        for l in range(d):
            h = h + component(C, d, k, l) * G[l]
        out += kron_apply([axes[j][3].T if j == k else axes[j][2].T for j in range(d)], w * h)
    return out


def general_stiffness_dense(axes, C: np.ndarray) -> np.ndarray:
    """The matrix A itself (tiny grids), column by column of the identity."""
    shape = tuple(ax[2].shape[1] for ax in reversed(axes))
    N = int(np.prod(shape))
    A = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        A[:, j] = general_stiffness_apply(e.reshape(shape), axes, C).ravel()
    return A
