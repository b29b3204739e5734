"""Tensor operators, PCG and spectral estimates (Sections 3, 4, 7) -- oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Array convention: a d-dimensional coefficient array is a numpy array of shape
(m_d, ..., m_2, m_1) in C order, so the first parametric direction x_1 is the
fastest index, as in the lexicographic basis of eq. "tp-B-basis". Direction k
(1-based, paper order) is numpy axis -k. Per-direction data is passed as a list
in paper order [direction 1, direction 2, ...].
"""

from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg


def apply_along(A, u: np.ndarray, direction: int) -> np.ndarray:
    """(I x .. x A x .. x I) u: multiply every pencil along ``direction``
    (1-based, paper order) by the matrix A (dense, or scipy.sparse)."""
    ax = u.ndim - direction
    if scipy.sparse.issparse(A):
        v = np.moveaxis(u, ax, 0)
        w = (A @ v.reshape(v.shape[0], -1)).reshape((A.shape[0],) + v.shape[1:])
        return np.moveaxis(w, 0, ax)
    return np.moveaxis(np.tensordot(A, u, axes=([1], [ax])), 0, ax)


def kron_apply(mats, u: np.ndarray) -> np.ndarray:
    """(A_d x ... x A_1) u for per-direction matrices mats = [A_1, ..., A_d]."""
    for k, A in enumerate(mats, start=1):
        u = apply_along(A, u, k)
    return u


# ------------------------------------------------------------ stiffness
def stiffness_apply(u: np.ndarray, MK) -> np.ndarray:
    """A^ u with A^ = sum_k (M_d x .. x K_k x .. x M_1) (eq. "system_matrix",
    written for d directions). MK = [(M_1, K_1), ..., (M_d, K_d)]."""
    d = u.ndim
    out = np.zeros_like(u)
    for k in range(1, d + 1):
        mats = [MK[j][1] if j + 1 == k else MK[j][0] for j in range(d)]
        out += kron_apply(mats, u)
    return out


def varcoef_stiffness_apply(u: np.ndarray, MK, MKs, c: float = 0.5) -> np.ndarray:
    """Stiffness of -div(a grad u) with a = 1 + c s_1(x_1) ... s_d(x_d).

    With the tensor (p+1)-point Gauss rule the integral of a grad u . grad v
    factorises exactly into A^ + c sum_k (M^s_d x .. x K^s_k x .. x M^s_1), where
    M^s, K^s are the 1D mass/stiffness matrices weighted by s (computed with the
    same per-element Gauss rule). MKs = [(M^s_1, K^s_1), ...]."""
    return stiffness_apply(u, MK) + c * stiffness_apply(u, MKs)


def dense_stiffness(MK) -> np.ndarray:
    """Assembled A^ for tiny grids (row index with x_1 fastest)."""
    d = len(MK)
    N = int(np.prod([M.shape[0] for M, _ in MK]))
    A = np.zeros((N, N))
    for k in range(d):
        term = np.ones((1, 1))
        for j in reversed(range(d)):      # slowest direction first
            term = np.kron(term, MK[j][1] if j == k else MK[j][0])
        A += term
    return A


# ------------------------------------------------- FD-type preconditioners
def diag_precond_apply(r: np.ndarray, Qs, lams) -> np.ndarray:
    """(Q_d x .. x Q_1) (sum_k Lambda_k)^{-1} (Q_d^T x .. x Q_1^T) r
    (eqs. "exact_diagonalization" and "preconditioner")."""
    d = r.ndim
    t = kron_apply([Q.T for Q in Qs], r)
    denom = np.zeros(t.shape)
    for k in range(1, d + 1):
        shape = [1] * d
        shape[d - k] = lams[k - 1].size
        denom = denom + lams[k - 1].reshape(shape)
    return kron_apply(Qs, t / denom)


def iffd_apply(r: np.ndarray, splits) -> np.ndarray:
    """IFFD preconditioner P^{-1} r with Q~, Lambda~ of each direction."""
    return diag_precond_apply(r, [s.Qt for s in splits], [s.lamt for s in splits])


def exact_fd_eig(M: np.ndarray, K: np.ndarray):
    """Generalized eigendecomposition K q = lambda M q, Q^T M Q = I
    (eq. "eigendecomposition"); scipy's symmetric-definite solver."""
    lam, Q = scipy.linalg.eigh(K, M)
    return Q, lam


def exact_fd_apply(r: np.ndarray, eigs) -> np.ndarray:
    """A^{-1} r by exact Fast Diagonalization; eigs = [(Q_1, lam_1), ...]."""
    return diag_precond_apply(r, [Q for Q, _ in eigs], [lam for _, lam in eigs])


# ------------------------------------------------------------------ PCG
def pcg(f: np.ndarray, apply_A, apply_P, rtol: float = 1e-8, maxit: int = 500):
    """Textbook preconditioned CG (Section 3) with zero initial guess.

    Stops at the first iterate with ||r_k||_2 <= rtol ||f||_2, r_k the
    recurrence residual; the iteration count is the number of products with A.
    Returns (u, iterations, relative residual history)."""
    u = np.zeros_like(f)
    r = f.copy()
    fnorm = np.linalg.norm(f.ravel())
    hist = [1.0]
    if fnorm == 0.0:
        return u, 0, hist
    z = apply_P(r)
    p = z.copy()
    rz = float(np.vdot(r, z))
    for it in range(1, maxit + 1):
        q = apply_A(p)
        alpha = rz / float(np.vdot(p, q))
        u += alpha * p
        r -= alpha * q
        rel = np.linalg.norm(r.ravel()) / fnorm
        hist.append(rel)
        if rel <= rtol:
            return u, it, hist
        z = apply_P(r)
        rz_new = float(np.vdot(r, z))
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return u, maxit, hist


# ------------------------------------------------------ spectral estimates
def kappa_dense(A: np.ndarray, Pinv: np.ndarray) -> float:
    """kappa(P^{-1} A) = lambda_max / lambda_min of the pencil (A, P)."""
    P = np.linalg.inv(Pinv)
    P = 0.5 * (P + P.T)
    ev = scipy.linalg.eigh(A, P, eigvals_only=True)
    return float(ev[-1] / ev[0])


def kappa_lanczos(splits, shape, apply_A, k: int = 60) -> float:
    """kappa(P^{-1} A^) for the IFFD preconditioner by Lanczos (scipy eigsh,
    implicitly restarted) on the symmetric operator
    S = Sigma^{-1/2} W^T A^ W Sigma^{-1/2}, W = (Q~_d x .. x Q~_1), which is
    similar to P^{-1} A^ because P^{-1} = W Sigma^{-1} W^T."""
    d = len(shape)
    Qs = [s.Qt for s in splits]
    denom = np.zeros(shape)
    for kk in range(1, d + 1):
        sh = [1] * d
        sh[d - kk] = splits[kk - 1].lamt.size
        denom = denom + splits[kk - 1].lamt.reshape(sh)
    isq = 1.0 / np.sqrt(denom)
    N = int(np.prod(shape))

    def mv(v):
        x = v.reshape(shape) * isq
        y = apply_A(kron_apply(Qs, x))
        return (kron_apply([Q.T for Q in Qs], y) * isq).ravel()

    op = scipy.sparse.linalg.LinearOperator((N, N), matvec=mv, dtype=np.float64)
    rng = np.random.default_rng(12345)
    v0 = rng.standard_normal(N)
    lmax = scipy.sparse.linalg.eigsh(op, k=1, which="LA", v0=v0, ncv=k,
                                     return_eigenvectors=False, tol=1e-10)[0]
    lmin = scipy.sparse.linalg.eigsh(op, k=1, which="SA", v0=v0, ncv=k,
                                     return_eigenvectors=False, tol=1e-10)[0]
    return float(lmax / lmin)


def prop1_bound(K: np.ndarray, Ktilde: np.ndarray) -> float:
    """max_k C_k / c_k of Proposition 1 for one direction: the extreme
    generalized eigenvalues of (K, K~)."""
    ev = scipy.linalg.eigh(K, 0.5 * (Ktilde + Ktilde.T), eigvals_only=True)
    return float(ev[-1] / ev[0])
