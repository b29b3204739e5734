"""Shared helpers of the GPU parity tests: build/load the library, run the oracle
on the same seeded inputs."""

import functools
import os

import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_20269_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2512_20269_gb300 import build
        build.build()
    return torch


@functools.lru_cache(maxsize=None)
def oracle_split(n, p):
    from oracle import splitting
    return splitting.axis_split(n, p, (0, 1))


@functools.lru_cache(maxsize=None)
def oracle_sparse_mk(n, p):
    import scipy.sparse
    s = oracle_split(n, p)
    return scipy.sparse.csr_matrix(s.M), scipy.sparse.csr_matrix(s.K)


@functools.lru_cache(maxsize=None)
def oracle_fd_eig(n, p):
    from oracle import operators
    s = oracle_split(n, p)
    return operators.exact_fd_eig(s.M, s.K)


def oracle_precond(r: np.ndarray, n: int, p: int) -> np.ndarray:
    from oracle import operators
    return operators.iffd_apply(r, [oracle_split(n, p)] * r.ndim)


def oracle_exact_fd(r: np.ndarray, n: int, p: int) -> np.ndarray:
    from oracle import operators
    return operators.exact_fd_apply(r, [oracle_fd_eig(n, p)] * r.ndim)


def oracle_stiffness(u: np.ndarray, n: int, p: int) -> np.ndarray:
    from oracle import operators
    return operators.stiffness_apply(u, [oracle_sparse_mk(n, p)] * u.ndim)


def oracle_pcg(f: np.ndarray, n: int, p: int, rtol=1e-8):
    from oracle import operators
    d = f.ndim
    return operators.pcg(f, lambda v: oracle_stiffness(v, n, p), lambda r: oracle_precond(r, n, p), rtol=rtol)


def rel_max_err(a: np.ndarray, b: np.ndarray) -> float:
    """max |a - b| / max |b| (elementwise, normalised by the reference's scale)."""
    return float(np.abs(a - b).max() / np.abs(b).max())


@functools.lru_cache(maxsize=None)
def oracle_sin_mk(n, p):
    """1D mass/stiffness weighted by s(x) = sin(2 pi x) (same Gauss rule)."""
    import scipy.sparse
    from oracle import splines
    Ms, Ks = splines.mass_stiffness(n, p, (0, 1), weight=lambda x: np.sin(2 * np.pi * x))
    return scipy.sparse.csr_matrix(Ms), scipy.sparse.csr_matrix(Ks)


def oracle_varcoef_stiffness(u: np.ndarray, n: int, p: int, c: float = 0.5) -> np.ndarray:
    from oracle import operators
    d = u.ndim
    return operators.varcoef_stiffness_apply(u, [oracle_sparse_mk(n, p)] * d, [oracle_sin_mk(n, p)] * d, c)


def oracle_varcoef_sampled(u: np.ndarray, n: int, p: int, points, c: float = 0.5):
    """(A_a u) at the given 3D points (k, j, i), each computed from its local
    (2p+1)^3 neighbourhood with the oracle's 1D matrices (same Kronecker form)."""
    M, K = (a.toarray() for a in oracle_sparse_mk(n, p))
    Ms, Ks = (a.toarray() for a in oracle_sin_mk(n, p))
    m = M.shape[0]
    out = []
    for (k, j, i) in points:
        ks = slice(max(0, k - p), min(m, k + p + 1))
        js = slice(max(0, j - p), min(m, j + p + 1))
        is_ = slice(max(0, i - p), min(m, i + p + 1))
        loc = u[ks, js, is_]

        def term(Az, Ay, Ax):
            return np.einsum("a,b,c,abc->", Az[k, ks], Ay[j, js], Ax[i, is_], loc)

        v = term(M, M, K) + term(M, K, M) + term(K, M, M)
        v += c * (term(Ms, Ms, Ks) + term(Ms, Ks, Ms) + term(Ks, Ms, Ms))
        out.append(v)
    return np.array(out)
