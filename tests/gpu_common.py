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
