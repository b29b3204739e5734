"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

Holds no arithmetic of the method: only the workload shapes and the random
right-hand sides (numpy ``default_rng(seed)``, drawn in x-fastest order, i.e.
C order of an array of shape (m_d, ..., m_1)). The paper's experiments use
random right-hand sides on the unit square / cube (Section 7); these configs
are the synthetic stand-ins.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    d: int
    n: int
    p: int
    dist: str   # "uniform" -> U[-1, 1], "normal" -> N(0, 1)
    seed: int

    @property
    def m(self) -> int:
        return self.n + self.p - 2

    @property
    def shape(self):
        return (self.m,) * self.d

    @property
    def N(self) -> int:
        return self.m ** self.d


# 2D, n = 64, p = 3: 65^2 = 4225 DoFs, f ~ U[-1, 1], seed 0
SQUARE_N64_P3 = Workload("square_n64_p3", 2, 64, 3, "uniform", 0)
# 3D, n = 256, p = 4: 258^3 = 17,173,512 DoFs, f ~ N(0, 1), seed 1
CUBE_N256_P4 = Workload("cube_n256_p4", 3, 256, 4, "normal", 1)
# its 64^3 subcase: n = 64, p = 4, 66^3 = 287,496 DoFs
CUBE_N64_P4 = Workload("cube_n64_p4", 3, 64, 4, "normal", 1)
# 3D, n = 384, p = 8: 390^3 = 59,319,000 DoFs, f ~ U[-1, 1], seed 2
CUBE_N384_P8 = Workload("cube_n384_p8", 3, 384, 8, "uniform", 2)


def rhs(shape, dist: str = "normal", seed: int = 0) -> np.ndarray:
    """Random right-hand side of the given array shape (float64, C order)."""
    rng = np.random.default_rng(seed)
    N = int(np.prod(shape))
    if dist == "uniform":
        v = rng.uniform(-1.0, 1.0, N)
    elif dist == "normal":
        v = rng.standard_normal(N)
    else:
        raise ValueError(dist)
    return v.reshape(shape)


def workload_rhs(w: Workload) -> np.ndarray:
    return rhs(w.shape, w.dist, w.seed)


# ---------------------------------------------------------------- batched
BATCH_N = (16, 24, 32, 48, 64, 96, 128)
BATCH_P = (2, 3, 4, 5, 6)


def batched_problems(count: int = 512, seed: int = 3):
    """512 independent 3D Dirichlet problems: n uniform in BATCH_N, p uniform in
    BATCH_P (seed 3); one right-hand side each, eight for the n = 64 problems.
    Returns [(d, n, p, nrhs), ...]."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(BATCH_N, count)
    ps = rng.choice(BATCH_P, count)
    return [(3, int(n), int(p), 8 if int(n) == 64 else 1) for n, p in zip(ns, ps)]


def device_rhs(N: int, seed: int, dist: str = "normal"):
    """Seeded right-hand side generated directly on the current CUDA device
    (torch generator), for workloads too large to draw on the host."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(int(seed))
    if dist == "normal":
        return torch.randn(N, generator=g, dtype=torch.float64, device="cuda")
    return torch.rand(N, generator=g, dtype=torch.float64, device="cuda") * 2.0 - 1.0


# ---------------------------------------------------------------- serving
@dataclass(frozen=True)
class Request:
    index: int
    t: float  # arrival time (s)
    d: int
    n: int
    p: int

    @property
    def N(self) -> int:
        return (self.n + self.p - 2) ** self.d


def serving_requests(rate: float = 2000.0, duration: float = 60.0, seed: int = 4):
    """Poisson arrivals at `rate` req/s over `duration` s (seed 4). Each request
    is 2D or 3D with equal probability; n uniform in 128..2048 (2D) or 32..256
    (3D); p uniform in 2..8."""
    rng = np.random.default_rng(seed)
    out, t, k = [], 0.0, 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            return out
        d = int(rng.integers(2, 4))
        n = int(rng.integers(128, 2049)) if d == 2 else int(rng.integers(32, 257))
        p = int(rng.integers(2, 9))
        out.append(Request(k, t, d, n, p))
        k += 1
