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
