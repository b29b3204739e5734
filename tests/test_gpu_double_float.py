"""GPU parity of the double-float transform passes: the FP64 IFFD
preconditioner of eq. "preconditioner" with every transform step in
double-float arithmetic (pairs of float32 values, about 48 significant bits)
on the FP32 pipe. It must meet the FP64 contract: 1e-12 relative (max-norm
and 2-norm) against the oracle's dense Q~ apply, on DST-II/III (even p) and
DST-I (odd p) directions of FFT length 64, 128 and 256, 2D and 3D, unequal
directions, ragged last tiles, inputs with zeros and with magnitudes far from
1; agree with the FP64-pipe kernels to rounding; and give PCG solves with the
oracle's iteration count +-1 and true residual <= 1.1e-8."""

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import oracle_pcg, oracle_precond, oracle_split, oracle_stiffness, rel_max_err, require_gpu

pytestmark = pytest.mark.gpu

# (d, n per direction, p): even p -> DST-II/III of length n; odd p -> DST-I of length 2n
SHAPES = [
    (3, 64, 4),      # 66^3, length 64
    (3, 32, 3),      # DST-I, length 64
    (2, 128, 6),     # length 128, n_out = 4
    (2, 64, 5),      # DST-I, length 128
    (3, 64, 7),      # DST-I, length 128, n_out = 6
    (2, 256, 8),     # length 256, p = 8
    (3, 128, 2),     # p = 2: no remainder space
    (2, 128, 3),     # DST-I, length 256
    # no warp-FFT length: the double-float block kernel
    (3, 96, 4),      # DST-II/III, length 96 = 2^5 3
    (2, 96, 3),      # DST-I, length 192
    (3, 40, 6),      # length 40 = 2^3 5, n_out = 4
    (2, 80, 5),      # DST-I, length 160
    (3, 48, 4),      # length 48
    (2, 56, 4),      # length 56 = 8 7: a direct-DFT stage of radix 7
    (2, 100, 6),     # length 100 = 4 25: radix-5 stages
]


def _gpu(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("d,n,p", SHAPES)
def test_double_float_preconditioner_matches_oracle(d, n, p):
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(d, n, p).set_geometry(0, double_float=True)  # small grids default to the FP64 kernel
    assert all(plan.tiles(a)["double_float"] for a in range(d))
    r = inputs.rhs(plan.shape, "normal", seed=800 + n + p)
    rg = _gpu(torch, r)
    z = plan.apply_preconditioner(rg).cpu().numpy()
    zo = oracle_precond(r, n, p)
    assert rel_max_err(z, zo) <= 1e-12
    assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)
    # the FP64-pipe block kernel: the same operator to rounding
    fp64 = IFFDPlan(d, n, p)
    for a in range(d):
        fp64.set_geometry(a, pipelined=False)
    assert not any(fp64.tiles(a)["double_float"] for a in range(d))
    zb = fp64.apply_preconditioner(rg).cpu().numpy()
    assert rel_max_err(z, zb) <= 1e-13


def test_double_float_unequal_directions_and_ragged_tiles():
    torch = require_gpu()
    from oracle import operators
    from paper_2512_20269_gb300 import IFFDPlan
    ns = (64, 128, 256)  # p = 4: lengths 64, 128, 256; 130 x 66 x 258 pencils leave ragged tiles
    plan = IFFDPlan(3, list(ns), 4).set_geometry(0, double_float=True)
    assert all(plan.tiles(a)["double_float"] for a in range(3))
    r = inputs.rhs(plan.shape, "uniform", seed=810)
    z = plan.apply_preconditioner(_gpu(torch, r)).cpu().numpy()
    zo = operators.iffd_apply(r, [oracle_split(n, 4) for n in ns])
    assert rel_max_err(z, zo) <= 1e-12


def test_double_float_warp_and_block_directions():
    """One plan whose directions mix the warp-FFT pass (length 64, 128) and
    the block kernel (length 96): the FP64 tolerance, and PCG."""
    torch = require_gpu()
    from oracle import operators
    from paper_2512_20269_gb300 import IFFDPlan
    ns = (64, 96, 128)
    plan = IFFDPlan(3, list(ns), 4).set_geometry(0, double_float=True)
    assert all(plan.tiles(a)["double_float"] for a in range(3))
    assert 3 in plan.tiles(1)["radices"]  # the block kernel's radix sequence
    r = inputs.rhs(plan.shape, "normal", seed=840)
    z = plan.apply_preconditioner(_gpu(torch, r)).cpu().numpy()
    zo = operators.iffd_apply(r, [oracle_split(n, 4) for n in ns])
    assert rel_max_err(z, zo) <= 1e-12
    f = inputs.rhs(plan.shape, "uniform", seed=841)
    _, info = plan.pcg_solve(_gpu(torch, f))
    assert info["status"] == 0 and info["true_rel_res"] <= 1.1e-8


@pytest.mark.parametrize("scale", [1e-25, 1e25, 0.0])
def test_double_float_zeros_and_far_magnitudes(scale):
    """Exact zeros, and magnitudes that take the conversion's FP64 route
    (1e-25) or sit far above 1 (1e25), keep the FP64 accuracy."""
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    n, p = 64, 4
    plan = IFFDPlan(3, n, p).set_geometry(0, double_float=True)
    r = inputs.rhs(plan.shape, "normal", seed=820)
    r[::3] = 0.0  # zeros inside every pencil
    if scale:
        r = r * scale
    else:
        r[1::3] *= 1e-30  # tiny next to O(1) values
    z = plan.apply_preconditioner(_gpu(torch, r)).cpu().numpy()
    zo = oracle_precond(r, n, p)
    assert rel_max_err(z, zo) <= 1e-12


@pytest.mark.parametrize("d,n,p", [(3, 64, 4), (2, 128, 3), (3, 32, 5)])
def test_double_float_pcg(d, n, p):
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(d, n, p).set_geometry(0, double_float=True)
    f = inputs.rhs(plan.shape, "uniform", seed=830 + n)
    u, info = plan.pcg_solve(_gpu(torch, f))
    uh = u.cpu().numpy()
    assert info["status"] == 0
    res = np.linalg.norm(f - oracle_stiffness(uh, n, p)) / np.linalg.norm(f)
    assert res <= 1.1e-8 and abs(res - info["true_rel_res"]) <= 1e-6 * res + 1e-13
    _, it_or, _ = oracle_pcg(f, n, p)
    assert abs(info["iters"] - it_or) <= 1


def test_double_float_switch():
    require_gpu()
    from paper_2512_20269_gb300 import IFFDError, IFFDPlan
    plan = IFFDPlan(3, 64, 4)
    plan.set_geometry(1, pencils_transform=8)  # an FP64-pipe geometry by hand: double-float off
    assert not plan.tiles(0)["double_float"] and plan.tiles(1)["pencils_transform"] == 8
    plan.set_geometry(0, double_float=True)
    assert all(plan.tiles(a)["double_float"] for a in range(3))
    t = plan.tiles(2)
    assert t["pencils_transform"] == 64 and t["radices"] == [8, 8]
    IFFDPlan(3, 40, 4).set_geometry(0, double_float=True)        # length 40: the double-float block kernel
    with pytest.raises(IFFDError):
        IFFDPlan(2, 67, 4).set_geometry(0, double_float=True)     # length 67 (prime): Bluestein, FP64 only
    with pytest.raises(IFFDError):
        IFFDPlan(3, 64, 4, precision="fp32").set_geometry(0, double_float=True)
    assert not any(IFFDPlan(3, 64, 4, precision="fp32").tiles(a)["double_float"] for a in range(3))
    t96 = IFFDPlan(3, 96, 4).tiles(0)                              # length 96: double-float block kernel
    assert t96["double_float"] and 3 in t96["radices"]
    # the default: double-float where the warp tiles fill the GPU (130^3: 16,900 / 32 pencils
    # per tile >= SMs), the FP64 block kernel with narrowed tiles on small grids
    assert all(IFFDPlan(3, 128, 4).tiles(a)["double_float"] for a in range(3))
    small = IFFDPlan(2, 64, 3)
    assert not small.tiles(0)["double_float"] and small.tiles(0)["pencils_transform"] == 2
