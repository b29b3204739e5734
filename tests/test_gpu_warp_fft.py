"""GPU parity of the warp-FFT transform pass (Dirichlet at both ends, FFT
length 64, 128, 256, 512: DST-II/III for even p with n_reg of that length,
DST-I for odd p with 2 (n_reg + 1) = 2 n): each pencil pair is transformed by
the lanes of one warp. FP32 (the default where eligible) is compared with the
oracle (tolerance 1e-5) and with the block kernel on the same plan (same
operator, different FP32 rounding); FP64 (opt-in, lengths up to 256) with the
oracle at 1e-12 and with the FP64 block kernel."""

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


def _gpu(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# (d, n per direction, p, knots): every warp length, 2D and 3D, ragged last
# tiles, directions that do not qualify next to ones that do (n = 40, 37, 30,
# 24), repeated knots (interior blocks in V_reg)
CASES = [
    (2, (64, 64), 4, None), (2, (128, 40), 2, None), (3, (64, 64, 64), 4, None), (3, (256, 37, 20), 6, None),
    (2, (512, 24), 4, None), (3, (128, 64, 30), 8, None), (2, (64, 128), 4, ({32: 1}, {20: 2, 100: 1})),
    (2, (64, 128), 6, ({1: 1}, {126: 3})),
    # DST-I (odd p): n = 32, 64, 128, 256
    (2, (32, 64), 3, None), (3, (128, 40, 64), 5, None), (2, (256, 24), 7, None), (2, (64, 48), 3, ({20: 2}, None)),
]


def _warp_len(n, p):
    L = n if p % 2 == 0 else 2 * n
    return L if L in (64, 128, 256, 512) else 0


@pytest.mark.parametrize("d,ns,p,knots", CASES)
def test_warp_pass_matches_oracle_and_block_kernel(d, ns, p, knots):
    torch = require_gpu()
    from oracle import operators, splitting
    from paper_2512_20269_gb300 import IFFDPlan
    kw = {} if knots is None else {"knots": list(knots)}
    plan = IFFDPlan(d, list(ns), p, precision="fp32", **kw)
    warp_axes = [a for a in range(d) if _warp_len(ns[a], p)]
    for a in warp_axes:
        plan.set_geometry(a, warp=True)
    for a in range(d):
        assert plan.tiles(a)["warp"] == (a in warp_axes)
    block = IFFDPlan(d, list(ns), p, precision="fp32", **kw)
    for a in range(d):
        block.set_geometry(a, pencils_transform=8)
        assert not block.tiles(a)["warp"]
    r = inputs.rhs(plan.shape, "normal", seed=900 + sum(ns) + p)
    rg = _gpu(torch, r)
    sp = [splitting.axis_split(n, p, (0, 1), rep=(knots[a] if knots else None)) for a, n in enumerate(ns)]
    zo = operators.iffd_apply(r, sp)
    z = plan.apply_preconditioner(rg).cpu().numpy()
    zb = block.apply_preconditioner(rg).cpu().numpy()
    assert _rel(z, zo) <= 1e-5
    assert _rel(zb, zo) <= 1e-5
    assert _rel(z, zb) <= 1e-5
    # deterministic: the same call gives the same bits
    assert np.array_equal(plan.apply_preconditioner(rg).cpu().numpy(), z)


def test_warp_pass_pcg():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    f = _gpu(torch, inputs.rhs((130, 130, 66), "normal", seed=5))
    _, i64 = IFFDPlan(3, (64, 128, 128), 4).pcg_solve(f)
    plan = IFFDPlan(3, (64, 128, 128), 4, precision="fp32")
    assert all(plan.tiles(a)["warp"] for a in range(3))
    _, i32 = plan.pcg_solve(f)
    assert i32["status"] == 0 and i32["true_rel_res"] <= 1.1e-8
    assert i32["iters"] <= i64["iters"] + 2


def test_warp_pass_default_fills_the_gpu():
    """The warp-FFT pass is the default where its tiles (16 to 64 pencils)
    still fill the GPU, or where the block kernel's would not either."""
    require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    assert all(IFFDPlan(3, 128, 4, precision="fp32").tiles(a)["warp"] for a in range(3))  # 529 tiles
    assert not any(IFFDPlan(3, 64, 4, precision="fp32").tiles(a)["warp"] for a in range(3))  # 68 tiles
    assert IFFDPlan(2, 512, 4, precision="fp32").tiles(0)["warp"]  # 33 tiles, block kernel 65


def test_warp_geometry_switches():
    require_gpu()
    from paper_2512_20269_gb300 import IFFDError, IFFDPlan
    plan = IFFDPlan(2, (64, 40), 4, precision="fp32")
    assert plan.tiles(0)["warp"] and not plan.tiles(1)["warp"]
    assert not plan.tiles(0)["paired"] and plan.tiles(0)["pencils_transform"] == 64
    assert IFFDPlan(2, (40, 64), 4, precision="fp32").tiles(1)["paired"]  # the last (fused) direction: paired
    plan.set_geometry(0, pencils_transform=4)
    assert not plan.tiles(0)["warp"] and plan.tiles(0)["pencils_transform"] == 4
    plan.set_geometry(0, warp=True)
    assert plan.tiles(0)["warp"] and not plan.tiles(0)["paired"] and plan.tiles(0)["pencils_transform"] == 64
    plan.set_geometry(0, paired=True)
    assert plan.tiles(0)["paired"] and plan.tiles(0)["pencils_transform"] == 128
    with pytest.raises(IFFDError):
        IFFDPlan(2, 512, 4, precision="fp32").set_geometry(0, paired=True)  # length 512: unpaired only
    with pytest.raises(IFFDError):
        IFFDPlan(2, 64, 4).set_geometry(0, paired=True)  # FP64 plan
    with pytest.raises(IFFDError):
        plan.set_geometry(1, warp=True)  # n_reg = 40
    with pytest.raises(IFFDError):
        IFFDPlan(2, 512, 4).set_geometry(0, warp=True)  # FP64 plan, length 512
    with pytest.raises(IFFDError):
        IFFDPlan(2, 40, 3, precision="fp32").set_geometry(0, warp=True)  # DST-I of length 80



# FP64 warp-FFT pass (opt-in): lengths 64, 128, 256, both transform kinds,
# directions that do not qualify (n = 40, 37, 30, 48, 512) next to ones that do,
# repeated knots
CASES64 = [
    (2, (64, 64), 4, None), (2, (128, 40), 2, None), (3, (64, 64, 64), 4, None), (3, (256, 37, 20), 6, None),
    (3, (128, 64, 30), 8, None), (2, (64, 128), 4, ({32: 1}, {20: 2, 100: 1})), (2, (32, 64), 3, None),
    (3, (128, 40, 64), 5, None), (2, (64, 48), 3, ({20: 2}, None)), (2, (512, 64), 4, None),
]


def _warp_len64(n, p):
    L = _warp_len(n, p)
    return L if L <= 256 else 0


@pytest.mark.parametrize("d,ns,p,knots", CASES64)
def test_fp64_warp_pass_matches_oracle_and_block_kernel(d, ns, p, knots):
    torch = require_gpu()
    from oracle import operators, splitting
    from paper_2512_20269_gb300 import IFFDPlan
    kw = {} if knots is None else {"knots": list(knots)}
    plan = IFFDPlan(d, list(ns), p, **kw)
    block = IFFDPlan(d, list(ns), p, **kw)
    warp_axes = [a for a in range(d) if _warp_len64(ns[a], p)]
    for a in range(d):
        # the FP64-pipe block kernel (plans whose every direction has a warp
        # pass default to the double-float passes instead)
        block.set_geometry(a, pipelined=False)
        plan.set_geometry(a, pipelined=False)
        assert not plan.tiles(a)["warp"]  # opt-in for FP64
    for a in warp_axes:
        plan.set_geometry(a, warp=True)
    for a in range(d):
        t = plan.tiles(a)
        assert t["warp"] == (a in warp_axes)
        if t["warp"]:
            assert t["pencils_transform"] == {64: 64, 128: 32, 256: 16}[_warp_len64(ns[a], p)]
    r = inputs.rhs(plan.shape, "normal", seed=930 + sum(ns) + p)
    rg = _gpu(torch, r)
    sp = [splitting.axis_split(n, p, (0, 1), rep=(knots[a] if knots else None)) for a, n in enumerate(ns)]
    zo = operators.iffd_apply(r, sp)
    z = plan.apply_preconditioner(rg).cpu().numpy()
    zb = block.apply_preconditioner(rg).cpu().numpy()
    assert np.max(np.abs(z - zo)) <= 1e-12 * np.max(np.abs(zo))
    assert _rel(z, zb) <= 1e-13
    assert np.array_equal(plan.apply_preconditioner(rg).cpu().numpy(), z)


def test_fp64_warp_pass_pcg():
    """PCG with FP64 warp-FFT passes on every direction (the fused dot
    products of the last backward pass included): same iteration count as the
    block kernel, true relative residual <= 1.1e-8, solutions within 1e-10."""
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    for ns, p in (((64, 128, 128), 4), ((64, 32, 64), 3)):
        plan = IFFDPlan(3, ns, p)
        for a in range(3):
            plan.set_geometry(a, pipelined=False)  # FP64-pipe block kernel
        f = _gpu(torch, inputs.rhs(plan.shape, "normal", seed=6 + p))
        ub, ib = plan.pcg_solve(f)
        for a in range(3):
            plan.set_geometry(a, warp=True)
        uw, iw = plan.pcg_solve(f)
        assert iw["status"] == 0 and iw["true_rel_res"] <= 1.1e-8 and iw["iters"] == ib["iters"]
        assert float(torch.linalg.norm(uw - ub) / torch.linalg.norm(ub)) <= 1e-10
