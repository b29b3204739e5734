"""GPU tests of the paired FP32 warp-FFT pass (the preconditioner of eq.
"preconditioner" with FP32 transforms): every lane group carries two complex
sequences, four pencils, at once, with the same FP32 operations per value as
the unpaired pass. Each pencil keeps the partner it has in the unpaired pass
(pencils 2s and 2s + 1 share a complex sequence), so the paired apply must
equal the unpaired apply bit for bit, and the partial sums of the dot
products fused into the last backward pass are formed per half tile in the
unpaired order, so a whole PCG solve must be bitwise the same as well. The
cases cover FFT lengths 64, 128, 256 (length 512 stays unpaired), both
transform kinds, 2D and 3D, ragged last tiles, grid lines whose four-pencil
groups are 16-byte aligned, 8-byte aligned or unaligned (odd m), and repeated
knots; the oracle checks the operator itself."""

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu

CASES = [
    (2, (64, 64), 4, None), (2, (128, 40), 2, None), (3, (64, 64, 64), 4, None), (3, (256, 37, 20), 6, None),
    (3, (128, 64, 30), 8, None), (2, (64, 128), 4, ({32: 1}, {20: 2, 100: 1})), (2, (32, 64), 3, None),
    (3, (128, 40, 64), 5, None), (2, (256, 24), 7, None), (2, (512, 64), 4, None), (3, (64, 128, 64), 3, None),
]


def _warp_len(n, p):
    L = n if p % 2 == 0 else 2 * n
    return L if L in (64, 128, 256, 512) else 0


def _plans(d, ns, p, knots):
    from paper_2512_20269_gb300 import IFFDPlan
    kw = {} if knots is None else {"knots": list(knots)}
    paired = IFFDPlan(d, list(ns), p, precision="fp32", **kw)
    single = IFFDPlan(d, list(ns), p, precision="fp32", **kw)
    axes = [a for a in range(d) if _warp_len(ns[a], p)]
    for a in axes:
        single.set_geometry(a, warp=True)
        if _warp_len(ns[a], p) <= 256:
            paired.set_geometry(a, paired=True)
        else:
            paired.set_geometry(a, warp=True)
    for a in range(d):
        t = paired.tiles(a)
        assert t["paired"] == (a in axes and _warp_len(ns[a], p) <= 256)
        if t["paired"]:
            assert t["pencils_transform"] == 2 * single.tiles(a)["pencils_transform"]
    return paired, single


@pytest.mark.parametrize("d,ns,p,knots", CASES)
def test_paired_apply_bitwise_equals_unpaired(d, ns, p, knots):
    torch = require_gpu()
    from oracle import operators, splitting
    paired, single = _plans(d, ns, p, knots)
    r = inputs.rhs(paired.shape, "normal", seed=1300 + sum(ns) + p)
    rg = torch.from_numpy(r).cuda()
    zp = paired.apply_preconditioner(rg)
    zs = single.apply_preconditioner(rg)
    assert torch.equal(zp, zs)
    sp = [splitting.axis_split(n, p, (0, 1), rep=(knots[a] if knots else None)) for a, n in enumerate(ns)]
    zo = operators.iffd_apply(r, sp)
    z = zp.cpu().numpy()
    assert np.linalg.norm(z - zo) <= 1e-5 * np.linalg.norm(zo)


@pytest.mark.parametrize("d,ns,p", [(3, (64, 128, 128), 4), (3, (64, 32, 64), 3), (2, (256, 128), 6)])
def test_paired_pcg_bitwise_equals_unpaired(d, ns, p):
    torch = require_gpu()
    paired, single = _plans(d, ns, p, None)
    f = torch.from_numpy(inputs.rhs(paired.shape, "normal", seed=1400 + p)).cuda()
    up, ip = paired.pcg_solve(f)
    us, is_ = single.pcg_solve(f)
    assert ip["status"] == 0 and ip["iters"] == is_["iters"]
    assert torch.equal(up, us)
    assert ip["true_rel_res"] <= 1.1e-8


def test_paired_dot_partials_with_a_ragged_half_tile():
    """The last backward pass along x of a grid whose x-pencil count leaves
    the last paired tile with an empty second half: the apply with the fused
    dot products (a PCG solve) still matches the unpaired pass bit for bit."""
    torch = require_gpu()
    # 3D, n = 64, p = 4: 66 x 66 = 4356 x-pencils = 136 tiles of 32 + 4 (unpaired: 272 + 1 of 16)
    paired, single = _plans(3, (64, 64, 64), 4, None)
    f = torch.from_numpy(inputs.rhs(paired.shape, "uniform", seed=1500)).cuda()
    up, ip = paired.pcg_solve(f)
    us, is_ = single.pcg_solve(f)
    assert ip["iters"] == is_["iters"] and torch.equal(up, us)



def test_paired_passes_in_the_batched_solve():
    """iffd_batch_solve runs the plans' own geometry through the engine's
    batched launches: with every direction paired (the last backward pass then
    forms its dot products per half tile in the batched kernel too), every
    solution equals the stand-alone paired solve bit for bit."""
    torch = require_gpu()
    from paper_2512_20269_gb300 import batch_solve
    plans, fs = [], []
    for k, (d, ns, p) in enumerate([(3, (64, 64, 64), 4), (2, (128, 256), 3), (3, (128, 64, 64), 6)]):
        paired, _ = _plans(d, ns, p, None)
        plans.append(paired)
        fs.append(torch.from_numpy(np.stack([inputs.rhs(paired.shape, "normal", seed=2000 + 10 * k + j)
                                              for j in range(2)])).cuda())
    us, infos = batch_solve(plans, fs)
    slot = 0
    for k, pl in enumerate(plans):
        for j in range(2):
            ua, ia = pl.pcg_solve(fs[k][j].contiguous())
            assert infos[slot]["status"] == 0 and infos[slot]["iters"] == ia["iters"]
            assert torch.equal(us[k][j], ua), (k, j)
            slot += 1
