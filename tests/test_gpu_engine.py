"""GPU tests of the batched / continuous-batching engine (iffd_engine_*):
every request's result equals the same problem solved alone by
iffd_pcg_solve with the same options (bitwise: same kernels, tiles and
reduction order), requests can join while others are iterating, and
admission follows the workspace budget."""

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import oracle_stiffness, require_gpu

pytestmark = pytest.mark.gpu

# A 2D system comes before 3D systems of the same degree (p = 4, 7): the 2D one
# has no middle sweep, so this checks that every system's sweeps run in order.
# (3, 64, 4) and (2, 128, 6) run their FP32 transforms as the warp-FFT pass.
MIX = [(2, 30, 4), (3, 16, 2), (3, 24, 3), (3, 32, 4), (3, 16, 5), (3, 24, 6), (2, 64, 3), (3, 48, 4), (2, 40, 2),
       (2, 33, 7), (3, 15, 7), (3, 64, 4), (2, 128, 6)]


def _alone(torch, d, n, p, f, precision):
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(d, n, p, precision=precision, true_residual=False)
    if precision == "fp64":
        # the engine runs FP64 systems on the FP64-pipe block kernel (not the
        # double-float passes that stand-alone FP64 plans take by default)
        for a in range(d):
            plan.set_geometry(a, pipelined=False)
    u, info = plan.pcg_solve(f)
    return u.clone(), info


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_engine_mix_equals_alone(precision):
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDEngine
    eng = IFFDEngine(4 << 30, precision=precision)
    reqs = {}
    for k, (d, n, p) in enumerate(MIX):
        m = n + p - 2
        f = torch.from_numpy(inputs.rhs((m,) * d, "normal", seed=200 + k)).cuda()
        u = torch.full_like(f, float("nan"))
        rid = eng.submit(d, n, p, f, u)
        assert rid is not None
        reqs[rid] = (d, n, p, f, u)
    done = dict(eng.run_to_completion(iterations_per_step=3))
    assert set(done) == set(reqs)
    for rid, (d, n, p, f, u) in reqs.items():
        ua, ia = _alone(torch, d, n, p, f, precision)
        assert done[rid]["status"] == 0
        assert done[rid]["iters"] == ia["iters"]
        assert torch.equal(u, ua), (d, n, p)
        fu = f.cpu().numpy()
        res = np.linalg.norm(fu - oracle_stiffness(u.cpu().numpy(), n, p)) / np.linalg.norm(fu)
        assert res <= 1.1e-8


def test_engine_continuous_batching_and_budget():
    """A small budget admits only some requests; the rest are admitted as
    earlier ones finish (while others are still iterating); every result still
    equals its stand-alone solve."""
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDEngine
    probe = IFFDEngine(1 << 20)
    need = [probe.request_bytes(d, n, p) for (d, n, p) in MIX]
    probe.close()
    budget = sum(sorted(need)[-3:]) + 4096  # room for about three requests at a time
    eng = IFFDEngine(budget, precision="fp32")
    pending = list(range(len(MIX)))
    tensors = {}
    for k, (d, n, p) in enumerate(MIX):
        m = n + p - 2
        f = torch.from_numpy(inputs.rhs((m,) * d, "uniform", seed=300 + k)).cuda()
        tensors[k] = (f, torch.empty_like(f))
    ids, results = {}, {}
    refused = 0
    steps = 0
    while pending or len(results) < len(MIX):
        still = []
        for k in pending:
            d, n, p = MIX[k]
            rid = eng.submit(d, n, p, *tensors[k])
            if rid is None:
                refused += 1
                still.append(k)
            else:
                ids[rid] = k
        pending = still
        eng.step(2)
        steps += 1
        for rid, info in eng.poll():
            results[ids[rid]] = info
        assert steps < 500
    assert refused > 0  # the budget did limit admission
    for k, (d, n, p) in enumerate(MIX):
        f, u = tensors[k]
        ua, ia = _alone(torch, d, n, p, f, "fp32")
        assert results[k]["iters"] == ia["iters"]
        assert torch.equal(u, ua)


def test_engine_rejects_oversized_and_bad_requests():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDEngine, IFFDError
    eng = IFFDEngine(1 << 20)
    f = torch.zeros(66 ** 3, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    with pytest.raises(IFFDError):
        eng.submit(3, 64, 4, f, u)   # needs far more than 1 MiB
    with pytest.raises(IFFDError):
        eng.submit(3, 4, 5, f, u)    # n <= p


def test_engine_mixed_boundaries_equal_alone():
    """Requests with natural conditions on some faces (generic Table 1
    transforms) share the engine's launches with Dirichlet requests and still
    equal their stand-alone solves bitwise."""
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDEngine, IFFDPlan
    mix = [(3, 20, 4, ((1, 0), (0, 1), (0, 0))), (3, 20, 4, None), (2, 33, 3, ((0, 0), (1, 1))),
           (3, 17, 5, ((0, 1), (1, 1), (1, 0)))]
    eng = IFFDEngine(2 << 30, precision="fp32")
    reqs = {}
    for k, (d, n, p, dirichlet) in enumerate(mix):
        plan = IFFDPlan(d, n, p, precision="fp32", true_residual=False, dirichlet=dirichlet)
        f = torch.from_numpy(inputs.rhs(plan.shape, "normal", seed=600 + k)).cuda().reshape(-1)
        u = torch.empty_like(f)
        reqs[eng.submit(d, n, p, f, u, dirichlet=dirichlet)] = (plan, f, u)
    done = dict(eng.run_to_completion(iterations_per_step=2))
    for rid, (plan, f, u) in reqs.items():
        ua, ia = plan.pcg_solve(f)
        assert done[rid]["status"] == 0 and done[rid]["iters"] == ia["iters"]
        assert torch.equal(u, ua.reshape(-1))
