"""GPU tests of the engine's persistent launch (iffd_engine_set_persistent):
every step runs its PCG iterations (Section 3, preconditioner of eq.
"preconditioner") of all active requests as one kernel launch walking a
device work queue of (request, phase, tile) items. Each result must equal
(bitwise) iffd_pcg_solve on a plan with the same kernels (block transform
passes), requests must be able to join while others iterate, and a bounded
device wait that runs out (made to run out by the test hook: an item waits on
a count nothing reaches) must end the step with IFFD_ERR_TIMEOUT instead of
hanging."""

import time

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import oracle_stiffness, require_gpu

pytestmark = pytest.mark.gpu

MIX = [(2, 30, 4), (3, 16, 2), (3, 24, 3), (3, 32, 4), (3, 16, 5), (3, 24, 6), (2, 64, 3), (3, 48, 4), (2, 40, 2),
       (2, 33, 7), (3, 15, 7), (3, 64, 4), (2, 128, 6), (3, 20, 8)]


def _alone(d, n, p, f, precision):
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(d, n, p, precision=precision, true_residual=False)
    for a in range(d):
        plan.set_geometry(a, pipelined=False)  # block transform kernels, as in the persistent launch
    u, info = plan.pcg_solve(f)
    return u.clone(), info


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_persistent_launch_equals_alone(precision):
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDEngine
    eng = IFFDEngine(4 << 30, precision=precision, persistent=True)
    reqs = {}
    for k, (d, n, p) in enumerate(MIX):
        m = n + p - 2
        f = torch.from_numpy(inputs.rhs((m,) * d, "normal", seed=900 + k)).cuda()
        u = torch.full_like(f, float("nan"))
        reqs[eng.submit(d, n, p, f, u)] = (d, n, p, f, u)
    k0 = eng.stats()["kernel_launches"]
    steps = 0
    done = {}
    while True:
        active = eng.step(3)
        steps += 1
        done.update(dict(eng.poll()))
        if active == 0:
            break
    launches = eng.stats()["kernel_launches"] - k0
    # per step: one persistent launch plus the state gather, and the
    # initialisation launches of the first step
    assert launches <= 2 * steps + 40
    assert set(done) == set(reqs)
    for rid, (d, n, p, f, u) in reqs.items():
        ua, ia = _alone(d, n, p, f, precision)
        assert done[rid]["status"] == 0 and done[rid]["iters"] == ia["iters"], (d, n, p)
        assert torch.equal(u, ua), (d, n, p)
        fu = f.cpu().numpy()
        res = np.linalg.norm(fu - oracle_stiffness(u.cpu().numpy(), n, p)) / np.linalg.norm(fu)
        assert res <= 1.1e-8


def test_persistent_continuous_batching():
    """Requests join while others are iterating; membership changes rebuild
    the queue; every result still equals its stand-alone solve."""
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDEngine
    eng = IFFDEngine(4 << 30, precision="fp32", persistent=True)
    pending = list(enumerate(MIX[:8]))
    tensors, ids, results = {}, {}, {}
    while pending or len(results) < 8:
        if pending:
            k, (d, n, p) = pending.pop(0)
            m = n + p - 2
            f = torch.from_numpy(inputs.rhs((m,) * d, "uniform", seed=950 + k)).cuda()
            u = torch.empty_like(f)
            tensors[k] = (d, n, p, f, u)
            ids[eng.submit(d, n, p, f, u)] = k
        eng.step(1)
        for rid, info in eng.poll():
            results[ids[rid]] = info
    for k, (d, n, p, f, u) in tensors.items():
        ua, ia = _alone(d, n, p, f, "fp32")
        assert results[k]["iters"] == ia["iters"]
        assert torch.equal(u, ua), (d, n, p)


def test_persistent_wait_limit_reports_timeout():
    """A wait that cannot be satisfied (test hook) runs out after the bounded
    number of polls: the step returns IFFD_ERR_TIMEOUT promptly, no hang."""
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDEngine, IFFDError
    eng = IFFDEngine(1 << 30, precision="fp32", persistent=True, wait_limit=2000, inject_stall=True)
    f = torch.from_numpy(inputs.rhs((26,) * 3, "normal", seed=960)).cuda()
    eng.submit(3, 24, 4, f, torch.empty_like(f))
    t0 = time.time()
    with pytest.raises(IFFDError) as exc:
        eng.step(2)
    assert exc.value.code == 8  # IFFD_ERR_TIMEOUT
    assert time.time() - t0 < 60
    eng.close()
    # the context is still usable
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(3, 16, 4)
    _, info = plan.pcg_solve(torch.from_numpy(inputs.rhs(plan.shape, "normal", seed=961)).cuda())
    assert info["status"] == 0


def test_persistent_mode_limits():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDEngine, IFFDError
    eng = IFFDEngine(1 << 30, persistent=True)
    f = torch.zeros(11 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(IFFDError):
        eng.submit(3, 2, 11, f, torch.empty_like(f))  # p = 11: outside the launch's degrees
    g = torch.zeros(26 ** 3, dtype=torch.float64, device="cuda")
    eng.submit(3, 24, 4, g, torch.empty_like(g))
    assert eng._lib.iffd_engine_set_persistent(eng._h, 0, 0, 0) == 1  # not while requests are active
