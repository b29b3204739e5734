"""GPU tests of the captured solve graphs of iffd_pcg_solve (Section 3's PCG
with the preconditioner of eq. "preconditioner"): a solve that repeats the
previous solve's (f, u, workspace) runs its chunks of iterations from CUDA
graphs captured on the plan's private stream. The graph solves must be
bitwise the direct solves (same kernels, same order; the direct path is
forced by per-launch event timing), count the same kernel launches, follow
a change of f, of u and of the launch geometry, and handle an iteration cap
that is not a multiple of the chunk. A solve's first chunk runs as many
iterations as the plan's last converged solve took, so repeated solves
enqueue no iterations past convergence."""

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import oracle_stiffness, require_gpu

pytestmark = pytest.mark.gpu

PLANS = [
    dict(d=3, n=24, p=4, precision="fp64"),                      # FP64 block passes
    dict(d=3, n=128, p=4, precision="fp64"),                     # double-float passes
    dict(d=3, n=64, p=3, precision="fp32"),                      # FP32 warp passes (flexible beta)
    dict(d=2, n=40, p=5, precision="fp64", precond="exact_fd"),  # exact FD comparator
]


def _direct(plan, f, u):
    """A solve with per-launch event timing on: always the direct launches."""
    plan.profile_enable(True)
    n0 = plan.launch_count()
    _, info = plan.pcg_solve(f, u, raise_on_error=False)
    n1 = plan.launch_count()
    plan.profile_enable(False)
    return u.clone(), info, n1 - n0


@pytest.mark.parametrize("kw", PLANS)
def test_graph_solves_bitwise_equal_direct(kw):
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(true_residual=False, **kw)
    f = torch.from_numpy(inputs.rhs(plan.shape, "normal", seed=1700 + kw["n"])).cuda()
    u = plan.empty()
    ud, idir, n_cold = _direct(plan, f, u)
    # the first chunk of a later solve runs as many iterations as this one
    # took, so no iteration is enqueued past convergence
    ud2, _, nd = _direct(plan, f, u)
    assert torch.equal(ud2, ud)
    surplus = (-idir["iters"]) % 4  # iterations past convergence in chunks of 4
    if surplus:
        assert nd < n_cold and (n_cold - nd) % surplus == 0
    else:
        assert nd == n_cold
    for _ in range(3):  # the first of these records (f, u), the second captures, the third replays
        u.fill_(float("nan"))
        n0 = plan.launch_count()
        _, info = plan.pcg_solve(f, u)
        assert plan.launch_count() - n0 == nd
        assert info["iters"] == idir["iters"] and info["status"] == 0
        assert torch.equal(u, ud)
    uh = u.cpu().numpy()
    fh = f.cpu().numpy()
    if kw["d"] == 3:
        assert np.linalg.norm(fh - oracle_stiffness(uh, kw["n"], kw["p"])) <= 1.1e-8 * np.linalg.norm(fh)


def test_graphs_follow_inputs_and_geometry():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(3, 64, 4, precision="fp32", true_residual=False)
    fa = torch.from_numpy(inputs.rhs(plan.shape, "normal", seed=1801)).cuda()
    fb = torch.from_numpy(inputs.rhs(plan.shape, "uniform", seed=1802)).cuda()
    ua, ub = plan.empty(), plan.empty()
    ref_a, _, _ = _direct(plan, fa, ua)
    ref_b, _, _ = _direct(plan, fb, ub)
    for _ in range(2):
        plan.pcg_solve(fa, ua)
    assert torch.equal(ua, ref_a)
    fa.copy_(fb)  # same pointers, new values: the graph reads them
    plan.pcg_solve(fa, ua)
    assert torch.equal(ua, ref_b)
    for _ in range(2):  # other pointers: recaptured
        plan.pcg_solve(fb, ub)
    assert torch.equal(ub, ref_b)
    plan.set_geometry(2, warp=True)  # unpaired fused pass: the graphs are dropped
    ref_c, _, _ = _direct(plan, fb, ub)
    for _ in range(2):
        plan.pcg_solve(fb, ub)
    assert torch.equal(ub, ref_c)


@pytest.mark.parametrize("maxit", [2, 5, 6, 9])
def test_graph_solves_with_an_iteration_cap(maxit):
    """A cap below, between and above chunks of 4 iterations: the same status
    and iterate as the direct solve."""
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(2, 128, 6, precision="fp64", maxit=maxit, rtol=1e-14, true_residual=False)
    f = torch.from_numpy(inputs.rhs(plan.shape, "normal", seed=1900)).cuda()
    u = plan.empty()
    ud, idir, _ = _direct(plan, f, u)
    for _ in range(3):
        _, info = plan.pcg_solve(f, u, raise_on_error=False)
        assert info["iters"] == idir["iters"] and info["status"] == idir["status"]
        assert torch.equal(u, ud)
