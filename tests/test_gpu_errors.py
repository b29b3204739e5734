"""GPU tests of the PCG failure paths (Section 3's PCG with its breakdown and
stopping conditions): a right-hand side holding NaN or Inf makes the solve
report IFFD_ERR_BREAKDOWN (the first inner product is not positive and
finite), an iteration cap below the needed count reports
IFFD_ERR_NOT_CONVERGED with exactly that many iterations, and in the batched
engine a failing request is retired with its status and frees its arena
memory while the requests beside it still give their stand-alone results.
The failures are made on the host (the inputs); no GPU fault is involved."""

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu

IFFD_ERR_NOT_CONVERGED = 6
IFFD_ERR_BREAKDOWN = 7


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_nonfinite_rhs_reports_breakdown(precision, bad):
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDError, IFFDPlan
    plan = IFFDPlan(3, 20, 4, precision=precision)
    fh = inputs.rhs(plan.shape, "normal", seed=7)
    fh.reshape(-1)[1234] = bad
    f = torch.from_numpy(fh).cuda()
    _, info = plan.pcg_solve(f, raise_on_error=False)
    assert info["status"] == IFFD_ERR_BREAKDOWN
    with pytest.raises(IFFDError) as exc:
        plan.pcg_solve(f)
    assert exc.value.code == IFFD_ERR_BREAKDOWN
    # the plan stays usable: a finite right-hand side solves normally
    ok = torch.from_numpy(inputs.rhs(plan.shape, "normal", seed=8)).cuda()
    _, info = plan.pcg_solve(ok)
    assert info["status"] == 0 and info["true_rel_res"] <= 1.1e-8


@pytest.mark.parametrize("maxit", [1, 2, 3])
def test_iteration_cap_reports_not_converged(maxit):
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDError, IFFDPlan
    plan = IFFDPlan(3, 24, 3, maxit=maxit)  # needs ~7 iterations to 1e-8
    f = torch.from_numpy(inputs.rhs(plan.shape, "uniform", seed=9)).cuda()
    u, info = plan.pcg_solve(f, raise_on_error=False)
    assert info["status"] == IFFD_ERR_NOT_CONVERGED
    assert info["iters"] == maxit
    assert info["rel_res"] > 1e-8 and np.isfinite(info["true_rel_res"])
    # the reported residual is that of the returned iterate (u holds the last iterate)
    assert abs(info["true_rel_res"] - info["rel_res"]) <= 1e-6 * info["rel_res"] + 1e-12
    with pytest.raises(IFFDError) as exc:
        plan.pcg_solve(f)
    assert exc.value.code == IFFD_ERR_NOT_CONVERGED
    assert np.isfinite(u.cpu().numpy()).all()


def test_engine_failing_request_is_retired_and_frees_its_memory():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDEngine, IFFDPlan
    eng = IFFDEngine(1 << 30, precision="fp32")
    free0 = eng.stats()["bytes_free"]
    good = [(3, 24, 4), (2, 40, 3), (3, 16, 6)]
    reqs = {}
    for k, (d, n, p) in enumerate(good):
        m = n + p - 2
        f = torch.from_numpy(inputs.rhs((m,) * d, "normal", seed=40 + k)).cuda()
        u = torch.empty_like(f)
        reqs[eng.submit(d, n, p, f, u)] = ("good", d, n, p, f, u)
    fb = inputs.rhs((26,) * 3, "normal", seed=44)
    fb.reshape(-1)[77] = float("nan")
    fbad = torch.from_numpy(fb).cuda()
    bad_id = eng.submit(3, 24, 4, fbad, torch.empty_like(fbad))
    reqs[bad_id] = ("bad",)
    assert eng.stats()["bytes_free"] < free0
    done = dict(eng.run_to_completion(iterations_per_step=2))
    assert set(done) == set(reqs)
    assert done[bad_id]["status"] == IFFD_ERR_BREAKDOWN
    for rid, entry in reqs.items():
        if entry[0] != "good":
            continue
        _, d, n, p, f, u = entry
        plan = IFFDPlan(d, n, p, precision="fp32", true_residual=False)
        ua, ia = plan.pcg_solve(f)
        assert done[rid]["status"] == 0 and done[rid]["iters"] == ia["iters"]
        assert torch.equal(u, ua)
    st = eng.stats()
    assert st["active"] == 0 and st["bytes_free"] == free0


def test_engine_iteration_cap():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDEngine
    eng = IFFDEngine(1 << 30, precision="fp64", maxit=2)
    free0 = eng.stats()["bytes_free"]
    f = torch.from_numpy(inputs.rhs((26,) * 3, "normal", seed=45)).cuda()
    rid = eng.submit(3, 24, 4, f, torch.empty_like(f))
    done = dict(eng.run_to_completion(iterations_per_step=1))
    assert done[rid]["status"] == IFFD_ERR_NOT_CONVERGED and done[rid]["iters"] == 2
    assert eng.stats()["bytes_free"] == free0
