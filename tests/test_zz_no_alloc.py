"""GPU test of iffd_apply_stiffness_noalloc, the allocation-free stiffness apply
for callers that cannot allocate device memory when they need A^ u (stream
capture, allocator-owned or fixed-budget device memory). Through the C ABI it
must give the same result as iffd_apply_stiffness with a workspace, on two
calls in a row (the static scratch keeps the previous call's contents), and
reject problems above its fixed scratch size.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test."""

import ctypes

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import rel_max_err, require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d,n,p", [(3, 60, 4), (2, 300, 3), (3, 25, 7)])
def test_noalloc_matches_workspace_entry_point(d, n, p):
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan, _lib
    lib = _lib.load()
    plan = IFFDPlan(d, n, p)
    assert plan.N <= _lib.IFFD_NOALLOC_MAX_DOFS
    stream = torch.cuda.current_stream()
    for call in range(2):
        u = torch.from_numpy(inputs.rhs(plan.shape, "normal", seed=500 + call)).cuda()
        ref = plan.apply_stiffness(u)
        out = torch.full_like(u, float("nan"))
        rc = lib.iffd_apply_stiffness_noalloc(plan._h, u.data_ptr(), out.data_ptr(), stream.cuda_stream)
        assert rc == 0, lib.iffd_last_error()
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(a).all()
        assert rel_max_err(a, b) <= 1e-13


def test_noalloc_rejects_problems_above_the_limit():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan, _lib
    lib = _lib.load()
    plan = IFFDPlan(3, 100, 4)  # 102^3 = 1,061,208 DoFs > 2^20
    assert plan.N > _lib.IFFD_NOALLOC_MAX_DOFS
    u = plan.empty().zero_()
    out = plan.empty()
    rc = lib.iffd_apply_stiffness_noalloc(plan._h, u.data_ptr(), out.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream)
    assert rc == 2
    assert b"IFFD_NOALLOC_MAX_DOFS" in lib.iffd_last_error()
    rc = lib.iffd_apply_stiffness_noalloc(plan._h, u.data_ptr(), u.data_ptr(), None)
    assert rc == 1
