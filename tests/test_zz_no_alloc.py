"""GPU test of iffd_apply_stiffness_noalloc, the allocation-free stiffness
apply. It serves callers that cannot allocate device memory where they need
A^ u: a framework whose caching allocator owns all device memory, a solver
with a device-memory budget fixed at start-up, or a loop that must not pay
cudaMalloc's implicit synchronisation. Through the C ABI it must give the same
result as iffd_apply_stiffness with a workspace, on two calls in a row (the
static scratch keeps the previous call's contents), match the oracle's
stiffness directly, and reject plans it does not serve.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test."""

import functools

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import rel_max_err, require_gpu

pytestmark = pytest.mark.gpu


def _dset(pair):
    return tuple(k for k, v in zip((0, 1), pair) if v)


@functools.lru_cache(maxsize=None)
def _oracle_mk(n, p, pair, rep):
    import scipy.sparse
    from oracle import splitting
    s = splitting.axis_split(n, p, _dset(pair), rep=dict(rep))
    return scipy.sparse.csr_matrix(s.M), scipy.sparse.csr_matrix(s.K)


# (d, n, p, Dirichlet flags per direction or None, repeated knots per direction or None)
CASES = [
    (3, 60, 4, None, None),
    (2, 300, 3, None, None),
    (3, 25, 7, None, None),
    (3, 40, 5, ((1, 0), (0, 1), (1, 1)), None),             # mixed Dirichlet / natural ends
    (2, 90, 4, ((0, 1), (1, 1)), ({30: 2}, {45: 1, 60: 3})),  # repeated interior knots
]


@pytest.mark.parametrize("d,n,p,dirichlet,knots", CASES)
def test_noalloc_matches_workspace_entry_point_and_oracle(d, n, p, dirichlet, knots):
    torch = require_gpu()
    from oracle import operators
    from paper_2512_20269_gb300 import IFFDPlan, _lib
    lib = _lib.load()
    plan = IFFDPlan(d, n, p, dirichlet=dirichlet, knots=knots)
    assert plan.N <= _lib.IFFD_NOALLOC_MAX_DOFS
    pairs = dirichlet or [(1, 1)] * d
    reps = knots or [None] * d
    mk = [_oracle_mk(n, p, tuple(pairs[k]), tuple(sorted((reps[k] or {}).items()))) for k in range(d)]
    stream = torch.cuda.current_stream()
    for call in range(2):
        uh = inputs.rhs(plan.shape, "normal", seed=500 + call)
        u = torch.from_numpy(uh).cuda()
        ref = plan.apply_stiffness(u)
        out = torch.full_like(u, float("nan"))
        rc = lib.iffd_apply_stiffness_noalloc(plan._h, u.data_ptr(), out.data_ptr(), stream.cuda_stream)
        assert rc == 0, lib.iffd_last_error()
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(a).all()
        assert rel_max_err(a, b) <= 1e-13
        assert rel_max_err(a, operators.stiffness_apply(uh, mk)) <= 1e-13


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


def test_noalloc_rejects_variable_coefficient_plans():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan, _lib
    lib = _lib.load()
    plan = IFFDPlan(3, 20, 3, coef="sin")
    u = plan.empty().zero_()
    out = plan.empty()
    rc = lib.iffd_apply_stiffness_noalloc(plan._h, u.data_ptr(), out.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream)
    assert rc == 2
    assert b"IFFD_COEF_CONST" in lib.iffd_last_error()
