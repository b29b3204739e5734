"""GPU tests of iffd_batch_solve (PCG of Section 3 with the preconditioner of
eq. "preconditioner", many plans and right-hand sides in one call), through
the C ABI: a mixed batch of FP32-transform and FP64 plans, several right-hand
sides per plan (eight for the 64^3 problem, as in the batched workload), mixed
boundary conditions, and plans the engine does not run (exact FD, variable
coefficient) solved on their workspace slices. Every solution must equal
(bitwise) iffd_pcg_solve on the same plan and right-hand side, satisfy the
stopping rule with the oracle's operator (true residual <= 1.1e-8), and take
the oracle PCG's iteration count +-1 (checked on a subset)."""

import functools

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import oracle_pcg, oracle_stiffness, oracle_varcoef_stiffness, require_gpu

pytestmark = pytest.mark.gpu


def _dset(pair):
    return tuple(k for k, v in zip((0, 1), pair) if v)


@functools.lru_cache(maxsize=None)
def _mixed_mk(n, p, pair):
    import scipy.sparse
    from oracle import splitting
    s = splitting.axis_split(n, p, _dset(pair))
    return scipy.sparse.csr_matrix(s.M), scipy.sparse.csr_matrix(s.K)


# (d, n, p, precision, precond, coef, dirichlet, nrhs, check oracle iterations)
BATCH = [
    (3, 24, 4, "fp32", "iffd", "const", None, 3, True),
    (2, 40, 3, "fp32", "iffd", "const", None, 1, True),
    (3, 16, 6, "fp32", "iffd", "const", None, 2, False),
    (3, 20, 5, "fp64", "iffd", "const", None, 2, True),
    (2, 33, 7, "fp64", "iffd", "const", None, 1, False),
    (3, 20, 4, "fp32", "iffd", "const", ((1, 0), (1, 1), (0, 1)), 2, False),
    (3, 12, 3, "fp64", "exact_fd", "const", None, 1, False),
    (3, 16, 4, "fp64", "iffd", "sin", None, 1, False),
    (3, 64, 4, "fp64", "iffd", "const", None, 2, False),  # double-float transforms: solved one by one
]


def _true_res(uh, fh, d, n, p, coef, dirichlet):
    if dirichlet is not None:
        from oracle import operators
        Au = operators.stiffness_apply(uh, [_mixed_mk(n, p, tuple(dirichlet[k])) for k in range(d)])
    elif coef == "sin":
        Au = oracle_varcoef_stiffness(uh, n, p)
    else:
        Au = oracle_stiffness(uh, n, p)
    return np.linalg.norm(fh - Au) / np.linalg.norm(fh)


def test_batch_solve_mixed_equals_alone_and_oracle():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan, batch_solve
    plans, fs, hosts = [], [], []
    for k, (d, n, p, prec, pc, coef, dirichlet, nrhs, _) in enumerate(BATCH):
        pl = IFFDPlan(d, n, p, precision=prec, precond=pc, coef=coef, dirichlet=dirichlet, true_residual=True)
        if (d, n, p, prec) == (3, 64, 4, "fp64"):
            pl.set_geometry(0, double_float=True)
        fh = np.stack([inputs.rhs(pl.shape, "normal", seed=600 + 10 * k + j) for j in range(nrhs)])
        plans.append(pl)
        hosts.append(fh)
        fs.append(torch.from_numpy(fh).cuda())
    us, infos = batch_solve(plans, fs)
    torch.cuda.synchronize()
    slot = 0
    for k, (d, n, p, prec, pc, coef, dirichlet, nrhs, chk_it) in enumerate(BATCH):
        pl = plans[k]
        for j in range(nrhs):
            info = infos[slot]
            slot += 1
            assert info["status"] == 0, (k, j, info)
            ua, ia = pl.pcg_solve(fs[k][j].contiguous())
            assert torch.equal(us[k][j], ua), (k, j)
            assert info["iters"] == ia["iters"]
            uh = us[k][j].cpu().numpy()
            tr = _true_res(uh, hosts[k][j], d, n, p, coef, dirichlet)
            assert tr <= 1.1e-8, (k, j, tr)
            assert abs(info["true_rel_res"] - tr) <= 1e-6 * tr + 1e-13
            if chk_it and j == 0:
                _, it_or, _ = oracle_pcg(hosts[k][j], n, p)
                assert abs(info["iters"] - it_or) <= 1, (k, info["iters"], it_or)
    assert slot == len(infos)


def test_batch_solve_eight_rhs_of_the_64_cube():
    """Config 4's eight right-hand sides of one 64^3 problem (n = 64, p = 4,
    FP32 transforms) in one call against one plan."""
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan, batch_solve
    pl = IFFDPlan(3, 64, 4, precision="fp32", true_residual=False)
    fh = np.stack([inputs.rhs(pl.shape, "normal", seed=700 + j) for j in range(8)])
    f = torch.from_numpy(fh).cuda()
    (u,), infos = batch_solve([pl], [f])
    assert len(infos) == 8
    for j in range(8):
        ua, ia = pl.pcg_solve(f[j].contiguous())
        assert infos[j]["status"] == 0 and infos[j]["iters"] == ia["iters"]
        assert infos[j]["true_rel_res"] == -1.0
        assert torch.equal(u[j], ua)
    uh = u[0].cpu().numpy()
    assert np.linalg.norm(fh[0] - oracle_stiffness(uh, 64, 4)) / np.linalg.norm(fh[0]) <= 1.1e-8


def test_batch_solve_statuses_and_arguments():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDError, IFFDPlan, _lib, batch_solve
    good = IFFDPlan(3, 16, 4, precision="fp32")
    capped = IFFDPlan(3, 16, 3, maxit=1)
    fg = torch.from_numpy(inputs.rhs(good.shape, "normal", seed=1)).cuda()
    fc = torch.from_numpy(inputs.rhs(capped.shape, "normal", seed=2)).cuda()
    _, infos = batch_solve([good, capped], [fg, fc], raise_on_error=False)
    assert infos[0]["status"] == 0 and infos[1]["status"] == 6 and infos[1]["iters"] == 1
    with pytest.raises(IFFDError) as exc:
        batch_solve([good, capped], [fg, fc])
    assert exc.value.code == 6
    lib = _lib.load()
    import ctypes
    h = (ctypes.c_void_p * 1)(good._h.value)
    n = (ctypes.c_int * 1)(-1)
    nb = ctypes.c_size_t()
    assert lib.iffd_batch_workspace_bytes(1, h, n, ctypes.byref(nb)) == 1
    n[0] = 0
    assert lib.iffd_batch_workspace_bytes(1, h, n, ctypes.byref(nb)) == 0 and nb.value == 0
    # zero systems: nothing to do
    assert lib.iffd_batch_solve(1, h, None, None, n, None, None, None) == 0
