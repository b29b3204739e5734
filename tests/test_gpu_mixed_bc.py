"""GPU parity for boundary sets other than Dirichlet on every face: each
direction may have Dirichlet data on both ends, on one end or on none (Table 1
of the paper: DST-I, DST-II/III on D = {0,1}; the six other transform types
through the generic zero-padded DFT). Compared element-wise with the oracle on
the same seeded inputs."""

import functools
import json
import os

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import rel_max_err, require_gpu

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dset(pair):
    return tuple(k for k, v in zip((0, 1), pair) if v)


@functools.lru_cache(maxsize=None)
def _split(n, p, pair):
    from oracle import splitting
    return splitting.axis_split(n, p, _dset(pair))


def _splits(n, p, dirichlet):
    return [_split(n, p, tuple(D)) for D in dirichlet]


def _mk(n, p, dirichlet):
    import scipy.sparse
    return [(scipy.sparse.csr_matrix(s.M), scipy.sparse.csr_matrix(s.K)) for s in _splits(n, p, dirichlet)]


def _gpu(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# (d, n, p, per-direction (x=0, x=1) Dirichlet flags): every Dirichlet set on
# both parities of p, 2D and 3D, ragged tiles, and a Bluestein length (n = 37)
CASES = [
    (2, 20, 3, ((1, 0), (0, 1))), (2, 20, 4, ((1, 0), (0, 1))),
    (2, 19, 3, ((0, 0), (1, 1))), (2, 18, 4, ((1, 1), (0, 0))),
    (2, 17, 5, ((0, 1), (1, 0))), (2, 16, 6, ((0, 0), (1, 0))),
    (2, 24, 2, ((1, 0), (0, 0))), (2, 21, 7, ((0, 1), (0, 0))),
    (2, 37, 4, ((1, 0), (0, 1))),
    (3, 12, 3, ((1, 0), (0, 1), (0, 0))), (3, 13, 4, ((1, 0), (0, 1), (0, 0))),
    (3, 10, 5, ((0, 0), (1, 1), (1, 0))), (3, 11, 2, ((0, 1), (1, 0), (1, 1))),
]


@pytest.mark.parametrize("d,n,p,dirichlet", CASES)
def test_mixed_preconditioner_and_stiffness_parity(d, n, p, dirichlet):
    torch = require_gpu()
    from oracle import operators
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(d, n, p, dirichlet=dirichlet)
    r = inputs.rhs(plan.shape, "normal", seed=80 + n + p)
    rg = _gpu(torch, r)
    zo = operators.iffd_apply(r, _splits(n, p, dirichlet))
    z = plan.apply_preconditioner(rg).cpu().numpy()
    assert rel_max_err(z, zo) <= 1e-12
    assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)
    Ao = operators.stiffness_apply(r, _mk(n, p, dirichlet))
    assert rel_max_err(plan.apply_stiffness(rg).cpu().numpy(), Ao) <= 1e-13
    z32 = IFFDPlan(d, n, p, precision="fp32", dirichlet=dirichlet).apply_preconditioner(rg).cpu().numpy()
    assert np.linalg.norm(z32 - zo) <= 1e-5 * np.linalg.norm(zo)
    # double-float transforms (the block kernel in pairs of FP32 values) where
    # no direction needs Bluestein's convolution: the FP64 tolerance
    from paper_2512_20269_gb300 import IFFDError
    dfp = IFFDPlan(d, n, p, dirichlet=dirichlet)
    try:
        dfp.set_geometry(0, double_float=True)
    except IFFDError:
        assert n == 37  # the Bluestein length
        return
    zq = dfp.apply_preconditioner(rg).cpu().numpy()
    assert rel_max_err(zq, zo) <= 1e-12


@pytest.mark.parametrize("d,n,p,dirichlet", [(2, 16, 3, ((1, 0), (0, 0))), (3, 9, 4, ((1, 0), (0, 1), (0, 0)))])
def test_mixed_exact_fd_parity(d, n, p, dirichlet):
    torch = require_gpu()
    from oracle import operators
    from paper_2512_20269_gb300 import IFFDPlan
    plan = IFFDPlan(d, n, p, precond="exact_fd", dirichlet=dirichlet)
    r = inputs.rhs(plan.shape, "normal", seed=90 + n)
    eigs = [operators.exact_fd_eig(s.M, s.K) for s in _splits(n, p, dirichlet)]
    zo = operators.exact_fd_apply(r, eigs)
    z = plan.apply_preconditioner(_gpu(torch, r)).cpu().numpy()
    assert rel_max_err(z, zo) <= 1e-12


@pytest.mark.parametrize("n", [64, 128])
def test_table_cube_iterations(n):
    """Table "tab:cube": unit cube, Dirichlet on x = 0 and y = 1, natural
    conditions elsewhere, p = 2..5, PCG iterations within +-1 of the paper's,
    equal to the oracle's on the same right-hand side (n = 64), true relative
    residual <= 1.1e-8."""
    torch = require_gpu()
    from oracle import operators
    from paper_2512_20269_gb300 import IFFDPlan
    g = json.load(open(os.path.join(GOLDEN, "table_cube_iterations.json")))
    ref = g["iterations"][g["n"].index(n)]
    dirichlet = [tuple(D) for D in g["dirichlet"]]
    for p, it_ref in zip(g["p"], ref):
        plan = IFFDPlan(3, n, p, dirichlet=dirichlet)
        f = np.random.default_rng(500 + p).uniform(-1, 1, plan.shape)
        u, info = plan.pcg_solve(_gpu(torch, f))
        assert info["status"] == 0 and abs(info["iters"] - it_ref) <= 1, (p, info)
        assert info["true_rel_res"] <= 1.1e-8
        if n == 64:
            sp = _splits(n, p, dirichlet)
            mk = _mk(n, p, dirichlet)
            _, it_o, _ = operators.pcg(f, lambda v: operators.stiffness_apply(v, mk),
                                       lambda r: operators.iffd_apply(r, sp), rtol=1e-8)
            assert abs(info["iters"] - it_o) <= 1
            true_rel = np.linalg.norm(f - operators.stiffness_apply(u.cpu().numpy(), mk)) / np.linalg.norm(f)
            assert true_rel <= 1.1e-8


def test_mixed_fp32_pcg_and_tuned_plan():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    dirichlet = ((1, 0), (0, 1), (0, 0))
    f = inputs.rhs((100, 99, 99), "normal", seed=7)  # n = 96, p = 4: m = 99, 99, 100
    fg = _gpu(torch, f)
    _, i64 = IFFDPlan(3, 96, 4, dirichlet=dirichlet).pcg_solve(fg)
    _, i32 = IFFDPlan(3, 96, 4, precision="fp32", dirichlet=dirichlet).autotune().pcg_solve(fg)
    assert i64["true_rel_res"] <= 1.1e-8 and i32["true_rel_res"] <= 1.1e-8
    assert i32["iters"] <= i64["iters"] + 2
