"""GPU parity at the benchmark workloads' full sizes, in the launch
configuration the bench times (one plan, the C ABI, default options).

* square n=64 p=3 (4,225 DoFs): preconditioner vs oracle, PCG vs the dense
  direct solve and the oracle's exact FD solve.
* cube n=64 p=4 (66^3): preconditioner and PCG iterate vs the oracle.
* cube n=256 p=4 (258^3 = 17.2 M DoFs): full preconditioner apply vs the oracle
  (1e-12), stiffness vs the oracle, PCG true residual <= 1e-8 checked with the
  oracle's stiffness, and the iteration count bounded as in Table "tab:square".
"""

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import (oracle_exact_fd, oracle_pcg, oracle_precond, oracle_split, oracle_stiffness, rel_max_err,
                        require_gpu)

pytestmark = pytest.mark.gpu


def _gpu(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_square_n64_p3_full():
    torch = require_gpu()
    from oracle import operators
    from paper_2512_20269_gb300 import IFFDPlan
    w = inputs.SQUARE_N64_P3
    f = inputs.workload_rhs(w)
    plan = IFFDPlan(w.d, w.n, w.p)
    z = plan.apply_preconditioner(_gpu(torch, f)).cpu().numpy()
    assert rel_max_err(z, oracle_precond(f, w.n, w.p)) <= 1e-12
    u, info = plan.pcg_solve(_gpu(torch, f))
    u = u.cpu().numpy()
    s = oracle_split(w.n, w.p)
    A = operators.dense_stiffness([(s.M, s.K)] * 2)
    ustar = np.linalg.solve(A, f.ravel()).reshape(f.shape)
    np.testing.assert_allclose(oracle_exact_fd(f, w.n, w.p), ustar, atol=1e-11 * np.abs(ustar).max())
    res = np.linalg.norm(f.ravel() - A @ u.ravel()) / np.linalg.norm(f)
    assert info["status"] == 0 and res <= 1.1e-8
    # error bound implied by the residual: ||u - u*|| <= ||A^{-1}|| ||f - A u||
    err = np.linalg.norm(u - ustar)
    bound = np.linalg.norm(np.linalg.solve(A, f.ravel() - A @ u.ravel())) * (1 + 1e-6) + 1e-14
    assert err <= bound
    _, it_o, _ = oracle_pcg(f, w.n, w.p)
    assert abs(info["iters"] - it_o) <= 1


def test_cube_n64_p4_subcase():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    w = inputs.CUBE_N64_P4
    f = inputs.workload_rhs(w)
    plan = IFFDPlan(w.d, w.n, w.p)
    z = plan.apply_preconditioner(_gpu(torch, f)).cpu().numpy()
    assert rel_max_err(z, oracle_precond(f, w.n, w.p)) <= 1e-12
    u, info = plan.pcg_solve(_gpu(torch, f))
    u = u.cpu().numpy()
    uo, it_o, _ = oracle_pcg(f, w.n, w.p)
    assert abs(info["iters"] - it_o) <= 1
    res = np.linalg.norm(f - oracle_stiffness(u, w.n, w.p)) / np.linalg.norm(f)
    assert res <= 1.1e-8
    ustar = oracle_exact_fd(f, w.n, w.p)
    # both iterates are within their residual bound of the exact solution
    assert np.linalg.norm(u - uo) <= 10 * (np.linalg.norm(u - ustar) + np.linalg.norm(uo - ustar)) + 1e-15


@pytest.mark.slow
def test_cube_n256_p4_full():
    torch = require_gpu()
    from paper_2512_20269_gb300 import IFFDPlan
    w = inputs.CUBE_N256_P4
    f = inputs.workload_rhs(w)
    plan = IFFDPlan(w.d, w.n, w.p)
    fg = _gpu(torch, f)
    z = plan.apply_preconditioner(fg).cpu().numpy()
    zo = oracle_precond(f, w.n, w.p)
    assert rel_max_err(z, zo) <= 1e-12
    assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)
    # FP32 transforms (the warp-FFT pass on every direction at this size)
    plan32 = IFFDPlan(w.d, w.n, w.p, precision="fp32")
    assert all(plan32.tiles(a)["warp"] for a in range(w.d))
    z32 = plan32.apply_preconditioner(fg).cpu().numpy()
    assert np.linalg.norm(z32 - zo) <= 1e-5 * np.linalg.norm(zo)
    del z, zo, z32
    Au = plan.apply_stiffness(fg).cpu().numpy()
    assert rel_max_err(Au, oracle_stiffness(f, w.n, w.p)) <= 1e-13
    del Au
    u, info = plan.pcg_solve(fg)
    assert info["status"] == 0 and info["iters"] <= 8
    u = u.cpu().numpy()
    res = np.linalg.norm(f - oracle_stiffness(u, w.n, w.p)) / np.linalg.norm(f)
    assert res <= 1.1e-8
    assert abs(res - info["true_rel_res"]) <= 1e-10
    u32, i32 = plan32.pcg_solve(fg)
    assert i32["status"] == 0 and i32["iters"] <= info["iters"] + 2
    res32 = np.linalg.norm(f - oracle_stiffness(u32.cpu().numpy(), w.n, w.p)) / np.linalg.norm(f)
    assert res32 <= 1.1e-8
