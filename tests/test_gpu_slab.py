"""GPU tests of the slab-decomposition building blocks (iffd_apply_pass,
iffd_slab_stiffness, iffd_copy_box, iffd_vec_dot, iffd_vec_axpby) against
the oracle, and of the whole slab-decomposed preconditioner, stiffness and PCG
(slab.py with the GPU backend) run as 1, 2 and 3 ranks on this one GPU. The
ranks are host threads with their own plans; they exchange data through a
test communicator that copies device buffers between host barriers, so no
kernel ever waits for another. Reference: the single-rank oracle (P^{-1} r to
1e-12, A^ u to 1e-13, PCG iterate with the oracle's iteration count)."""

import ctypes
import threading

import numpy as np
import pytest

from paper_2512_20269_gb300 import inputs

from gpu_common import oracle_split, require_gpu

pytestmark = pytest.mark.gpu


def _gpu(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


class ThreadComm:
    """size ranks as threads of one process: all-to-all and all-reduce by
    device copies between host barriers (test communicator)."""

    class Shared:
        def __init__(self, size):
            self.size = size
            self.bar = threading.Barrier(size)
            self.slot = [None] * size

    def __init__(self, shared, rank):
        self.sh, self.rank, self.size = shared, rank, shared.size

    def alltoall(self, out, inp, out_splits, in_splits):
        import torch
        torch.cuda.synchronize()
        self.sh.slot[self.rank] = (inp, list(in_splits))
        self.sh.bar.wait()
        pos = 0
        for s in range(self.size):
            src, splits = self.sh.slot[s]
            start = sum(splits[:self.rank])
            n = splits[self.rank]
            assert n == out_splits[s]
            if n:
                out[pos:pos + n].copy_(src[start:start + n])
            pos += n
        torch.cuda.synchronize()
        self.sh.bar.wait()

    def allreduce_sum(self, t):
        self.sh.slot[self.rank] = t.clone()
        self.sh.bar.wait()
        tot = sum(self.sh.slot[s].cpu() for s in range(self.size))
        self.sh.bar.wait()
        t.copy_(tot.to(t.device))


@pytest.mark.parametrize("world", [1, 2, 3])
@pytest.mark.parametrize("d,n,p", [(3, 16, 4), (3, 14, 5), (2, 40, 3)])
def test_slab_solver_on_virtual_ranks(world, d, n, p):
    torch = require_gpu()
    from oracle import operators
    from paper_2512_20269_gb300 import IFFDPlan
    from paper_2512_20269_gb300.slab import GpuBackend, SlabPartition, SlabSolver
    s = oracle_split(n, p)
    m = s.M.shape[0]
    shape = (m,) * d
    part = SlabPartition([m] * d, world)
    r = inputs.rhs(shape, "normal", seed=21)
    u = inputs.rhs(shape, "uniform", seed=22)
    f = inputs.rhs(shape, "normal", seed=23)
    MK = [(s.M, s.K)] * d
    z_ref = operators.iffd_apply(r, [s] * d)
    Au_ref = operators.stiffness_apply(u, MK)
    u_ref, it_ref, _ = operators.pcg(f, lambda v: operators.stiffness_apply(v, MK),
                                     lambda v: operators.iffd_apply(v, [s] * d), rtol=1e-8)
    shared = ThreadComm.Shared(world)
    out, errs = {}, []

    def rank_main(rank):
        try:
            torch.cuda.set_device(0)
            plan = IFFDPlan(d, n, p)
            zmax = max(b - a for a, b in part.z)
            solver = SlabSolver(GpuBackend(plan, zmax), part, ThreadComm(shared, rank))
            z0, z1 = part.z[rank]
            loc = lambda a: _gpu(torch, a[z0:z1].ravel())
            z = solver.apply_preconditioner(loc(r)).cpu().numpy()
            Au = solver.apply_stiffness(loc(u)).cpu().numpy()
            us, info = solver.pcg_solve(loc(f))
            out[rank] = (z, Au, us.cpu().numpy(), info)
        except Exception as exc:  # reported by the main thread
            errs.append(repr(exc))
            shared.bar.abort()

    th = [threading.Thread(target=rank_main, args=(k,)) for k in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    assert not errs, errs
    for rank in range(world):
        z0, z1 = part.z[rank]
        z, Au, us, info = out[rank]
        assert np.abs(z - z_ref[z0:z1].ravel()).max() <= 1e-12 * np.abs(z_ref).max()
        assert np.abs(Au - Au_ref[z0:z1].ravel()).max() <= 1e-13 * np.abs(Au_ref).max()
        assert info["status"] == 0 and info["iters"] == it_ref
        assert np.abs(us - u_ref[z0:z1].ravel()).max() <= 1e-10 * np.abs(u_ref).max()


def test_slab_building_blocks_and_errors():
    torch = require_gpu()
    from oracle import operators
    from paper_2512_20269_gb300 import IFFDPlan, _lib
    lib = _lib.load()
    n, p = 18, 4
    plan = IFFDPlan(3, n, p)
    s = oracle_split(n, p)
    m = s.M.shape[0]
    st = torch.cuda.current_stream().cuda_stream
    i3 = lambda v: (ctypes.c_int * 3)(*v)
    # fused pass on the box of y rows [5, 12), whole pencils along z
    t = inputs.rhs((m, 7, m), "normal", seed=31)
    tg = _gpu(torch, t)
    assert lib.iffd_apply_pass(plan._h, 2, 2, i3([m, 7, m]), i3([0, 5, 0]), tg.data_ptr(), tg.data_ptr(), st) == 0
    lam = s.lamt
    den = lam[:, None, None] + lam[None, 5:12, None] + lam[None, None, :]
    ref = operators.apply_along(s.Qt, operators.apply_along(s.Qt.T, t, 3) / den, 3)
    got = tg.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # stiffness of the rows [6, 11) from the rows [2, 15) of u
    u = inputs.rhs((m, m, m), "uniform", seed=32)
    Au_ref = operators.stiffness_apply(u, [(s.M, s.K)] * 3)
    nb = ctypes.c_size_t()
    assert lib.iffd_slab_workspace_bytes(plan._h, 5, ctypes.byref(nb)) == 0
    ws = torch.empty(nb.value // 8 + 64, dtype=torch.float64, device="cuda")
    wsp = (ws.data_ptr() + 255) // 256 * 256
    ue = _gpu(torch, u[2:15])
    Au = torch.empty(5 * m * m, dtype=torch.float64, device="cuda")
    assert lib.iffd_slab_stiffness(plan._h, 6, 5, ue.data_ptr(), Au.data_ptr(), wsp, st) == 0
    ref = Au_ref[6:11].ravel()
    assert np.abs(Au.cpu().numpy() - ref).max() <= 1e-13 * np.abs(Au_ref).max()
    # box copy, dot, axpby
    a = _gpu(torch, inputs.rhs((9, 8, 7), "normal", seed=33))
    b = torch.zeros(3 * 4 * 5, dtype=torch.float64, device="cuda")
    assert lib.iffd_copy_box(a.data_ptr(), i3([7, 8, 9]), i3([2, 3, 4]), b.data_ptr(), i3([5, 4, 3]), i3([0, 0, 0]),
                             i3([5, 4, 3]), st) == 0
    assert torch.equal(b.reshape(3, 4, 5), a[4:7, 3:7, 2:7])
    x = _gpu(torch, inputs.rhs((100003,), "normal", seed=34))
    y = _gpu(torch, inputs.rhs((100003,), "normal", seed=35))
    dws = torch.empty(4096, dtype=torch.float64, device="cuda")
    res = torch.empty(1, dtype=torch.float64, device="cuda")
    assert lib.iffd_vec_dot(x.data_ptr(), y.data_ptr(), x.numel(), res.data_ptr(), dws.data_ptr(), st) == 0
    xd, yd = x.cpu().numpy(), y.cpu().numpy()
    assert abs(res.item() - float(np.dot(xd, yd))) <= 1e-12 * np.linalg.norm(xd) * np.linalg.norm(yd)
    assert lib.iffd_vec_axpby(x.numel(), 2.5, x.data_ptr(), -0.5, y.data_ptr(), st) == 0
    assert np.abs(y.cpu().numpy() - (2.5 * xd - 0.5 * yd)).max() <= 1e-15 * np.abs(yd).max() * 8
    # argument errors
    assert lib.iffd_apply_pass(plan._h, 2, 2, i3([m, 7, m - 1]), i3([0, 5, 0]), tg.data_ptr(), tg.data_ptr(), st) == 1
    assert lib.iffd_apply_pass(plan._h, 0, 2, i3([m, 7, m]), i3([0, 5, 0]), tg.data_ptr(), tg.data_ptr(), st) == 1
    assert lib.iffd_copy_box(a.data_ptr(), i3([7, 8, 9]), i3([3, 3, 4]), b.data_ptr(), i3([5, 4, 3]), i3([0, 0, 0]),
                             i3([5, 4, 3]), st) == 1
    p32 = IFFDPlan(3, n, p, precision="fp32")
    assert lib.iffd_apply_pass(p32._h, 0, 0, i3([m, m, m]), i3([0, 0, 0]), tg.data_ptr(), tg.data_ptr(), st) == 2
