"""The slab-decomposed solve (paper_2512_20269_gb300/slab.py) on 2 and 4
gloo ranks on the CPU: the partition, the two all-to-all re-splits of the
preconditioner (eq. "preconditioner"), the halo exchange of the stiffness (eq.
"system_matrix") and the distributed PCG (Section 3) must reproduce the
single-rank oracle: P^{-1} r to 1e-12, A^ u to 1e-13, and the PCG iterate
with the same iteration count. Each rank's local steps run on a backend made
of the oracle's 1D operators (test infrastructure), so these tests check the
decomposition logic without a GPU; the GPU kernels of the local steps are
checked against the oracle in test_gpu_slab.py."""

import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


class OracleBackend:
    """SlabSolver's local steps with the oracle's dense 1D operators on CPU
    torch tensors (gloo exchanges CPU tensors)."""

    def __init__(self, splits, p):
        self.s = splits  # per direction (direction 0 first): oracle AxisSplit
        self.p = p

    # -- arrays
    def empty(self, n):
        return torch.empty(int(n), dtype=torch.float64)

    def zeros_like(self, x):
        return torch.zeros_like(x)

    def copy(self, x):
        return x.clone()

    def host_vector(self, vals):
        return torch.tensor(vals, dtype=torch.float64)

    def to_list(self, t):
        return t.tolist()

    @staticmethod
    def _arr(x, ext):
        return x.numpy().reshape(tuple(reversed(ext)))

    def copy_box(self, src, ext, boff, dst, pos, bext):
        a = self._arr(src, ext)
        sl = tuple(slice(o, o + e) for o, e in zip(reversed(boff), reversed(bext)))
        blk = a[sl].ravel()
        dst[pos:pos + blk.size] = torch.from_numpy(np.ascontiguousarray(blk))

    def copy_box_into(self, src, pos, bext, dst, ext, doff):
        n = math.prod(bext)
        blk = src[pos:pos + n].numpy().reshape(tuple(reversed(bext)))
        a = self._arr(dst, ext)
        sl = tuple(slice(o, o + e) for o, e in zip(reversed(doff), reversed(bext)))
        a[sl] = blk

    def copy_range(self, src, spos, dst, dpos, n):
        if n > 0:
            dst[dpos:dpos + n] = src[spos:spos + n]

    # -- operators
    def pass_(self, axis, mode, x, ext, off):
        from oracle import operators
        d = len(ext)
        a = self._arr(x, ext).copy()
        Q = self.s[axis].Qt
        if mode == "fwd":
            a = operators.apply_along(Q.T, a, axis + 1)
        elif mode == "bwd":
            a = operators.apply_along(Q, a, axis + 1)
        else:
            a = operators.apply_along(Q.T, a, axis + 1)
            den = np.zeros(a.shape)
            for k in range(d):
                lam = self.s[k].lamt[off[k]:off[k] + ext[k]]
                sh = [1] * d
                sh[d - 1 - k] = lam.size
                den = den + lam.reshape(sh)
            a = operators.apply_along(Q, a / den, axis + 1)
        x[:] = torch.from_numpy(np.ascontiguousarray(a).ravel())
        return x

    def slab_stiffness(self, z0, nz, u_ext):
        from oracle import operators
        d = len(self.s)
        L = d - 1
        m = self.s[L].M.shape[0]
        e0, e1 = max(0, z0 - self.p), min(m, z0 + nz + self.p)
        plane = u_ext.numel() // (e1 - e0)
        shape_ext = (e1 - e0,) + tuple(s.M.shape[0] for s in reversed(self.s[:L]))
        u = u_ext.numpy().reshape(shape_ext)
        ML, KL = self.s[L].M[z0:z0 + nz, e0:e1], self.s[L].K[z0:z0 + nz, e0:e1]
        T1 = operators.apply_along(ML, u, d)
        T2 = operators.apply_along(KL, u, d)
        out = np.zeros(T1.shape)
        for k in range(L):  # the directions inside the slab
            mats = [self.s[j].K if j == k else self.s[j].M for j in range(L)]
            out += operators.kron_apply(mats, T1)
        out += operators.kron_apply([self.s[j].M for j in range(L)], T2)
        assert out.size == plane * nz
        return torch.from_numpy(out.ravel())

    def dot(self, a, b):
        return float(np.dot(a.numpy(), b.numpy()))

    def axpby(self, a, x, b, y):
        y.mul_(b).add_(x, alpha=a)


# (d, n, p, Dirichlet sets per direction): thin slabs (world 4 on m = 13, p = 5:
# the halo spans several ranks), 2D, mixed boundary conditions
CASES = [
    (3, 12, 3, None),
    (3, 10, 5, None),
    (2, 20, 4, None),
    (3, 11, 4, ((1, 0), (1, 1), (0, 1))),
]


def _dset(pair):
    return tuple(k for k, v in zip((0, 1), pair) if v)


def _worker(rank, world, port, case, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import operators, splitting
        from paper_2512_20269_gb300 import inputs
        from paper_2512_20269_gb300.slab import SlabPartition, SlabSolver, TorchComm
        d, n, p, dirichlet = case
        D = dirichlet or [(1, 1)] * d
        splits = [splitting.axis_split(n, p, _dset(pair)) for pair in D]
        m = [s.M.shape[0] for s in splits]
        shape = tuple(reversed(m))
        part = SlabPartition(m, world)
        solver = SlabSolver(OracleBackend(splits, p), part, TorchComm())
        z0, z1 = part.z[rank]
        loc = lambda a: torch.from_numpy(np.ascontiguousarray(a[z0:z1]).ravel())

        r = inputs.rhs(shape, "normal", seed=11)
        z_ref = operators.iffd_apply(r, splits)
        z = solver.apply_preconditioner(loc(r)).numpy()
        e_pre = float(np.abs(z - z_ref[z0:z1].ravel()).max() / np.abs(z_ref).max())

        u = inputs.rhs(shape, "uniform", seed=12)
        MK = [(s.M, s.K) for s in splits]
        Au_ref = operators.stiffness_apply(u, MK)
        Au = solver.apply_stiffness(loc(u)).numpy()
        e_stiff = float(np.abs(Au - Au_ref[z0:z1].ravel()).max() / np.abs(Au_ref).max())

        f = inputs.rhs(shape, "normal", seed=13)
        u_ref, it_ref, _ = operators.pcg(f, lambda v: operators.stiffness_apply(v, MK),
                                         lambda v: operators.iffd_apply(v, splits), rtol=1e-8)
        us, info = solver.pcg_solve(loc(f))
        e_pcg = float(np.abs(us.numpy() - u_ref[z0:z1].ravel()).max() / np.abs(u_ref).max())
        q.put((rank, e_pre, e_stiff, e_pcg, info["iters"], it_ref, info["status"]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("case", CASES)
def test_slab_decomposition_reproduces_single_rank_oracle(world, case):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=300) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert sorted(r[0] for r in res) == list(range(world))
    for rank, e_pre, e_stiff, e_pcg, it, it_ref, status in res:
        assert e_pre <= 1e-12, (rank, e_pre)
        assert e_stiff <= 1e-13, (rank, e_stiff)
        assert status == 0 and it == it_ref, (rank, it, it_ref)
        assert e_pcg <= 1e-10, (rank, e_pcg)


def test_partition_and_halo_ranges():
    from paper_2512_20269_gb300.slab import SlabPartition, halo_ranges, split
    assert split(10, 4) == [(0, 3), (3, 6), (6, 8), (8, 10)]
    P = SlabPartition((7, 9, 13), 4)
    assert P.z == split(13, 4) and P.t == split(9, 4)
    # every rank sends every other rank exactly the L-rows it owns and T-rows the receiver owns
    tot = sum(P.block_elems(r, s) for r in range(4) for s in range(4))
    assert tot == 7 * 9 * 13
    # halo: rank 1 owns [4, 7); with p = 5 it needs rows [0, 12) -> from 0: [0, 4), from 2: [7, 10), from 3: [10, 12)
    assert [halo_ranges(P, 5, 1, s) for s in range(4)] == [(0, 4), (0, 0), (7, 10), (10, 12)]
    assert halo_ranges(P, 1, 0, 3) == (0, 0)
    with pytest.raises(ValueError):
        SlabPartition((4, 3, 8), 4)  # fewer rows of T than ranks
