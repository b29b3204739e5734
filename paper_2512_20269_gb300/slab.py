"""Slab-decomposed IFFD-PCG of one problem over several GPUs (one process per
GPU, torch.distributed for the exchanges).

The grid is split into slabs along its slowest direction L = d - 1: rank r
owns the rows [z0_r, z1_r) of that direction (all of the others). Then:

* Preconditioner (eq. "preconditioner"): the forward passes along the
  directions 0 .. d - 2 run on each rank's slab as they are (their pencils lie
  inside the slab). One all-to-all then re-splits the data along direction
  T = d - 2 so that every rank holds whole pencils along L (rank s owns rows
  [t0_s, t1_s) of T); the fused pass (Q~^T, the eigenvalue scaling, Q~ along L)
  runs there, its box offset placing it among the eigenvalues of T; a second
  all-to-all restores the slabs and the backward passes follow. The received
  blocks of the first exchange are already in the layout of the re-split
  array; the second exchange's blocks are written into the slab by box copies.
* Stiffness (eq. "system_matrix"): each rank receives from the ranks that own
  them the up to p rows on each side of its slab that the banded sweep along
  L reads (the halo), then applies A^ to its rows (iffd_slab_stiffness).
* PCG (Section 3): vectors stay distributed; every inner product is the sum of
  the ranks' deterministic partial dot products (an all-reduce). The products
  (r, r) and (r, z) of one iteration travel in one all-reduce, so an
  iteration takes two.

There is no collective inside a kernel: the ranks exchange data only between
launches, through the communicator. The local steps go through a backend
object: GpuBackend runs them with the library's kernels (C ABI, CUDA tensors);
the CPU tests give a backend built from the oracle's 1D operators, which checks
the partition and exchange logic on gloo ranks without a GPU.
"""

from __future__ import annotations

import ctypes
import math


def split(n: int, parts: int):
    """Balanced contiguous split of range(n) into `parts` ranges [a, b)."""
    q, r = divmod(n, parts)
    out, a = [], 0
    for k in range(parts):
        b = a + q + (1 if k < r else 0)
        out.append((a, b))
        a = b
    return out


class SlabPartition:
    """Slabs of an (m_0, .., m_{d-1}) grid (direction 0 fastest) over `size`
    ranks: rows of the slowest direction L (the resting layout) and rows of
    direction T = d - 2 (the layout of the fused pass)."""

    def __init__(self, m, size: int):
        self.m = tuple(int(v) for v in m)
        self.d = len(self.m)
        if self.d not in (2, 3):
            raise ValueError("d must be 2 or 3")
        self.size = size
        self.L, self.T = self.d - 1, self.d - 2
        if self.m[self.L] < size or self.m[self.T] < size:
            raise ValueError("every rank needs at least one row in both splits")
        self.z = split(self.m[self.L], size)
        self.t = split(self.m[self.T], size)

    def plane(self) -> int:
        return math.prod(self.m[:self.L])

    def slab_shape(self, r: int):
        """Resting layout of rank r: numpy shape (rows of L, .., m_0)."""
        z0, z1 = self.z[r]
        return (z1 - z0,) + tuple(reversed(self.m[:self.L]))

    def slab_box(self, r: int):
        """(extent, offset) per direction of rank r's slab, direction 0 first."""
        z0, z1 = self.z[r]
        ext = list(self.m[:self.L]) + [z1 - z0]
        off = [0] * self.L + [z0]
        return ext, off

    def tbox(self, s: int):
        """(extent, offset) of rank s's box in the fused-pass layout: rows
        [t0, t1) of direction T, whole pencils along L."""
        t0, t1 = self.t[s]
        ext = list(self.m)
        ext[self.T] = t1 - t0
        off = [0] * self.d
        off[self.T] = t0
        return ext, off

    def block_elems(self, r: int, s: int) -> int:
        """Elements rank r sends to rank s in the forward re-split: rows of L
        owned by r, rows of T owned by s."""
        z0, z1 = self.z[r]
        t0, t1 = self.t[s]
        other = math.prod(self.m[:self.T])
        return other * (t1 - t0) * (z1 - z0)



def halo_ranges(part: SlabPartition, p: int, r: int, s: int):
    """Rows [a, b) of the slowest direction that rank s sends to rank r for
    the banded sweep of A^ on r's rows (empty: a == b). r needs the rows
    [z0 - p, z1 + p) clipped to the grid; s owns [z0_s, z1_s)."""
    if r == s:
        return (0, 0)
    z0, z1 = part.z[r]
    lo, hi = max(0, z0 - p), min(part.m[part.L], z1 + p)
    a, b = max(lo, part.z[s][0]), min(hi, part.z[s][1])
    return (a, b) if a < b else (0, 0)


class TorchComm:
    """Exchanges through torch.distributed (NCCL for CUDA tensors, gloo for
    CPU tensors): all_to_all_single with uneven splits and a sum all-reduce."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def alltoall(self, out, inp, out_splits, in_splits):
        self.dist.all_to_all_single(out, inp, out_splits, in_splits, group=self.group)

    def allreduce_sum(self, t):
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)


class SlabSolver:
    """Preconditioner, stiffness and PCG of one problem split over the ranks of
    `comm` (see the module docstring). `backend` provides the local steps on
    this rank's data; vectors are flat arrays of the backend's type holding the
    rank's slab in the resting layout."""

    def __init__(self, backend, part: SlabPartition, comm):
        if part.size != comm.size:
            raise ValueError("partition and communicator sizes differ")
        self.be, self.part, self.comm = backend, part, comm
        self.rank = comm.rank
        self.p = backend.p

    # ---------------------------------------------------------------- helpers
    def _exchange(self, send, sizes_out, sizes_in):
        recv = self.be.empty(sum(sizes_in))
        self.comm.alltoall(recv, send, list(sizes_in), list(sizes_out))
        return recv

    def _allreduce(self, vals):
        t = self.be.host_vector(vals)
        self.comm.allreduce_sum(t)
        return [float(v) for v in self.be.to_list(t)]

    # ---------------------------------------------------------- preconditioner
    def apply_preconditioner(self, r_loc):
        """z = P^{-1} r on this rank's slab."""
        P, be, me = self.part, self.be, self.rank
        ext, off = P.slab_box(me)
        t = be.copy(r_loc)
        for a in range(P.L):
            t = be.pass_(a, "fwd", t, ext, off)
        # forward re-split: rank s gets rows T in [t0_s, t1_s) of this slab
        send = be.empty(sum(P.block_elems(me, s) for s in range(P.size)))
        pos = 0
        for s in range(P.size):
            n = P.block_elems(me, s)
            bext = list(ext)
            bext[P.T] = P.t[s][1] - P.t[s][0]
            boff = [0] * P.d
            boff[P.T] = P.t[s][0]
            be.copy_box(t, ext, boff, send, pos, bext)
            pos += n
        sizes_out = [P.block_elems(me, s) for s in range(P.size)]
        sizes_in = [P.block_elems(r, me) for r in range(P.size)]
        y = self._exchange(send, sizes_out, sizes_in)  # blocks of L rows in rank order: the fused-pass layout
        text, toff = P.tbox(me)
        y = be.pass_(P.L, "fused", y, text, toff)
        # backward re-split: the rows of L owned by rank r go back to r
        back = self._exchange(y, sizes_in, sizes_out)
        z = be.empty(len_of(ext))
        pos = 0
        for s in range(P.size):
            bext = list(ext)
            bext[P.T] = P.t[s][1] - P.t[s][0]
            doff = [0] * P.d
            doff[P.T] = P.t[s][0]
            be.copy_box_into(back, pos, bext, z, ext, doff)
            pos += sizes_out[s]
        for a in reversed(range(P.L)):
            z = be.pass_(a, "bwd", z, ext, off)
        return z

    # ---------------------------------------------------------------- stiffness
    def apply_stiffness(self, u_loc):
        """A^ u on this rank's rows of the slowest direction."""
        P, be, me, p = self.part, self.be, self.rank, self.p
        plane = P.plane()
        z0, z1 = P.z[me]
        # rows this rank sends to each rank r, and receives from each rank s
        out_rng = [halo_ranges(P, p, r, me) for r in range(P.size)]
        in_rng = [halo_ranges(P, p, me, s) for s in range(P.size)]
        sizes_out = [(b - a) * plane for a, b in out_rng]
        sizes_in = [(b - a) * plane for a, b in in_rng]
        send = be.empty(sum(sizes_out))
        pos = 0
        for (a, b), n in zip(out_rng, sizes_out):
            if n:
                be.copy_range(u_loc, (a - z0) * plane, send, pos, n)
            pos += n
        recv = self._exchange(send, sizes_out, sizes_in)
        e0, e1 = max(0, z0 - p), min(P.m[P.L], z1 + p)
        u_ext = be.empty((e1 - e0) * plane)
        be.copy_range(u_loc, 0, u_ext, (z0 - e0) * plane, (z1 - z0) * plane)
        pos = 0
        for (a, b), n in zip(in_rng, sizes_in):
            if n:
                be.copy_range(recv, pos, u_ext, (a - e0) * plane, n)
            pos += n
        return be.slab_stiffness(z0, z1 - z0, u_ext)

    # --------------------------------------------------------------------- PCG
    def pcg_solve(self, f_loc, rtol: float = 1e-8, maxit: int = 500):
        """Textbook PCG (Section 3), zero start, stop at ||r|| <= rtol ||f||.
        Returns (u_loc, info) with info iters, rel_res, status (0, or 6 when
        maxit was reached, 7 on breakdown)."""
        be = self.be
        u = be.zeros_like(f_loc)
        r = be.copy(f_loc)
        (ff,) = self._allreduce([be.dot(f_loc, f_loc)])
        if ff == 0.0:
            return u, {"iters": 0, "rel_res": 0.0, "status": 0}
        z = self.apply_preconditioner(r)
        (rz,) = self._allreduce([be.dot(r, z)])
        if not (rz > 0.0) or not math.isfinite(rz):
            return u, {"iters": 0, "rel_res": 1.0, "status": 7}
        pvec = be.copy(z)
        rr = ff
        for it in range(1, maxit + 1):
            q = self.apply_stiffness(pvec)
            (pq,) = self._allreduce([be.dot(pvec, q)])
            if not (pq > 0.0) or not math.isfinite(pq):
                return u, {"iters": it, "rel_res": math.sqrt(rr / ff), "status": 7}
            alpha = rz / pq
            be.axpby(alpha, pvec, 1.0, u)
            be.axpby(-alpha, q, 1.0, r)
            z = self.apply_preconditioner(r)
            rr, rz_new = self._allreduce([be.dot(r, r), be.dot(r, z)])
            if not math.isfinite(rr):
                return u, {"iters": it, "rel_res": float("nan"), "status": 7}
            if rr <= rtol * rtol * ff:
                return u, {"iters": it, "rel_res": math.sqrt(rr / ff), "status": 0}
            if not (rz_new > 0.0):
                return u, {"iters": it, "rel_res": math.sqrt(rr / ff), "status": 7}
            beta = rz_new / rz
            rz = rz_new
            be.axpby(1.0, z, beta, pvec)  # p = z + beta p
        return u, {"iters": maxit, "rel_res": math.sqrt(rr / ff), "status": 6}


def len_of(ext) -> int:
    return math.prod(ext)


class GpuBackend:
    """The local steps of SlabSolver with the library's kernels on CUDA
    tensors (float64, flat): transform passes (iffd_apply_pass), the slab
    stiffness (iffd_slab_stiffness), box and range copies (iffd_copy_box),
    inner products (iffd_vec_dot) and vector updates (iffd_vec_axpby). The plan
    is the global problem's (its 1D tables); `zmax` bounds the slab rows."""

    def __init__(self, plan, zmax: int, stream=None):
        import torch

        from . import _lib
        from ._lib import check
        self.torch, self.lib, self.check = torch, _lib.load(), check
        self.plan, self.p = plan, plan.p
        self.stream = stream
        nb = ctypes.c_size_t()
        check(self.lib.iffd_slab_workspace_bytes(plan._h, int(zmax), ctypes.byref(nb)), "iffd_slab_workspace_bytes")
        self._ws = torch.empty(nb.value + 256, dtype=torch.uint8, device="cuda")
        self._wsp = (int(self._ws.data_ptr()) + 255) // 256 * 256
        check(self.lib.iffd_vec_dot_workspace_bytes(ctypes.byref(nb)), "iffd_vec_dot_workspace_bytes")
        self._dws = torch.empty(nb.value // 8 + 1, dtype=torch.float64, device="cuda")
        self._dot = torch.empty(1, dtype=torch.float64, device="cuda")

    def _st(self):
        s = self.stream or self.torch.cuda.current_stream()
        return int(s.cuda_stream)

    @staticmethod
    def _i3(v):
        """Extents, direction 0 first, padded with 1 to three directions."""
        v = list(v) + [1] * (3 - len(v))
        return (ctypes.c_int * 3)(*v)

    @staticmethod
    def _o3(v):
        """Offsets, padded with 0 to three directions."""
        v = list(v) + [0] * (3 - len(v))
        return (ctypes.c_int * 3)(*v)

    def empty(self, n):
        return self.torch.empty(int(n), dtype=self.torch.float64, device="cuda")

    def zeros_like(self, x):
        return self.torch.zeros_like(x)

    def copy(self, x):
        y = self.empty(x.numel())
        self.copy_range(x, 0, y, 0, x.numel())
        return y

    def host_vector(self, vals):
        return self.torch.tensor(vals, dtype=self.torch.float64, device="cuda")

    def to_list(self, t):
        return t.cpu().tolist()

    def pass_(self, axis, mode, x, ext, off):
        m = {"fwd": 0, "bwd": 1, "fused": 2}[mode]
        self.check(self.lib.iffd_apply_pass(self.plan._h, axis, m, self._i3(ext), self._o3(off), int(x.data_ptr()),
                                            int(x.data_ptr()), self._st()), "iffd_apply_pass")
        return x

    def copy_box(self, src, ext, boff, dst, pos, bext):
        """dst[pos:] <- the box (offset boff, extent bext) of src (extent ext)."""
        self.check(self.lib.iffd_copy_box(int(src.data_ptr()), self._i3(ext), self._o3(boff),
                                          int(dst.data_ptr()) + 8 * pos, self._i3(bext), self._o3([]),
                                          self._i3(bext), self._st()), "iffd_copy_box")

    def copy_box_into(self, src, pos, bext, dst, ext, doff):
        """The box (extent ext, offset doff) of dst <- src[pos:] (extent bext)."""
        self.check(self.lib.iffd_copy_box(int(src.data_ptr()) + 8 * pos, self._i3(bext), self._o3([]),
                                          int(dst.data_ptr()), self._i3(ext), self._o3(doff), self._i3(bext),
                                          self._st()), "iffd_copy_box")

    def copy_range(self, src, spos, dst, dpos, n):
        if n <= 0:
            return
        dims = self._i3([n])
        zero = self._o3([])
        self.check(self.lib.iffd_copy_box(int(src.data_ptr()) + 8 * spos, dims, zero, int(dst.data_ptr()) + 8 * dpos,
                                          dims, zero, dims, self._st()), "iffd_copy_box")

    def slab_stiffness(self, z0, nz, u_ext):
        out = self.empty(self.part_plane() * nz)
        self.check(self.lib.iffd_slab_stiffness(self.plan._h, int(z0), int(nz), int(u_ext.data_ptr()),
                                                int(out.data_ptr()), self._wsp, self._st()), "iffd_slab_stiffness")
        return out

    def part_plane(self):
        return math.prod(self.plan.m[:-1])

    def dot(self, a, b):
        self.check(self.lib.iffd_vec_dot(int(a.data_ptr()), int(b.data_ptr()), a.numel(), int(self._dot.data_ptr()),
                                         int(self._dws.data_ptr()), self._st()), "iffd_vec_dot")
        return float(self._dot.item())

    def axpby(self, a, x, b, y):
        self.check(self.lib.iffd_vec_axpby(y.numel(), float(a), int(x.data_ptr()), float(b), int(y.data_ptr()),
                                           self._st()), "iffd_vec_axpby")
