"""GB300 (sm_103a) IFFD-preconditioned PCG for the B-spline Galerkin Poisson system.

The compute path is the C ABI of ``libiffd.so`` (include/iffd.h): hand-written
CUDA passes for the IFFD preconditioner, the Kronecker stiffness and the PCG
vector updates. This package only marshals arguments; PyTorch provides device
memory and streams. There is no CPU fallback.
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import IFFDError, check, iffd_options, iffd_pcg_info

PRECISION = {"fp64": 0, "fp32": 1}
PRECOND = {"iffd": 0, "exact_fd": 1, "none": 2}
COEF = {"const": 0, "sin": 1}

__all__ = ["IFFDPlan", "IFFDEngine", "IFFDError", "batch_solve", "host_axis", "measure_peak", "PRECISION",
           "PRECOND"]


def _ptr(t) -> int:
    return int(t.data_ptr())


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def host_transform(n: int, p: int, precision: str = "fp64", dirichlet=(1, 1)) -> dict:
    """How the transform passes of one direction run (library's host planner,
    no GPU): DFT length L, FFT length F (F > L: Bluestein), pencils per tile."""
    lib = _lib.load()
    dir_arr = (ctypes.c_int * 2)(*dirichlet)
    L, F, pp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(lib.iffd_host_transform(n, p, dir_arr, PRECISION[precision], ctypes.byref(L), ctypes.byref(F),
                                  ctypes.byref(pp)), "iffd_host_transform")
    return {"L": L.value, "F": F.value, "bluestein": F.value > L.value, "pencils": pp.value}


def _rep_pairs(rep) -> list:
    """{knot: extra} or [(knot, extra), ...] -> flat [knot, extra, ...]."""
    items = sorted(rep.items()) if isinstance(rep, dict) else [tuple(t) for t in (rep or [])]
    return [int(v) for kv in items for v in kv]


def host_axis(n: int, p: int, dirichlet=(1, 1), rep=None) -> dict:
    """1D tables of one direction computed by the library's host setup (no GPU).
    `rep` = {knot: extra}: breakpoint knot/n repeated `extra` more times
    (reduced regularity)."""
    lib = _lib.load()
    dir_arr = (ctypes.c_int * 2)(*dirichlet)
    flat = _rep_pairs(rep)
    nrep = len(flat) // 2
    rep_arr = (ctypes.c_int * max(1, len(flat)))(*flat)
    m, nr, no = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(lib.iffd_host_axis_knots(n, p, dir_arr, nrep, rep_arr, ctypes.byref(m), ctypes.byref(nr),
                                   ctypes.byref(no), None, None, None, None, None, None), "iffd_host_axis_knots")
    m, nr, no = m.value, nr.value, no.value
    bw = 2 * p + 1
    out = {"m": m, "n_reg": nr, "n_out": no,
           "M_band": np.zeros(m * bw), "K_band": np.zeros(m * bw), "lam": np.zeros(m),
           "dtilde": np.zeros(nr), "V_reg": np.zeros(m * nr), "W": np.zeros(max(1, m * no))}
    dp = lambda a: a.ctypes.data_as(_lib.c_double_p)
    check(lib.iffd_host_axis_knots(n, p, dir_arr, nrep, rep_arr, None, None, None, dp(out["M_band"]),
                                   dp(out["K_band"]), dp(out["lam"]), dp(out["dtilde"]), dp(out["V_reg"]),
                                   dp(out["W"])), "iffd_host_axis_knots")
    out["M_band"] = out["M_band"].reshape(m, bw)
    out["K_band"] = out["K_band"].reshape(m, bw)
    out["V_reg"] = out["V_reg"].reshape(m, nr)
    out["W"] = out["W"][:m * no].reshape(m, no)
    return out


def host_quad_axis(n: int, p: int, dirichlet=(1, 1), rep=None) -> dict:
    """Gauss points, weights and the dense value / derivative matrices of the
    kept B-splines at them, from the tables the general-coefficient operator
    uses (iffd_host_quad_axis; no GPU)."""
    lib = _lib.load()
    dir_arr = (ctypes.c_int * 2)(*dirichlet)
    flat = _rep_pairs(rep)
    rep_arr = (ctypes.c_int * max(1, len(flat)))(*flat)
    nq, m = ctypes.c_int(), ctypes.c_int()
    check(lib.iffd_host_quad_axis(n, p, dir_arr, len(flat) // 2, rep_arr, ctypes.byref(nq), ctypes.byref(m), None,
                                  None, None, None), "iffd_host_quad_axis")
    nq, m = nq.value, m.value
    out = {"x": np.zeros(nq), "w": np.zeros(nq), "B": np.zeros(nq * m), "D": np.zeros(nq * m)}
    dp = lambda a: a.ctypes.data_as(_lib.c_double_p)
    check(lib.iffd_host_quad_axis(n, p, dir_arr, len(flat) // 2, rep_arr, None, None, dp(out["x"]), dp(out["w"]),
                                  dp(out["B"]), dp(out["D"])), "iffd_host_quad_axis")
    out["B"] = out["B"].reshape(nq, m)
    out["D"] = out["D"].reshape(nq, m)
    return out


def measure_peak(kind: str = "fp64", stream=None) -> dict:
    """FMA rate of the current GPU (iffd_measure_peak): kind "fp64", "fp32" or
    "fp32x2" (packed pairs);
    returns {"tflops": ..., "sm_count": ...}."""
    lib = _lib.load()
    sms, tf = ctypes.c_int(), ctypes.c_double()
    check(lib.iffd_measure_peak({"fp64": 0, "fp32": 1, "fp32x2": 2}[kind], _stream_handle(stream), ctypes.byref(sms),
                                ctypes.byref(tf)), "iffd_measure_peak")
    return {"tflops": tf.value, "sm_count": sms.value}


class IFFDPlan:
    """One problem (d, n per direction, p, boundary conditions) on the current CUDA device.

    Vectors are float64 CUDA tensors of N = prod(m_k) entries, direction 1 (x)
    fastest; a tensor of shape (m_d, ..., m_1) in C order has that layout.
    `dirichlet`: one (at x_k = 0, at x_k = 1) flag pair per direction, 1 for
    homogeneous Dirichlet data, 0 for the natural condition (default: Dirichlet
    on every face). `knots`: per direction, None or {knot: extra} repeated
    interior breakpoints (reduced regularity, iffd_setup_knots).
    """

    def __init__(self, d: int, n, p: int, precision: str = "fp64", precond: str = "iffd", rtol: float = 1e-8,
                 maxit: int = 500, true_residual: bool = True, flexible: bool = False, coef: str = "const",
                 coef_amp: float = 0.5, stream=None, dirichlet=None, knots=None):
        import torch
        self._lib = _lib.load()
        n = [int(n)] * d if np.isscalar(n) else [int(x) for x in n]
        self.d, self.n, self.p = d, n, p
        opt = iffd_options()
        self._lib.iffd_default_options(ctypes.byref(opt))
        opt.precision = PRECISION[precision]
        opt.precond = PRECOND[precond]
        opt.rtol = rtol
        opt.maxit = maxit
        opt.true_residual = int(true_residual)
        opt.flexible = int(flexible)
        opt.coef = COEF[coef]
        opt.coef_amp = coef_amp
        self.options = opt
        nn = (ctypes.c_int * d)(*n)
        flags = [1] * (2 * d) if dirichlet is None else [int(v) for pair in dirichlet for v in pair]
        if len(flags) != 2 * d:
            raise ValueError("dirichlet needs one (x=0, x=1) pair per direction")
        self.dirichlet = [tuple(flags[2 * k:2 * k + 2]) for k in range(d)]
        dd = (ctypes.c_int * (2 * d))(*flags)
        h = ctypes.c_void_p()
        if knots is None:
            check(self._lib.iffd_setup(d, nn, p, dd, ctypes.byref(opt), _stream_handle(stream), ctypes.byref(h)),
                  "iffd_setup")
        else:
            if len(knots) != d:
                raise ValueError("knots needs one entry per direction")
            flat = [_rep_pairs(k) for k in knots]
            nrep = (ctypes.c_int * d)(*[len(f) // 2 for f in flat])
            allp = [v for f in flat for v in f]
            reps = (ctypes.c_int * max(1, len(allp)))(*allp)
            check(self._lib.iffd_setup_knots(d, nn, p, dd, nrep, reps, ctypes.byref(opt), _stream_handle(stream),
                                             ctypes.byref(h)), "iffd_setup_knots")
        self.knots = knots
        self._h = h
        self.m = []
        for a in range(d):
            m, nr, no = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            check(self._lib.iffd_get_dims(h, a, ctypes.byref(m), ctypes.byref(nr), ctypes.byref(no)), "iffd_get_dims")
            self.m.append(m.value)
        self.N = int(np.prod(self.m))
        self.shape = tuple(reversed(self.m))
        nb = ctypes.c_size_t()
        check(self._lib.iffd_workspace_bytes(h, ctypes.byref(nb)), "iffd_workspace_bytes")
        self.workspace_bytes = nb.value
        self._ws = torch.empty(nb.value + 256, dtype=torch.uint8, device="cuda")
        self._ws_ptr = (_ptr(self._ws) + 255) // 256 * 256

    # -- helpers
    def _check_vec(self, t, name):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                and t.numel() == self.N):
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor with {self.N} entries")

    def empty(self):
        import torch
        return torch.empty(self.shape, dtype=torch.float64, device="cuda")

    def get_1d(self, axis: int) -> dict:
        """Host copies of the 1D tables of direction `axis` (iffd_get_1d):
        banded M and K, Lambda~, D~_reg, dense V_reg (m x n_reg) and
        W = V_out Q_out (m x n_out)."""
        m, nr, no = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(self._lib.iffd_get_dims(self._h, axis, ctypes.byref(m), ctypes.byref(nr), ctypes.byref(no)),
              "iffd_get_dims")
        m, nr, no = m.value, nr.value, no.value
        bw = 2 * self.p + 1
        out = {"M_band": np.zeros(m * bw), "K_band": np.zeros(m * bw), "lam": np.zeros(m),
               "dtilde": np.zeros(nr), "V_reg": np.zeros(m * nr), "W": np.zeros(max(1, m * no))}
        dp = lambda a: a.ctypes.data_as(_lib.c_double_p)
        check(self._lib.iffd_get_1d(self._h, axis, dp(out["M_band"]), dp(out["K_band"]), dp(out["lam"]),
                                    dp(out["dtilde"]), dp(out["V_reg"]), dp(out["W"])), "iffd_get_1d")
        out["M_band"] = out["M_band"].reshape(m, bw)
        out["K_band"] = out["K_band"].reshape(m, bw)
        out["V_reg"] = out["V_reg"].reshape(m, nr)
        out["W"] = out["W"][:m * no].reshape(m, no)
        return out

    # -- C ABI calls
    def iffd_apply_preconditioner(self, r, z=None, stream=None):
        z = self.empty() if z is None else z
        self._check_vec(r, "r")
        self._check_vec(z, "z")
        check(self._lib.iffd_apply_preconditioner(self._h, _ptr(r), _ptr(z), self._ws_ptr, _stream_handle(stream)),
              "iffd_apply_preconditioner")
        return z

    def iffd_apply_stiffness(self, u, Au=None, stream=None):
        Au = self.empty() if Au is None else Au
        self._check_vec(u, "u")
        self._check_vec(Au, "Au")
        check(self._lib.iffd_apply_stiffness(self._h, _ptr(u), _ptr(Au), self._ws_ptr, _stream_handle(stream)),
              "iffd_apply_stiffness")
        return Au

    def iffd_pcg_solve(self, f, u=None, stream=None, raise_on_error: bool = True):
        u = self.empty() if u is None else u
        self._check_vec(f, "f")
        self._check_vec(u, "u")
        info = iffd_pcg_info()
        rc = self._lib.iffd_pcg_solve(self._h, _ptr(f), _ptr(u), self._ws_ptr, _stream_handle(stream),
                                      ctypes.byref(info))
        if raise_on_error:
            check(rc, "iffd_pcg_solve")
        return u, {"iters": info.iters, "rel_res": info.rel_res, "true_rel_res": info.true_rel_res,
                   "status": info.status}

    def iffd_apply_stiffness_noalloc(self, u, Au, stream=None):
        """A^ u without a workspace (static scratch inside the library, for
        callers that cannot allocate; problems up to IFFD_NOALLOC_MAX_DOFS)."""
        self._check_vec(u, "u")
        self._check_vec(Au, "Au")
        check(self._lib.iffd_apply_stiffness_noalloc(self._h, _ptr(u), _ptr(Au), _stream_handle(stream)),
              "iffd_apply_stiffness_noalloc")
        return Au

    # -- general coefficient: stiffness of -div(C grad u) at the Gauss points
    def quad_points(self, axis: int):
        """Gauss points and weights of one direction on [0, 1] (iffd_quad_points)."""
        nq = ctypes.c_int()
        check(self._lib.iffd_quad_points(self._h, axis, ctypes.byref(nq), None, None), "iffd_quad_points")
        x = np.empty(nq.value)
        w = np.empty(nq.value)
        check(self._lib.iffd_quad_points(self._h, axis, None, x.ctypes.data_as(_lib.c_double_p),
                                         w.ctypes.data_as(_lib.c_double_p)), "iffd_quad_points")
        return x, w

    @property
    def quad_shape(self):
        """Shape of one coefficient component: (nq_{d-1}, ..., nq_0), x fastest."""
        if getattr(self, "_quad_shape", None) is None:
            self._quad_shape = tuple(self.quad_points(a)[0].size for a in reversed(range(self.d)))
        return self._quad_shape

    def _gws(self):
        import torch
        if getattr(self, "_gws_buf", None) is None:
            nb = ctypes.c_size_t()
            check(self._lib.iffd_general_workspace_bytes(self._h, ctypes.byref(nb)), "iffd_general_workspace_bytes")
            self._gws_buf = torch.empty(nb.value + 256, dtype=torch.uint8, device="cuda")
        return (_ptr(self._gws_buf) + 255) // 256 * 256

    def _check_coef(self, C):
        import torch
        if not (C.is_cuda and C.dtype == torch.float64 and C.is_contiguous()):
            raise ValueError("C must be a contiguous float64 CUDA tensor")
        nq = int(np.prod(self.quad_shape))
        ncomp = C.numel() // nq
        if ncomp * nq != C.numel():
            raise ValueError(f"C must hold ncomp x {self.quad_shape} values")
        return ncomp

    def iffd_apply_stiffness_general(self, C, u, Au=None, stream=None):
        """Au = A_C u; C of shape (ncomp,) + quad_shape, ncomp 1 (scalar) or
        d (d + 1) / 2 (upper triangle of the symmetric tensor, row by row)."""
        Au = self.empty() if Au is None else Au
        self._check_vec(u, "u")
        self._check_vec(Au, "Au")
        ncomp = self._check_coef(C)
        check(self._lib.iffd_apply_stiffness_general(self._h, _ptr(C), ncomp, _ptr(u), _ptr(Au), self._gws(),
                                                     _stream_handle(stream)), "iffd_apply_stiffness_general")
        return Au

    def iffd_pcg_solve_general(self, C, f, u=None, stream=None, raise_on_error: bool = True):
        """PCG on A_C u = f with the plan's IFFD preconditioner."""
        u = self.empty() if u is None else u
        self._check_vec(f, "f")
        self._check_vec(u, "u")
        ncomp = self._check_coef(C)
        info = iffd_pcg_info()
        rc = self._lib.iffd_pcg_solve_general(self._h, _ptr(C), ncomp, _ptr(f), _ptr(u), self._ws_ptr, self._gws(),
                                              _stream_handle(stream), ctypes.byref(info))
        if raise_on_error:
            check(rc, "iffd_pcg_solve_general")
        return u, {"iters": info.iters, "rel_res": info.rel_res, "true_rel_res": info.true_rel_res,
                   "status": info.status}

    apply_stiffness_general = iffd_apply_stiffness_general
    pcg_solve_general = iffd_pcg_solve_general

    # -- profiling (CUDA events around every launch of this plan)
    KERNEL_KINDS = 12

    def autotune(self, stream=None):
        """Tune tiles and radix sequences on this GPU (iffd_autotune; uses the
        plan's workspace, synchronizes the stream)."""
        check(self._lib.iffd_autotune(self._h, self._ws_ptr, _stream_handle(stream)), "iffd_autotune")
        return self

    def set_geometry(self, axis: int, pencils_transform: int = 0, pencils_stiffness: int = 0, pipelined=None,
                     warp: bool = False, double_float: bool = False, paired: bool = False):
        """Set one direction's launch geometry by hand (iffd_set_geometry).
        `warp`: run the warp-FFT transform pass (its tile is fixed; the FP32
        default where eligible, opt-in for FP64 plans up to FFT length 256).
        `paired`: the FP32 warp-FFT pass with two sequences per lane group
        (FFT length up to 256; the FP32 default there); `warp` alone selects
        the unpaired pass.
        `double_float`: FP64 plans, every transform pass in double-float
        arithmetic on the FP32 pipe (the default where every direction has a
        warp-FFT pass; any other FP64 transform geometry set here turns it off)."""
        pl = 3 if double_float else (4 if paired else (2 if warp else (-1 if pipelined is None
                                                                        else int(bool(pipelined)))))
        check(self._lib.iffd_set_geometry(self._h, axis, int(pencils_transform), int(pencils_stiffness), pl),
              "iffd_set_geometry")
        return self

    def tiles(self, axis: int) -> dict:
        """Launch geometry of one direction (iffd_get_tiles)."""
        pt, ps, ns, pl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        rad = (ctypes.c_int * 12)()
        check(self._lib.iffd_get_tiles(self._h, axis, ctypes.byref(pt), ctypes.byref(ps), rad, ctypes.byref(ns),
                                       ctypes.byref(pl)), "iffd_get_tiles")
        return {"pencils_transform": pt.value, "pencils_stiffness": ps.value, "radices": list(rad[:ns.value]),

                "pipelined": pl.value == 1, "warp": pl.value in (2, 3, 4), "double_float": pl.value in (3, 5),
                "paired": pl.value == 4}

    def profile_enable(self, on: bool = True):
        check(self._lib.iffd_profile_enable(self._h, int(on)), "iffd_profile_enable")

    def profile_reset(self):
        check(self._lib.iffd_profile_reset(self._h), "iffd_profile_reset")

    def profile_read(self) -> dict:
        """{kind name: (launches, total ms)} since the last reset."""
        out = {}
        for k in range(self.KERNEL_KINDS):
            n, ms, name = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_char_p()
            check(self._lib.iffd_profile_read(self._h, k, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(name)),
                  "iffd_profile_read")
            out[name.value.decode()] = (n.value, ms.value)
        return out

    def launch_count(self) -> int:
        n = ctypes.c_longlong()
        check(self._lib.iffd_launch_count(self._h, ctypes.byref(n)), "iffd_launch_count")
        return n.value

    apply_preconditioner = iffd_apply_preconditioner
    apply_stiffness = iffd_apply_stiffness
    pcg_solve = iffd_pcg_solve

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.iffd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_solve(plans, fs, us=None, stream=None, raise_on_error: bool = True):
    """iffd_batch_solve: plans[i] with the right-hand sides fs[i] (a float64
    CUDA tensor of nrhs_i * N_i entries, right-hand side after right-hand side;
    nrhs_i = numel / N_i). Returns (us, infos): us[i] like fs[i], infos a list
    (in (i, j) order) of dicts as IFFDPlan.pcg_solve returns them."""
    import torch
    lib = _lib.load()
    count = len(plans)
    if len(fs) != count:
        raise ValueError("one right-hand-side tensor per plan")
    nrhs = []
    for pl, f in zip(plans, fs):
        if not (isinstance(f, torch.Tensor) and f.is_cuda and f.dtype == torch.float64 and f.is_contiguous()
                and f.numel() % pl.N == 0):
            raise ValueError("fs[i] must be a contiguous float64 CUDA tensor of nrhs * N entries")
        nrhs.append(f.numel() // pl.N)
    if us is None:
        us = [torch.empty_like(f) for f in fs]
    for f, u in zip(fs, us):
        if not (u.is_cuda and u.dtype == torch.float64 and u.is_contiguous() and u.numel() == f.numel()):
            raise ValueError("us[i] must match fs[i]")
    harr = (ctypes.c_void_p * max(1, count))(*[pl._h.value for pl in plans])
    narr = (ctypes.c_int * max(1, count))(*nrhs)
    nb = ctypes.c_size_t()
    check(lib.iffd_batch_workspace_bytes(count, harr, narr, ctypes.byref(nb)), "iffd_batch_workspace_bytes")
    ws = torch.empty(nb.value + 256, dtype=torch.uint8, device="cuda")
    wsp = (_ptr(ws) + 255) // 256 * 256
    farr = (ctypes.c_void_p * max(1, count))(*[_ptr(f) for f in fs])
    uarr = (ctypes.c_void_p * max(1, count))(*[_ptr(u) for u in us])
    nsys = sum(nrhs)
    infos = (iffd_pcg_info * max(1, nsys))()
    rc = lib.iffd_batch_solve(count, harr, farr, uarr, narr, wsp, _stream_handle(stream), infos)
    if raise_on_error:
        check(rc, "iffd_batch_solve")
    out = [{"iters": infos[k].iters, "rel_res": infos[k].rel_res, "true_rel_res": infos[k].true_rel_res,
            "status": infos[k].status} for k in range(nsys)]
    return us, out


class IFFDEngine:
    """Batched / continuously batched IFFD-PCG solves (iffd_engine_* of the C ABI).

    Requests (d, n, p, f, u) with caller-owned float64 CUDA tensors are admitted
    while their workspace fits the device arena of `budget_bytes`; step() runs
    one engine step (initialise new requests, `iterations` PCG iterations of
    every active request, retire finished ones); poll() returns completions.
    `persistent`: each step's iterations run as one persistent launch over a
    device work queue (iffd_engine_set_persistent); `wait_limit` bounds its
    device waits (polls), `inject_stall` is the test hook of that call.
    """

    def __init__(self, budget_bytes: int, precision: str = "fp32", rtol: float = 1e-8, maxit: int = 500,
                 flexible: bool = False, stream=None, autotune: bool = False, persistent: bool = False,
                 wait_limit: int = 0, inject_stall: bool = False):
        self._lib = _lib.load()
        opt = iffd_options()
        self._lib.iffd_default_options(ctypes.byref(opt))
        opt.precision = PRECISION[precision]
        opt.rtol = rtol
        opt.maxit = maxit
        opt.flexible = int(flexible)
        opt.autotune = int(autotune)
        self.options = opt
        self._stream = stream
        h = ctypes.c_void_p()
        check(self._lib.iffd_engine_create(ctypes.byref(opt), int(budget_bytes), _stream_handle(stream),
                                           ctypes.byref(h)), "iffd_engine_create")
        self._h = h
        self._keep = {}  # request id -> (f, u) tensors kept alive until completion
        if persistent or inject_stall:
            check(self._lib.iffd_engine_set_persistent(h, int(persistent), int(wait_limit), int(inject_stall)),
                  "iffd_engine_set_persistent")

    @staticmethod
    def _flags(d, dirichlet):
        if dirichlet is None:
            return None
        flags = [int(v) for pair in dirichlet for v in pair]
        if len(flags) != 2 * d:
            raise ValueError("dirichlet needs one (x=0, x=1) pair per direction")
        return (ctypes.c_int * (2 * d))(*flags)

    def request_bytes(self, d: int, n: int, p: int, dirichlet=None) -> int:
        nb = ctypes.c_size_t()
        check(self._lib.iffd_engine_request_bytes(self._h, d, n, p, self._flags(d, dirichlet), ctypes.byref(nb)),
              "iffd_engine_request_bytes")
        return nb.value

    def submit(self, d: int, n: int, p: int, f, u, dirichlet=None):
        """Returns the request id, or None if the arena has no room right now.
        dirichlet: one (x=0, x=1) flag pair per direction (default: all Dirichlet)."""
        rid = ctypes.c_longlong()
        rc = self._lib.iffd_engine_submit(self._h, d, n, p, self._flags(d, dirichlet), _ptr(f), _ptr(u),
                                          ctypes.byref(rid))
        if rc == 4:  # IFFD_ERR_WORKSPACE: admission refused for now
            return None
        check(rc, "iffd_engine_submit")
        self._keep[rid.value] = (f, u)
        return rid.value

    def step(self, iterations: int = 1) -> int:
        active = ctypes.c_int()
        check(self._lib.iffd_engine_step(self._h, int(iterations), ctypes.byref(active)), "iffd_engine_step")
        return active.value

    def poll(self, capacity: int = 4096):
        buf = (_lib.iffd_completion * capacity)()
        cnt = ctypes.c_int()
        check(self._lib.iffd_engine_poll(self._h, buf, capacity, ctypes.byref(cnt)), "iffd_engine_poll")
        out = []
        for k in range(cnt.value):
            c = buf[k]
            self._keep.pop(c.id, None)
            out.append((c.id, {"iters": c.info.iters, "rel_res": c.info.rel_res, "status": c.info.status}))
        return out

    def stats(self) -> dict:
        a, fb, kl = ctypes.c_int(), ctypes.c_size_t(), ctypes.c_longlong()
        check(self._lib.iffd_engine_stats(self._h, ctypes.byref(a), ctypes.byref(fb), ctypes.byref(kl)),
              "iffd_engine_stats")
        return {"active": a.value, "bytes_free": fb.value, "kernel_launches": kl.value}

    def run_to_completion(self, iterations_per_step: int = 4) -> list:
        done = []
        while True:
            active = self.step(iterations_per_step)
            done += self.poll()
            if active == 0:
                return done

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.iffd_engine_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
