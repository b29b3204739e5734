"""ctypes binding of the C ABI declared in include/iffd.h (argument marshalling only).

Every function keeps the C name. The library is loaded from this package's
directory; there is no fallback: if ``libiffd.so`` is missing the import of any
entry point raises.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libiffd.so")

c_int_p = ctypes.POINTER(ctypes.c_int)
c_double_p = ctypes.POINTER(ctypes.c_double)
c_size_t_p = ctypes.POINTER(ctypes.c_size_t)

IFFD_OK = 0
# Largest problem served by iffd_apply_stiffness_noalloc (include/iffd.h).
IFFD_NOALLOC_MAX_DOFS = 1 << 20
STATUS_NAMES = {0: "IFFD_OK", 1: "IFFD_ERR_INVALID_ARG", 2: "IFFD_ERR_UNSUPPORTED", 3: "IFFD_ERR_SINGULAR",
                4: "IFFD_ERR_WORKSPACE", 5: "IFFD_ERR_CUDA", 6: "IFFD_ERR_NOT_CONVERGED",
                7: "IFFD_ERR_BREAKDOWN", 8: "IFFD_ERR_TIMEOUT"}


class iffd_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("precond", ctypes.c_int), ("rtol", ctypes.c_double),
                ("maxit", ctypes.c_int), ("coef", ctypes.c_int), ("true_residual", ctypes.c_int),
                ("flexible", ctypes.c_int), ("coef_amp", ctypes.c_double), ("autotune", ctypes.c_int)]


class iffd_pcg_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_res", ctypes.c_double), ("true_rel_res", ctypes.c_double),
                ("status", ctypes.c_int)]


class iffd_completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("info", iffd_pcg_info)]


# (name, restype, argtypes) of every exported entry point of include/iffd.h
SIGNATURES = [
    ("iffd_default_options", ctypes.c_int, [ctypes.POINTER(iffd_options)]),
    ("iffd_setup", ctypes.c_int, [ctypes.c_int, c_int_p, ctypes.c_int, c_int_p, ctypes.POINTER(iffd_options),
                                  ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("iffd_setup_knots", ctypes.c_int, [ctypes.c_int, c_int_p, ctypes.c_int, c_int_p, c_int_p, c_int_p,
                                        ctypes.POINTER(iffd_options), ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    ("iffd_workspace_bytes", ctypes.c_int, [ctypes.c_void_p, c_size_t_p]),
    ("iffd_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("iffd_set_geometry", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("iffd_get_tiles", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_int_p, c_int_p, c_int_p, c_int_p, c_int_p]),
    ("iffd_get_dims", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_int_p, c_int_p, c_int_p]),
    ("iffd_get_1d", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [c_double_p] * 6),
    ("iffd_host_axis", ctypes.c_int, [ctypes.c_int, ctypes.c_int, c_int_p, c_int_p, c_int_p, c_int_p]
     + [c_double_p] * 6),
    ("iffd_host_axis_knots", ctypes.c_int, [ctypes.c_int, ctypes.c_int, c_int_p, ctypes.c_int, c_int_p, c_int_p,
                                            c_int_p, c_int_p] + [c_double_p] * 6),
    ("iffd_host_transform", ctypes.c_int, [ctypes.c_int, ctypes.c_int, c_int_p, ctypes.c_int, c_int_p, c_int_p,
                                           c_int_p]),
    ("iffd_apply_preconditioner", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p]),
    ("iffd_apply_stiffness", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p]),
    ("iffd_apply_stiffness_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                    ctypes.c_void_p]),
    ("iffd_pcg_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.POINTER(iffd_pcg_info)]),
    ("iffd_host_quad_axis", ctypes.c_int, [ctypes.c_int, ctypes.c_int, c_int_p, ctypes.c_int, c_int_p, c_int_p,
                                           c_int_p] + [c_double_p] * 4),
    ("iffd_quad_points", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_int_p, c_double_p, c_double_p]),
    ("iffd_general_workspace_bytes", ctypes.c_int, [ctypes.c_void_p, c_size_t_p]),
    ("iffd_apply_stiffness_general", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                    ctypes.c_void_p]),
    ("iffd_pcg_solve_general", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.POINTER(iffd_pcg_info)]),
    ("iffd_profile_enable", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("iffd_profile_reset", ctypes.c_int, [ctypes.c_void_p]),
    ("iffd_profile_read", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                         c_double_p, ctypes.POINTER(ctypes.c_char_p)]),
    ("iffd_launch_count", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)]),
    ("iffd_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("iffd_engine_create", ctypes.c_int, [ctypes.POINTER(iffd_options), ctypes.c_size_t, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_void_p)]),
    ("iffd_engine_request_bytes", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 c_int_p, c_size_t_p]),
    ("iffd_engine_submit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, c_int_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)]),
    ("iffd_engine_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_int_p]),
    ("iffd_engine_poll", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(iffd_completion), ctypes.c_int, c_int_p]),
    ("iffd_engine_stats", ctypes.c_int, [ctypes.c_void_p, c_int_p, c_size_t_p, ctypes.POINTER(ctypes.c_longlong)]),
    ("iffd_engine_set_persistent", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_int]),
    ("iffd_engine_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("iffd_batch_workspace_bytes", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), c_int_p,
                                                  c_size_t_p]),
    ("iffd_batch_solve", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), c_int_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(iffd_pcg_info)]),
    ("iffd_apply_pass", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, c_int_p, c_int_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("iffd_slab_workspace_bytes", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_size_t_p]),
    ("iffd_slab_stiffness", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("iffd_copy_box", ctypes.c_int, [ctypes.c_void_p, c_int_p, c_int_p, ctypes.c_void_p, c_int_p, c_int_p, c_int_p,
                                     ctypes.c_void_p]),
    ("iffd_vec_dot_workspace_bytes", ctypes.c_int, [c_size_t_p]),
    ("iffd_vec_dot", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    ("iffd_vec_axpby", ctypes.c_int, [ctypes.c_longlong, ctypes.c_double, ctypes.c_void_p, ctypes.c_double,
                                      ctypes.c_void_p, ctypes.c_void_p]),
    ("iffd_measure_peak", ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, c_int_p, c_double_p]),
    ("iffd_last_error", ctypes.c_char_p, []),
]

_lib = None


def load() -> ctypes.CDLL:
    """Load libiffd.so (built in-tree by build.py) and declare its signatures."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2512_20269_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class IFFDError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = load().iffd_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(code: int, where: str) -> int:
    if code != IFFD_OK:
        raise IFFDError(code, where)
    return code


def __getattr__(name):
    if name.startswith("iffd_"):
        return getattr(load(), name)
    raise AttributeError(name)
