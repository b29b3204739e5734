"""CPU checks of the C ABI: the in-tree library loads, exports every entry point
declared in include/iffd.h, and its host-side 1D setup (no GPU involved)
matches the oracle's independent construction of the same objects."""

import ctypes
import os
import re

import numpy as np
import pytest

from oracle import splitting

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:int|const char\*)\s+(iffd_\w+)\s*\(", txt, re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2512_20269_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2512_20269_gb300 import build
        build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2512_20269_gb300 import _lib
    names = declared_symbols()
    assert "iffd_pcg_solve" in names and "iffd_setup" in names
    bound = {s[0] for s in _lib.SIGNATURES}
    for name in names:
        assert hasattr(lib, name), name
        assert name in bound, f"{name} has no ctypes signature"


def test_error_paths_without_gpu(lib):
    """Argument errors are reported with a status and a message, not a crash."""
    import ctypes
    from paper_2512_20269_gb300 import _lib
    d = (ctypes.c_int * 2)(1, 1)
    rc = lib.iffd_host_axis(4, 4, d, None, None, None, None, None, None, None, None, None)
    assert rc == 2 and b"exceed" in lib.iffd_last_error()
    rc = lib.iffd_host_axis(16, 3, (ctypes.c_int * 2)(0, 1), None, None, None, None, None, None, None, None, None)
    assert rc == 0  # mixed Dirichlet / natural ends are supported
    rc = lib.iffd_host_axis(16, 17, d, None, None, None, None, None, None, None, None, None)
    assert rc == 2 and b"outside" in lib.iffd_last_error()
    assert lib.iffd_default_options(None) == 1
    assert lib.iffd_destroy(None) == 0
    h = ctypes.c_void_p()
    rc = lib.iffd_setup(4, (ctypes.c_int * 3)(8, 8, 8), 3, (ctypes.c_int * 8)(*[1] * 8), None, None, ctypes.byref(h))
    assert rc == 1
    rc = lib.iffd_setup(2, (ctypes.c_int * 2)(8, 8), 3, (ctypes.c_int * 4)(0, 0, 0, 0), None, None, ctypes.byref(h))
    assert rc == 3  # all-Neumann: singular


DIRICHLET_SETS = [(1, 1), (1, 0), (0, 1), (0, 0)]


@pytest.mark.parametrize("D", DIRICHLET_SETS)
@pytest.mark.parametrize("n,p", [(16, 1), (16, 2), (16, 3), (16, 4), (17, 5), (20, 6), (21, 7), (24, 8),
                                 (64, 3), (256, 4)])
def test_host_setup_matches_oracle(lib, n, p, D):
    """Banded M/K, V_reg (knot insertion vs L2 projection), Lambda_reg, D~_reg
    and the remainder operator W diag(1/Lambda_out) W^T (basis independent),
    for every Dirichlet set of Table 1."""
    from paper_2512_20269_gb300 import host_axis
    h = host_axis(n, p, D)
    s = splitting.axis_split(n, p, tuple(k for k, v in zip((0, 1), D) if v))
    m, bw = s.m, 2 * p + 1
    assert (h["m"], h["n_reg"], h["n_out"]) == (s.m, s.n_reg, s.n_out)
    M = np.zeros((m, m))
    K = np.zeros((m, m))
    for i in range(m):
        for dd in range(bw):
            j = i + dd - p
            if 0 <= j < m:
                M[i, j] = h["M_band"][i, dd]
                K[i, j] = h["K_band"][i, dd]
    np.testing.assert_allclose(M, s.M, atol=1e-14 * np.abs(s.M).max())
    np.testing.assert_allclose(K, s.K, atol=1e-13 * np.abs(s.K).max())
    np.testing.assert_allclose(h["V_reg"], s.V_reg, atol=1e-12)
    nr = h["n_reg"]
    # Lambda_reg: relative, except the zero eigenvalue of the constant mode (D empty)
    lam_scale = np.abs(s.lam_reg).max()
    np.testing.assert_allclose(h["lam"][:nr], s.lam_reg, rtol=1e-12, atol=1e-13 * lam_scale)
    np.testing.assert_allclose(h["dtilde"], s.Dt, rtol=1e-12)
    if s.n_out:
        lo, W = h["lam"][nr:], h["W"]
        A1 = W @ np.diag(1 / lo) @ W.T
        Wo = s.V_out @ s.Q_out
        A2 = Wo @ np.diag(1 / s.lam_out) @ Wo.T
        np.testing.assert_allclose(A1, A2, atol=1e-12 * np.abs(A2).max())
        np.testing.assert_allclose(lo, s.lam_out, rtol=1e-12)


def _largest_prime_factor(x):
    f, best = 2, 1
    while f * f <= x:
        while x % f == 0:
            best, x = f, x // f
        f += 1
    return max(best, x) if x > 1 else best


@pytest.mark.parametrize("n,p", [(256, 4), (64, 3), (384, 8), (149, 5), (134, 6), (61, 4), (37, 4),
                                 (557, 3), (1939, 3), (2048, 3), (7, 1), (9, 8)])
def test_transform_planner(lib, n, p):
    """The DST's complex DFT has length n_reg (DST-II/III, even p) or
    2 (n_reg + 1) (DST-I, odd p); lengths with a large prime factor run as
    Bluestein over a 5-smooth F >= 2L - 1, smooth lengths run directly."""
    from paper_2512_20269_gb300 import host_transform
    n_reg = n if p % 2 == 0 else n - 1
    L_expected = n_reg if p % 2 == 0 else 2 * (n_reg + 1)
    for prec in ("fp64", "fp32"):
        t = host_transform(n, p, prec)
        assert t["L"] == L_expected
        assert t["pencils"] >= 2 and t["pencils"] % 2 == 0
        if t["bluestein"]:
            F = t["F"]
            assert F >= 2 * t["L"] - 1 and _largest_prime_factor(F) <= 5
            assert _largest_prime_factor(t["L"]) > 13
        else:
            assert t["F"] == t["L"]
        if _largest_prime_factor(t["L"]) <= 5:
            assert not t["bluestein"]
    # a large prime factor with room in shared memory always takes Bluestein
    if _largest_prime_factor(L_expected) >= 37 and L_expected <= 1200:
        assert host_transform(n, p, "fp64")["bluestein"] and host_transform(n, p, "fp32")["bluestein"]
    # two FP64 length-F buffers no longer fit for L = 3878: FP64 keeps the
    # direct FFT while FP32 runs Bluestein
    if (n, p) == (1939, 3):
        assert not host_transform(n, p, "fp64")["bluestein"] and host_transform(n, p, "fp32")["bluestein"]


# repeated interior knots (Remark "reduced_regularity"): interior knots, knots
# next to an end (their block joins the edge block), several knots, the
# largest multiplicity, and tiny n where V_reg is kept as one dense block
REP_HOST_CASES = [
    (16, 3, (1, 1), {8: 2}), (16, 4, (1, 1), {5: 1, 11: 3}), (17, 2, (1, 0), {9: 1}),
    (20, 5, (0, 0), {10: 4}), (18, 6, (0, 1), {6: 2, 12: 5}), (40, 4, (1, 1), {20: 1}),
    (64, 3, (1, 1), {10: 1, 11: 2, 40: 1}), (30, 8, (1, 0), {15: 7}), (16, 4, (1, 1), {1: 1}),
    (16, 4, (1, 1), {2: 3}), (16, 3, (0, 0), {15: 2}), (8, 7, (1, 1), {4: 6}),
    (10, 3, (1, 1), {k: 1 for k in range(1, 10)}), (5, 4, (1, 1), {}), (3, 2, (1, 0), {}), (9, 8, (0, 1), {}),
]


@pytest.mark.parametrize("n,p,D,rep", REP_HOST_CASES)
def test_host_setup_reduced_regularity_matches_oracle(lib, n, p, D, rep):
    """With repeated knots: banded M/K on the knot vector with repeats, V_reg
    (knot insertion, as the device passes apply it, vs the oracle's L2
    projection), the unchanged Lambda_reg and D~_reg, and the remainder
    operator including the jump constraints at the repeated knots."""
    from paper_2512_20269_gb300 import host_axis
    h = host_axis(n, p, D, rep)
    s = splitting.axis_split(n, p, tuple(k for k, v in zip((0, 1), D) if v), rep=rep)
    m, bw = s.m, 2 * p + 1
    assert (h["m"], h["n_reg"], h["n_out"]) == (s.m, s.n_reg, s.n_out)
    M = np.zeros((m, m))
    K = np.zeros((m, m))
    for i in range(m):
        for dd in range(bw):
            j = i + dd - p
            if 0 <= j < m:
                M[i, j] = h["M_band"][i, dd]
                K[i, j] = h["K_band"][i, dd]
    np.testing.assert_allclose(M, s.M, atol=1e-14 * np.abs(s.M).max())
    np.testing.assert_allclose(K, s.K, atol=1e-13 * np.abs(s.K).max())
    np.testing.assert_allclose(h["V_reg"], s.V_reg, atol=1e-12)
    nr = h["n_reg"]
    lam_scale = np.abs(s.lam_reg).max()
    np.testing.assert_allclose(h["lam"][:nr], s.lam_reg, rtol=1e-12, atol=1e-13 * lam_scale)
    np.testing.assert_allclose(h["dtilde"], s.Dt, rtol=1e-12)
    if s.n_out:
        lo, W = h["lam"][nr:], h["W"]
        A1 = W @ np.diag(1 / lo) @ W.T
        Wo = s.V_out @ s.Q_out
        A2 = Wo @ np.diag(1 / s.lam_out) @ Wo.T
        np.testing.assert_allclose(A1, A2, atol=1e-11 * np.abs(A2).max())
        np.testing.assert_allclose(lo, s.lam_out, rtol=1e-11)


@pytest.mark.parametrize("rep,msg", [({0: 1}, b"outside"), ({16: 1}, b"outside"), ({5: 4}, b"outside 1..p-1"),
                                     ({5: 0}, b"outside 1..p-1")])
def test_reduced_regularity_input_errors(lib, rep, msg):
    from paper_2512_20269_gb300 import IFFDError, host_axis
    with pytest.raises(IFFDError):
        host_axis(16, 4, (1, 1), rep)
    assert msg in lib.iffd_last_error()
    d = (ctypes.c_int * 2)(1, 1)
    reps = (ctypes.c_int * 4)(5, 1, 5, 2)  # the same knot twice
    assert lib.iffd_host_axis_knots(16, 4, d, 2, reps, None, None, None, None, None, None, None, None, None) == 2
    assert lib.iffd_host_axis_knots(16, 4, d, 1, None, None, None, None, None, None, None, None, None, None) == 1
    assert lib.iffd_host_axis_knots(16, 4, d, -1, reps, None, None, None, None, None, None, None, None, None) == 1


@pytest.mark.parametrize("n,p,dirichlet,rep", [(7, 3, (1, 1), None), (6, 4, (1, 0), {3: 2}), (5, 2, (0, 0), None),
                                                (9, 5, (0, 1), {2: 1, 6: 4})])
def test_library_gauss_tables_match_the_oracle(n, p, dirichlet, rep):
    """The library's host tables of the general-coefficient operator (points,
    weights, and the sparse value / derivative matrices, expanded) equal the
    oracle's quad_axis: independent evaluations of the same B-splines."""
    from oracle import general
    from paper_2512_20269_gb300 import host_quad_axis
    t = host_quad_axis(n, p, dirichlet, rep=rep)
    dset = tuple(k for k, v in zip((0, 1), dirichlet) if v)
    x, w, B, D = general.quad_axis(n, p, dset, rep=rep)
    assert np.max(np.abs(t["x"] - x)) <= 1e-15 and np.max(np.abs(t["w"] - w)) <= 1e-15
    assert t["B"].shape == B.shape
    assert np.max(np.abs(t["B"] - B)) <= 1e-13
    assert np.max(np.abs(t["D"] - D)) <= 1e-11 * max(1.0, np.max(np.abs(D)))


def test_host_quad_axis_input_errors():
    from paper_2512_20269_gb300 import IFFDError, host_quad_axis
    with pytest.raises(IFFDError):
        host_quad_axis(8, 3, (1, 1), rep={0: 1})  # knot 0 is not interior
    with pytest.raises(IFFDError):
        host_quad_axis(8, 3, (1, 1), rep={4: 3})  # multiplicity above p - 1
    t = host_quad_axis(8, 3, (1, 1), rep={4: 2})
    assert t["B"].shape == (32, 8 + 3 + 2 - 2)
