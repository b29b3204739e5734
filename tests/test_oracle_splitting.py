"""Pins of the oracle's splitting / eigendata layer (Sections 4-6, Table 1,
Lemma 3, Theorem 3) against what the paper and the mathematics fix."""

import itertools

import numpy as np
import pytest
import scipy.fft
import scipy.linalg

from oracle import splines, splitting

ALL_D = [(0, 1), (0,), (1,), ()]


def null_dim(G: np.ndarray, m: int) -> int:
    if G.shape[0] == 0:
        return m
    s = np.linalg.svd(G / np.abs(G).max(axis=1, keepdims=True), compute_uv=False)
    return m - int((s > 1e-9 * s[0]).sum())


@pytest.mark.parametrize("p", range(1, 9))
@pytest.mark.parametrize("D", ALL_D)
def test_p3_reg_dimension_all_cases(p, D):
    """P3: the null space of the derivative conditions of eq. "reg_space" has the
    dimension n_reg printed in eq. "reg_space_dim", for all 8 (parity, D) cases,
    and the special basis of Section 6 has exactly that many functions."""
    n = 3 * p + 5
    m = n + p - len(D)
    G = splitting.constraint_matrix(n, p, D)
    assert null_dim(G, m) == splitting.n_reg_formula(n, p, D)
    assert m - splitting.n_reg_formula(n, p, D) == splitting.n_out_formula(n, p, D)
    assert len(splitting.special_basis_combinations(n, p, D)) == splitting.n_reg_formula(n, p, D)


@pytest.mark.parametrize("p", range(1, 9))
@pytest.mark.parametrize("D", ALL_D)
def test_special_basis_spans_reg_space(p, D):
    """The special basis (eq. "special_basis") lies in S_{p,h,D} (zero coefficient
    on removed Dirichlet B-splines), satisfies every condition of eq. "reg_space",
    and is linearly independent -- so its span is exactly S^reg."""
    n = 2 * p + 7
    V, dropped = splitting.V_reg_matrix(n, p, D, return_dropped=True)
    if dropped.size:
        assert np.abs(dropped).max() < 1e-12
    G = splitting.constraint_matrix(n, p, D)
    if G.shape[0]:
        rel = np.abs(G @ V) / (np.abs(G).sum(axis=1, keepdims=True) * np.abs(V).max())
        assert rel.max() < 1e-11
    s = np.linalg.svd(V, compute_uv=False)
    assert s[-1] > 1e-8 * s[0]
    assert V.shape[1] == splitting.n_reg_formula(n, p, D)


@pytest.mark.parametrize("p", range(1, 9))
@pytest.mark.parametrize("D", ALL_D)
def test_p4_theorem3_collocation_eigenvectors(p, D):
    """P4 (Theorem 3): C_reg U_reg = U_reg Theta, Theta_jj the cardinal symbol."""
    n = 2 * p + 6
    C = splitting.collocation_matrix(n, p, D)
    U = splitting.U_reg(n, p, D)
    th = splitting.theta_closed_form(n, p, D)
    np.testing.assert_allclose(C @ U, U * th[None, :], atol=1e-13)


@pytest.mark.parametrize("p", range(1, 9))
@pytest.mark.parametrize("D", ALL_D)
def test_p5_p6_diagonalisation_and_closed_forms(p, D):
    """P5: U_reg diagonalises V_reg^T M V_reg and V_reg^T K V_reg (Theorem 2 and
    the special-basis statement of Section 6).
    P6: the numeric D~_reg and Lambda_reg equal the closed forms (Lemma 3 read
    with 1/h^2; D~ derived from the periodic symbols)."""
    n = 3 * p + 7
    s = splitting.axis_split(n, p, D)
    V, U = s.V_reg, s.U
    for A in (s.M, s.K):
        B = U.T @ V.T @ A @ V @ U
        off = B - np.diag(np.diag(B))
        assert np.abs(off).max() <= 1e-12 * np.abs(np.diag(B)).max()
    lam_numeric = np.diag(U.T @ V.T @ s.K @ V @ U) / s.Dt ** 2   # eq. "Lambda reg"
    np.testing.assert_allclose(s.lam_reg, lam_numeric, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(s.Dt, splitting.dtilde_closed_form(n, p, D), rtol=1e-11)


@pytest.mark.parametrize("n,p", [(12, 1), (12, 2), (13, 3), (16, 4), (17, 5), (20, 6), (21, 7), (24, 8)])
@pytest.mark.parametrize("D", ALL_D)
def test_p7_identities(n, p, D):
    """P7: Q~^T M Q~ = I (eq. "orthogonality"), Q~^T K~ Q~ = Lambda~ with the
    basis-free K~, Q~ Q~^T = M^{-1}, V_reg^T M V_out = 0, P_r + P_o = I."""
    s = splitting.axis_split(n, p, D)
    m = s.m
    assert s.n_reg + s.n_out == m
    np.testing.assert_allclose(s.Qt.T @ s.M @ s.Qt, np.eye(m), atol=1e-11)
    Kt = splitting.ktilde_basis_free(s.M, s.K, s.V_reg)
    scale = np.abs(s.lamt).max()
    np.testing.assert_allclose(s.Qt.T @ Kt @ s.Qt, np.diag(s.lamt), atol=1e-10 * scale)
    Minv = np.linalg.inv(s.M)
    np.testing.assert_allclose(s.Qt @ s.Qt.T, Minv, atol=1e-10 * np.abs(Minv).max())
    if s.n_out:
        assert np.abs(s.V_reg.T @ s.M @ s.V_out).max() < 1e-12 * np.abs(s.V_reg).max() * np.abs(s.V_out).max() * m
    Pr = s.V_reg @ np.linalg.solve(s.V_reg.T @ s.M @ s.V_reg, s.V_reg.T @ s.M)
    np.testing.assert_allclose(Pr @ Pr, Pr, atol=1e-11)


def test_p9_no_remainder_cases():
    """P9 (end of Section 4): S^reg = S for p = 1 (any D... here {0,1}) and for
    p = 2 with D = {0,1}; then Q~, Lambda~ is the exact eigendecomposition."""
    for p in (1, 2):
        s = splitting.axis_split(19, p, (0, 1))
        assert s.n_out == 0
        lam, Q = scipy.linalg.eigh(s.K, s.M)
        np.testing.assert_allclose(np.sort(s.lamt), lam, rtol=1e-11)
        Kt = splitting.ktilde_basis_free(s.M, s.K, s.V_reg)
        np.testing.assert_allclose(Kt, s.K, atol=1e-10 * np.abs(s.K).max())


@pytest.mark.parametrize("p,D", list(itertools.product([1, 2, 3, 4], ALL_D)))
def test_p13_table1_transform_types(p, D):
    """P13: U_reg of Table 1 is the named trigonometric transform (library DST/DCT
    of scipy, unnormalised convention y = 2 * sum ...)."""
    n = 16
    U = splitting.U_reg(n, p, D)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(U.shape[0])
    Ux = U @ x
    D = frozenset(D)
    if p % 2 == 1:
        if D == {0, 1}:
            ref = scipy.fft.dst(x, type=1) / 2
        elif D == {0}:
            ref = scipy.fft.dst(x, type=2) / 2
        elif D == {1}:
            ref = scipy.fft.dct(x, type=2) / 2
        else:
            k = np.arange(x.size)
            ref = (scipy.fft.dct(x, type=1) + x[0] + (-1.0) ** k * x[-1]) / 2
    else:
        if D == {0, 1}:
            # U is DST-III, U^T is DST-II (Table 1)
            ref = None
            np.testing.assert_allclose(U.T @ x, scipy.fft.dst(x, type=2) / 2, atol=1e-12)
            k = np.arange(x.size)
            ref = (scipy.fft.dst(x, type=3) + (-1.0) ** k * x[-1]) / 2
        elif D == {0}:
            ref = scipy.fft.dst(x, type=4) / 2
        elif D == {1}:
            ref = scipy.fft.dct(x, type=4) / 2
        else:
            ref = (scipy.fft.dct(x, type=3) + x[0]) / 2
    np.testing.assert_allclose(Ux, ref, atol=1e-12)


def test_prop1_bound_bounded_in_h_and_p():
    """Theorem 1 / Corollary: the 1D spectral-equivalence ratio max eig(K, K~) /
    min eig(K, K~) is bounded independently of h and p (it must not grow as h
    shrinks)."""
    from oracle import operators
    for p in range(2, 9):
        ratios = []
        for n in (16, 32, 64):
            s = splitting.axis_split(n, p, (0, 1))
            Kt = splitting.ktilde_basis_free(s.M, s.K, s.V_reg)
            ratios.append(operators.prop1_bound(s.K, Kt))
        assert max(ratios) < 4.0, (p, ratios)
        assert ratios[-1] <= ratios[0] * 1.05 + 1e-12, (p, ratios)


# ------------------------------------------- reduced regularity (Remark)
REP_CASES = [(16, 3, (0, 1), {8: 2}), (16, 4, (0, 1), {5: 1, 11: 3}), (17, 2, (0,), {9: 1}),
             (20, 5, (), {10: 4}), (18, 6, (1,), {6: 2, 12: 5}), (15, 1, (0, 1), {})]


@pytest.mark.parametrize("n,p,D,rep", REP_CASES)
def test_reduced_regularity_dimensions(n, p, D, rep):
    """Remark "reduced_regularity": S^reg does not change when interior knots
    are repeated, and every added knot adds one function to S^out."""
    base = splitting.axis_split(n, p, D)
    s = splitting.axis_split(n, p, D, rep=rep)
    extra = sum(rep.values())
    assert s.m == base.m + extra
    assert s.n_reg == base.n_reg
    assert s.n_out == base.n_out + extra


@pytest.mark.parametrize("n,p,D,rep", REP_CASES[:5])
def test_reduced_regularity_regular_space_unchanged(n, p, D, rep):
    """The special functions written in the basis with repeated knots (V_reg,
    by L2 projection) are the same functions: evaluated through the B-splines
    they equal the cardinal combinations at points of every element."""
    s = splitting.axis_split(n, p, D, rep=rep)
    knots = splines.open_knots(n, p, rep)
    keep = splines.kept_indices(n, p, D, rep)
    size = splines.n_basis(n, p, rep)
    combos = splitting.special_basis_combinations(n, p, D)
    full = np.zeros((size, s.n_reg))
    full[keep] = s.V_reg
    h = 1.0 / n
    worst = 0.0
    for e in range(n):
        x = e * h + h * np.array([0.13, 0.5, 0.91])
        B = splines.bspline_derivs(knots, p, e, x, 0)
        s0 = int(np.searchsorted(knots, e / n, side="right")) - 1 - p
        vals = B @ full[s0:s0 + p + 1]
        ref = np.zeros_like(vals)
        for j, c in enumerate(combos):
            for v, k in c:
                ref[:, j] += v * splines.cardinal_bspline(p, (x - splitting.node(k, n, p)) / h)
        worst = max(worst, np.abs(vals - ref).max())
    assert worst < 1e-12


@pytest.mark.parametrize("n,p,D,rep", REP_CASES[:5])
def test_reduced_regularity_identities(n, p, D, rep):
    """P1 and P7 with repeated knots: partition of unity, K 1 = 0, Q~^T M Q~ = I,
    Q~^T K~ Q~ = Lambda~, V_reg^T M V_out = 0."""
    Mf, Kf = splines.assemble_full(n, p, rep=rep)
    assert abs(Mf.sum() - 1.0) < 1e-13
    assert np.abs(Kf @ np.ones(Kf.shape[0])).max() < 1e-10 * np.abs(Kf).max()
    s = splitting.axis_split(n, p, D, rep=rep)
    m = s.m
    np.testing.assert_allclose(s.Qt.T @ s.M @ s.Qt, np.eye(m), atol=1e-11)
    Kt = splitting.ktilde_basis_free(s.M, s.K, s.V_reg)
    np.testing.assert_allclose(s.Qt.T @ Kt @ s.Qt, np.diag(s.lamt), atol=1e-10 * np.abs(s.lamt).max())
    assert np.abs(s.V_reg.T @ s.M @ s.V_out).max() < 1e-11 * np.abs(s.V_reg).max() * np.abs(s.V_out).max() * m


def test_reduced_regularity_condition_bounded():
    """IFFD stays a good preconditioner with a C^0 line (the plate-with-hole
    situation of Section 7): kappa(P^{-1} A^) in 2D with a knot of full
    multiplicity at x = 1/2 stays bounded as h shrinks (and close to its value
    without the repeated knot, 1.25)."""
    from oracle import operators
    import scipy.sparse
    ks = []
    for n in (16, 32):
        p = 3
        rep = {n // 2: p - 1}
        sx = splitting.axis_split(n, p, (0, 1), rep=rep)
        sy = splitting.axis_split(n, p, (0, 1))
        MK = [(scipy.sparse.csr_matrix(sx.M), scipy.sparse.csr_matrix(sx.K)),
              (scipy.sparse.csr_matrix(sy.M), scipy.sparse.csr_matrix(sy.K))]
        ks.append(operators.kappa_lanczos([sx, sy], (sy.m, sx.m), lambda v: operators.stiffness_apply(v, MK)))
    assert ks[1] <= ks[0] + 0.05 and ks[1] < 1.5, ks  # measured: 1.30 (n = 16), 1.25 (n = 32)
