"""Pins of the oracle's tensor operators, preconditioners and PCG (Sections 3,
4, 7) against direct Galerkin assembly, dense solves, Proposition 1 and the
iteration counts printed in Table "tab:square"."""

import json
import os

import numpy as np
import pytest

from oracle import operators, splines, splitting

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def direct_galerkin(n, p, d, coef=None):
    """Assemble int a grad B_I . grad B_J over [0,1]^d directly by tensor Gauss
    quadrature of the tensor-product basis (no Kronecker algebra), with the
    Dirichlet basis of Section 2 and x_1 fastest (eq. "tp-B-basis")."""
    knots = splines.open_knots(n, p)
    keep = splines.kept_indices(n, p, (0, 1))
    m = keep.size
    nq = p + 1
    N = m ** d
    A = np.zeros((N, N))
    pos = {g: i for i, g in enumerate(keep)}
    for elem in np.ndindex(*([n] * d)):           # elem[k] = element index in direction k+1
        pts, wts, vals, ders = [], [], [], []
        for k in range(d):
            e = elem[k]
            xg, wg = splines.gauss_rule(nq, e / n, (e + 1) / n)
            pts.append(xg)
            wts.append(wg)
            vals.append(splines.bspline_derivs(knots, p, e, xg, 0))
            ders.append(splines.bspline_derivs(knots, p, e, xg, 1))
        for q in np.ndindex(*([nq] * d)):
            w = np.prod([wts[k][q[k]] for k in range(d)])
            if coef is not None:
                w *= coef([pts[k][q[k]] for k in range(d)])
            for loc in np.ndindex(*([p + 1] * d)):
                gidx = [elem[k] + loc[k] for k in range(d)]
                if any(g not in pos for g in gidx):
                    continue
                grad = []
                for k in range(d):
                    g = 1.0
                    for j in range(d):
                        g *= ders[j][q[j], loc[j]] if j == k else vals[j][q[j], loc[j]]
                    grad.append(g)
                I = sum(pos[gidx[k]] * m ** k for k in range(d))
                for loc2 in np.ndindex(*([p + 1] * d)):
                    gidx2 = [elem[k] + loc2[k] for k in range(d)]
                    if any(g not in pos for g in gidx2):
                        continue
                    grad2 = []
                    for k in range(d):
                        g = 1.0
                        for j in range(d):
                            g *= ders[j][q[j], loc2[j]] if j == k else vals[j][q[j], loc2[j]]
                        grad2.append(g)
                    J = sum(pos[gidx2[k]] * m ** k for k in range(d))
                    A[I, J] += w * sum(a * b for a, b in zip(grad, grad2))
    return A


@pytest.mark.parametrize("n,p,d", [(4, 2, 2), (5, 3, 2), (3, 2, 3)])
def test_stiffness_equals_direct_galerkin(n, p, d):
    """eq. "system_matrix": the Kronecker form equals direct Galerkin assembly of
    int grad u . grad v, which also pins the index ordering (x_1 fastest)."""
    A = direct_galerkin(n, p, d)
    MK = [splines.mass_stiffness(n, p, (0, 1))] * d
    np.testing.assert_allclose(operators.dense_stiffness(MK), A, atol=1e-12 * np.abs(A).max())
    m = MK[0][0].shape[0]
    u = np.random.default_rng(0).standard_normal((m,) * d)
    np.testing.assert_allclose(operators.stiffness_apply(u, MK).ravel(), A @ u.ravel(), atol=1e-11 * np.abs(A).max())


@pytest.mark.parametrize("n,p,d", [(4, 2, 2), (3, 3, 2), (3, 2, 3)])
def test_varcoef_equals_direct_galerkin(n, p, d):
    """The separable coefficient a = 1 + 0.5 prod_k sin(2 pi x_k) integrated with
    the tensor (p+1)-point Gauss rule equals the rank-2 Kronecker form."""
    s = lambda x: np.sin(2 * np.pi * x)
    coef = lambda xs: 1.0 + 0.5 * np.prod([s(x) for x in xs])
    A = direct_galerkin(n, p, d, coef)
    MK = [splines.mass_stiffness(n, p, (0, 1))] * d
    MKs = [splines.mass_stiffness(n, p, (0, 1), weight=s)] * d
    m = MK[0][0].shape[0]
    u = np.random.default_rng(1).standard_normal((m,) * d)
    np.testing.assert_allclose(operators.varcoef_stiffness_apply(u, MK, MKs).ravel(), A @ u.ravel(),
                               atol=1e-11 * np.abs(A).max())


@pytest.mark.parametrize("n,p,d", [(8, 2, 2), (9, 3, 2), (7, 4, 2), (5, 3, 3), (4, 4, 3)])
def test_p10_exact_fd_equals_dense_solve(n, p, d):
    """P10: exact Fast Diagonalization (eq. "exact_diagonalization") = A^{-1}."""
    MK = [splines.mass_stiffness(n, p, (0, 1))] * d
    A = operators.dense_stiffness(MK)
    m = MK[0][0].shape[0]
    r = np.random.default_rng(2).standard_normal((m,) * d)
    eigs = [operators.exact_fd_eig(M, K) for M, K in MK]
    z = operators.exact_fd_apply(r, eigs)
    np.testing.assert_allclose(z.ravel(), np.linalg.solve(A, r.ravel()), rtol=0,
                               atol=1e-10 * np.abs(z).max())


@pytest.mark.parametrize("n,p,d", [(12, 3, 2), (10, 4, 2), (9, 5, 2), (16, 8, 2), (6, 4, 3), (7, 3, 3)])
def test_p8_iffd_equals_fd_of_basis_free_pencil(n, p, d):
    """P8: the structured IFFD apply (Q~ built from V_reg, U_reg, D~, V_out, Q_out)
    equals the exact FD of the pencil (K~, M), K~ formed from the subspace S^reg
    alone (eq. "preconditioner2" and the proof of the Corollary)."""
    splits = [splitting.axis_split(n, p, (0, 1))] * d
    m = splits[0].m
    r = np.random.default_rng(3).standard_normal((m,) * d)
    z = operators.iffd_apply(r, splits)
    eigs = []
    for s in splits:
        Kt = splitting.ktilde_basis_free(s.M, s.K, s.V_reg)
        eigs.append(operators.exact_fd_eig(s.M, 0.5 * (Kt + Kt.T)))
    z2 = operators.exact_fd_apply(r, eigs)
    np.testing.assert_allclose(z, z2, atol=1e-11 * np.abs(z).max())


def test_p14_preconditioner_symmetric_positive():
    """P14: P^{-1} is symmetric positive definite."""
    splits = [splitting.axis_split(11, 5, (0, 1))] * 3
    m = splits[0].m
    rng = np.random.default_rng(4)
    x, y = rng.standard_normal((2, m, m, m))
    Px, Py = operators.iffd_apply(x, splits), operators.iffd_apply(y, splits)
    a, b = np.vdot(x, Py), np.vdot(Px, y)
    assert abs(a - b) <= 1e-14 * np.sqrt(np.vdot(x, Px) * np.vdot(y, Py)) * m ** 1.5
    assert np.vdot(x, Px) > 0


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_p12_prop1_condition_bound(p):
    """P12 (Proposition 1): kappa(P^{-1} A^) <= max_k C_k / c_k, the extreme
    generalized eigenvalues of (K_k, K~_k); and the dense kappa agrees with the
    Lanczos estimate."""
    n = 8
    s = splitting.axis_split(n, p, (0, 1))
    splits = [s, s]
    MK = [(s.M, s.K)] * 2
    A = operators.dense_stiffness(MK)
    m = s.m
    Pinv = np.zeros_like(A)
    for j in range(m * m):
        e = np.zeros(m * m)
        e[j] = 1.0
        Pinv[:, j] = operators.iffd_apply(e.reshape(m, m), splits).ravel()
    kap = operators.kappa_dense(A, Pinv)
    Kt = splitting.ktilde_basis_free(s.M, s.K, s.V_reg)
    bound = operators.prop1_bound(s.K, Kt)
    assert kap <= bound * (1 + 1e-9)
    if p == 2:
        assert abs(kap - 1.0) < 1e-9
    kl = operators.kappa_lanczos(splits, (m, m), lambda u: operators.stiffness_apply(u, MK), k=min(40, m * m - 1))
    assert abs(kl - kap) <= 1e-6 * kap


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 7, 8])
def test_kappa_lanczos_bounded_in_h_and_p(p):
    """Theorem 1 / Proposition 1 / Table "tab:square": kappa(P^{-1} A^) of the
    2D tensor system, found by Lanczos, stays below the Proposition 1 bound of
    the 1D pencil (K, K~), does not grow as h = 1/n shrinks (n = 16, 32, 64),
    and stays bounded uniformly in p (it is 1 for p = 2, where IFFD is exact)."""
    kap = []
    for n in (16, 32, 64):
        s = splitting.axis_split(n, p, (0, 1))
        MK = [(s.M, s.K)] * 2
        k = operators.kappa_lanczos([s, s], (s.m, s.m), lambda u: operators.stiffness_apply(u, MK), k=60)
        bound = operators.prop1_bound(s.K, splitting.ktilde_basis_free(s.M, s.K, s.V_reg))
        assert 1.0 - 1e-9 <= k <= bound * (1 + 1e-6)
        kap.append(k)
    assert kap[2] <= kap[0] * (1 + 1e-6) and kap[1] <= kap[0] * (1 + 1e-6)
    assert max(kap) <= 1.3
    if p == 2:
        assert max(kap) <= 1.0 + 1e-9


@pytest.mark.parametrize("p", [3, 4])
def test_kappa_lanczos_3d_bounded_in_h(p):
    """The same in 3D (n = 8, 16): kappa does not grow with 1/h and stays below
    the Proposition 1 bound."""
    kap = []
    for n in (8, 16):
        s = splitting.axis_split(n, p, (0, 1))
        MK = [(s.M, s.K)] * 3
        k = operators.kappa_lanczos([s] * 3, (s.m,) * 3, lambda u: operators.stiffness_apply(u, MK), k=60)
        bound = operators.prop1_bound(s.K, splitting.ktilde_basis_free(s.M, s.K, s.V_reg))
        assert 1.0 <= k <= bound * (1 + 1e-6)
        kap.append(k)
    assert kap[1] <= kap[0] * (1 + 1e-6)


def test_pcg_matches_dense_solve_and_p9_one_iteration():
    """Textbook PCG converges to A^{-1} f within the residual bound; with p = 2
    and D = {0,1} the IFFD is exact so PCG stops after 1 iteration (P9)."""
    for p, expect_one in ((2, True), (3, False)):
        s = splitting.axis_split(10, p, (0, 1))
        MK = [(s.M, s.K)] * 2
        A = operators.dense_stiffness(MK)
        f = np.random.default_rng(5).uniform(-1, 1, (s.m, s.m))
        u, it, hist = operators.pcg(f, lambda v: operators.stiffness_apply(v, MK),
                                    lambda r: operators.iffd_apply(r, [s, s]), rtol=1e-8)
        assert hist[-1] <= 1e-8
        if expect_one:
            assert it == 1
        ustar = np.linalg.solve(A, f.ravel())
        kappaA = np.linalg.cond(A)
        assert np.linalg.norm(u.ravel() - ustar) <= kappaA * 1e-8 * np.linalg.norm(ustar)
        res = np.linalg.norm(f.ravel() - A @ u.ravel()) / np.linalg.norm(f)
        assert res <= 2e-8


def _table_counts(n, plist):
    out = []
    for p in plist:
        s = splitting.axis_split(n, p, (0, 1))
        MK = [(s.M, s.K)] * 2
        f = np.random.default_rng(100 + p).uniform(-1, 1, (s.m, s.m))
        _, it, _ = operators.pcg(f, lambda v: operators.stiffness_apply(v, MK),
                                 lambda r: operators.iffd_apply(r, [s, s]), rtol=1e-8)
        out.append(it)
    return out


def test_p11_table_square_iterations_n128():
    """P11: Table "tab:square" -- 2D Dirichlet, n = 128, p = 2..7: 1/7/6/6/6/6
    PCG iterations (+-1 because the random right-hand side differs)."""
    g = json.load(open(os.path.join(GOLDEN, "table_square_iterations.json")))
    ref = g["iterations"][g["n"].index(128)]
    got = _table_counts(128, g["p"])
    assert got[0] == 1
    for a, b in zip(got, ref):
        assert abs(a - b) <= 1, (got, ref)


@pytest.mark.slow
def test_p11_table_square_iterations_n256():
    g = json.load(open(os.path.join(GOLDEN, "table_square_iterations.json")))
    ref = g["iterations"][g["n"].index(256)]
    got = _table_counts(256, g["p"])
    for a, b in zip(got, ref):
        assert abs(a - b) <= 1, (got, ref)


def test_sparse_and_dense_apply_agree():
    """The sparse route of apply_along (used for large grids) equals the dense one."""
    import scipy.sparse
    M, K = splines.mass_stiffness(9, 3, (0, 1))
    u = np.random.default_rng(7).standard_normal((M.shape[0],) * 3)
    MK = [(M, K)] * 3
    MKs = [(scipy.sparse.csr_matrix(M), scipy.sparse.csr_matrix(K))] * 3
    np.testing.assert_allclose(operators.stiffness_apply(u, MKs), operators.stiffness_apply(u, MK), rtol=1e-13,
                               atol=1e-13 * np.abs(K).max())


def _cube_counts(n, plist, dirichlet):
    """Oracle IFFD-PCG iterations on the unit cube with one Dirichlet set per
    direction (x, y, z), U[-1,1] right-hand side of seed 500 + p."""
    import scipy.sparse
    out = []
    for p in plist:
        sp = [splitting.axis_split(n, p, tuple(k for k, v in zip((0, 1), D) if v)) for D in dirichlet]
        MK = [(scipy.sparse.csr_matrix(s.M), scipy.sparse.csr_matrix(s.K)) for s in sp]
        shape = tuple(s.m for s in reversed(sp))
        f = np.random.default_rng(500 + p).uniform(-1, 1, shape)
        _, it, _ = operators.pcg(f, lambda v: operators.stiffness_apply(v, MK),
                                 lambda r: operators.iffd_apply(r, sp), rtol=1e-8)
        out.append(it)
    return out


def test_p11_table_cube_iterations_n64():
    """Table "tab:cube" -- unit cube, Dirichlet on x = 0 and y = 1, natural
    conditions elsewhere (the three directions have the Dirichlet sets {0},
    {1} and the empty set), n = 64, p = 2..5: 7/7/7/6 PCG iterations (+-1,
    the random right-hand side differs)."""
    g = json.load(open(os.path.join(GOLDEN, "table_cube_iterations.json")))
    ref = g["iterations"][g["n"].index(64)]
    got = _cube_counts(64, g["p"], g["dirichlet"])
    for a, b in zip(got, ref):
        assert abs(a - b) <= 1, (got, ref)
