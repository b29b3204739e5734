"""Space splitting and approximate 1D eigendecomposition (Sections 4-6) -- oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Notation follows the paper: n elements, degree p, h = 1/n, Dirichlet set D,
m = dim S_{p,h,D}, n_reg / n_out the dimensions of S^reg / S^out,
V_reg / V_out coordinate bases of the two subspaces, U_reg the trigonometric
matrix of Table 1, D~_reg its normalisation, Q_out / Lambda_out the remainder
eigenpairs, and Q~ = [V_reg U D~^{-1}, V_out Q_out], Lambda~ = blkdiag(Lambda_reg,
Lambda_out).

Readings of the paper taken here:

* Neumann ends carry the odd-derivative conditions of all orders <= p-1
  (eq. "reg_space"; the printed range k = 0..floor(p/2) overshoots p-1).
* The cardinal B-spline with index i is B~_p((x - x_i)/h), maximal at x_i
  (eq. "Btilde"; the printed argument x/h - x_i is read this way).
* For 1 not in D and p even the right block of the special basis runs over
  i = n-p/2+1..n (p/2 functions), which is what n_reg = n requires.
* V_out spans the L2-orthogonal complement of S^reg: V_out = M^{-1} N with N an
  orthonormal basis of the Euclidean complement of range(V_reg). (The printed
  formula for V_out is dimensionally inconsistent; any basis of the same
  subspace gives the same preconditioner.)
* D~_reg is computed numerically as (U^T V_reg^T M V_reg U)^{1/2} (end of
  Section 6). Its closed form is derived from the periodic symbols (see
  ``dtilde_closed_form``). Lambda_reg is taken from Lemma 3, read with 1/h^2.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg

from .splines import (assemble_full, bspline_derivs, cardinal_bspline, gauss_rule,
                      kept_indices, open_knots)


def normalize_dirichlet(dirichlet) -> frozenset:
    return frozenset(int(x) for x in dirichlet)


# ---------------------------------------------------------------- dimensions
def n_reg_formula(n: int, p: int, dirichlet) -> int:
    """n_reg as printed in eq. "reg_space_dim"."""
    D = normalize_dirichlet(dirichlet)
    if p % 2 == 1 and D == {0, 1}:
        return n - 1
    if p % 2 == 1 and not D:
        return n + 1
    return n


def n_out_formula(n: int, p: int, dirichlet) -> int:
    """n_out as printed in eq. "reg_space_dim"."""
    D = normalize_dirichlet(dirichlet)
    if p % 2 == 0 and D == {0, 1}:
        return p - 2
    if p % 2 == 0 and not D:
        return p
    return p - 1


def constraint_orders(p: int, end_in_dirichlet: bool):
    """Derivative orders that vanish on S^reg at one end (eq. "reg_space"):
    even orders 2..p-1 at a Dirichlet end, odd orders 1..p-1 at a free end."""
    if end_in_dirichlet:
        return [2 * k for k in range(1, (p - 1) // 2 + 1)]
    return [2 * k + 1 for k in range(0, p) if 2 * k + 1 <= p - 1]


def constraint_matrix(n: int, p: int, dirichlet) -> np.ndarray:
    """Rows: the derivative functionals of eq. "reg_space" evaluated on the kept
    B-spline basis of S_{p,h,D}. S^reg is exactly the null space of this matrix."""
    D = normalize_dirichlet(dirichlet)
    knots = open_knots(n, p)
    keep = kept_indices(n, p, D)
    rows = []
    for end, e, x in ((0, 0, 0.0), (1, n - 1, 1.0)):
        for order in constraint_orders(p, end in D):
            vals = bspline_derivs(knots, p, e, np.array([x]), order)[0]
            full = np.zeros(n + p)
            full[e:e + p + 1] = vals
            rows.append(full[keep])
    if not rows:
        return np.zeros((0, len(keep)))
    return np.array(rows)


# ------------------------------------------------------ nodes and Table 1
def delta_p(p: int) -> int:
    """eq. "delta": 0 for odd p, 1 for even p."""
    return 0 if p % 2 == 1 else 1


def node(i, n: int, p: int):
    """Periodic nodes of eq. "nodes": x_i = i h (p odd), (i - 1/2) h (p even)."""
    h = 1.0 / n
    return np.asarray(i, dtype=np.float64) * h if p % 2 == 1 \
        else (np.asarray(i, dtype=np.float64) - 0.5) * h


def table1(n: int, p: int, dirichlet):
    """Row-node positions, alpha_j and beta of Table 1 for the 8 cases.

    Returns (nodes[0..n_reg-1], alpha[0..n_reg-1], beta); U_reg[i, j] =
    sin(nodes[i] * alpha[j] + beta)."""
    D = normalize_dirichlet(dirichlet)
    h = 1.0 / n
    nr = n_reg_formula(n, p, D)
    i = np.arange(1, nr + 1, dtype=np.float64)
    j = np.arange(1, nr + 1, dtype=np.float64)
    if p % 2 == 1:
        x = i * h if 0 in D else (i - 1) * h
    else:
        x = (i - 0.5) * h
    if D == {0, 1}:
        alpha, beta = j * np.pi, 0.0
    elif D == {0}:
        alpha, beta = (j - 0.5) * np.pi, 0.0
    elif D == {1}:
        alpha, beta = (j - 0.5) * np.pi, np.pi / 2
    else:
        alpha, beta = (j - 1) * np.pi, np.pi / 2
    return x, alpha, beta


def U_reg(n: int, p: int, dirichlet) -> np.ndarray:
    """U_reg = [sin(x_i alpha_j + beta)]_{i,j=1}^{n_reg} (Table 1)."""
    x, alpha, beta = table1(n, p, dirichlet)
    return np.sin(np.outer(x, alpha) + beta)


# ------------------------------------------------------- special basis
def cardinal_index_range(n: int, p: int):
    """Indices of the cardinal B-splines active on (0,1) (eq. "Btilde")."""
    return range(-((p - 1) // 2), n + p // 2 + 1)


def special_basis_combinations(n: int, p: int, dirichlet):
    """The special basis B = B_L u B_I u B_R of Section 6 as a list of
    combinations [(coef, cardinal index), ...]."""
    D = normalize_dirichlet(dirichlet)
    dp = delta_p(p)
    left, right = [], []
    if 0 in D:
        for i in range(1, p // 2 + 1):
            left.append([(1.0, i), (-1.0, dp - i)])
    elif p % 2 == 0:
        for i in range(1, p // 2 + 1):
            left.append([(1.0, i), (1.0, 1 - i)])
    else:
        left.append([(1.0, 0)])
        for i in range(1, (p - 1) // 2 + 1):
            left.append([(1.0, i), (1.0, -i)])
    if 1 in D:
        for i in range(n - (p - 1) // 2, n - 1 + dp + 1):
            right.append([(1.0, i), (-1.0, 2 * n + dp - i)])
    elif p % 2 == 0:
        for i in range(n - p // 2 + 1, n + 1):
            right.append([(1.0, i), (1.0, 2 * n + 1 - i)])
    else:
        for i in range(n - (p - 1) // 2, n):
            right.append([(1.0, i), (1.0, 2 * n - i)])
        right.append([(1.0, n)])
    inner = [[(1.0, i)] for i in range(p // 2 + 1, n - (p + 1) // 2 + 1)]
    combos = []
    for c in left + inner + right:
        # a cardinal B-spline paired with itself cancels (odd p, index 0)
        merged: dict = {}
        for coef, k in c:
            merged[k] = merged.get(k, 0.0) + coef
        combos.append([(v, k) for k, v in merged.items() if v != 0.0])
    return combos


def cardinal_coefficients(n: int, p: int, rep=None) -> tuple[np.ndarray, list]:
    """Coefficients of every active cardinal B-spline B~_k (restricted to [0,1])
    in the full open-knot basis of S_{p,h} (with the repeated knots ``rep``),
    by exact L2 projection (the cardinal B-splines are C^{p-1} piecewise
    polynomials on the same elements, hence in the space)."""
    knots = open_knots(n, p, rep)
    h = 1.0 / n
    ks = list(cardinal_index_range(n, p))
    Mfull, _ = assemble_full(n, p, rep=rep)
    nq = p + 1
    E = np.zeros((len(ks), Mfull.shape[0]))
    xs, ws = [], []
    for e in range(n):
        xg, wg = gauss_rule(nq, e / n, (e + 1) / n)
        xs.append(xg)
        ws.append(wg)
    xs = np.concatenate(xs)
    ws = np.concatenate(ws)
    T = (xs[None, :] - node(np.array(ks), n, p)[:, None]) / h
    card = cardinal_bspline(p, T)               # (ncard, n*nq)
    for e in range(n):
        sl = slice(e * nq, (e + 1) * nq)
        B = bspline_derivs(knots, p, e, xs[sl], 0)   # (nq, p+1)
        s0 = int(np.searchsorted(knots, e / n, side="right")) - 1 - p
        E[:, s0:s0 + p + 1] += (card[:, sl] * ws[None, sl]) @ B
    coef = np.linalg.solve(Mfull, E.T).T       # rows: cardinal k
    return coef, ks


def V_reg_matrix(n: int, p: int, dirichlet, return_dropped: bool = False, rep=None):
    """V_reg: coordinates of the special basis in the kept B-spline basis
    (with the repeated knots ``rep``: the regular space is unchanged,
    Remark "reduced_regularity", only its coordinates change)."""
    D = normalize_dirichlet(dirichlet)
    coef, ks = cardinal_coefficients(n, p, rep)
    row = {k: r for r, k in enumerate(ks)}
    combos = special_basis_combinations(n, p, D)
    size = coef.shape[1]
    full = np.zeros((size, len(combos)))
    for j, c in enumerate(combos):
        for v, k in c:
            full[:, j] += v * coef[row[k]]
    keep = kept_indices(n, p, D, rep)
    dropped = np.setdiff1d(np.arange(size), keep)
    V = full[keep, :]
    if return_dropped:
        return V, full[dropped, :]
    return V


# ---------------------------------------------------- 1D eigendata
@dataclass
class AxisSplit:
    """All 1D data of one parametric direction."""
    n: int
    p: int
    dirichlet: frozenset
    M: np.ndarray
    K: np.ndarray
    V_reg: np.ndarray
    V_out: np.ndarray
    U: np.ndarray
    Dt: np.ndarray          # diagonal of D~_reg
    lam_reg: np.ndarray
    Q_out: np.ndarray
    lam_out: np.ndarray
    Qt: np.ndarray          # Q~ (m x m)
    lamt: np.ndarray        # diagonal of Lambda~

    @property
    def m(self) -> int:
        return self.M.shape[0]

    @property
    def n_reg(self) -> int:
        return self.V_reg.shape[1]

    @property
    def n_out(self) -> int:
        return self.V_out.shape[1]


def axis_split(n: int, p: int, dirichlet=(0, 1), rep=None) -> AxisSplit:
    """Build Q~ and Lambda~ of one direction (Sections 4 and 6); ``rep`` =
    {k: extra} repeats interior knots (Remark "reduced_regularity": the regular
    space and its transform are unchanged, S^out grows by one per extra knot)."""
    D = normalize_dirichlet(dirichlet)
    Mf, Kf = assemble_full(n, p, rep=rep)
    keep = kept_indices(n, p, D, rep)
    M = Mf[np.ix_(keep, keep)]
    K = Kf[np.ix_(keep, keep)]
    V = V_reg_matrix(n, p, D, rep=rep)
    U = U_reg(n, p, D)
    # D~_reg = (U^T V_reg^T M V_reg U)^{1/2} (end of Section 6). Lambda_reg from
    # Lemma 3: the numeric diag(U^T V_reg^T K V_reg U) / D~^2 of eq. "Lambda reg"
    # loses ~1e-13 on the lowest modes to the conditioning of K (it is kept as
    # a pin in the tests).
    MU = U.T @ (V.T @ M @ V) @ U
    Dt = np.sqrt(np.diag(MU))
    lam_reg = lambda_reg_closed_form(n, p, D)
    # V_out = M^{-1} N, N orthonormal basis of range(V_reg)^perp (Section 4)
    N = scipy.linalg.null_space(V.T)
    if N.shape[1] > 0:
        Vout = np.linalg.solve(M, N)
        lam_out, Q_out = scipy.linalg.eigh(Vout.T @ K @ Vout, Vout.T @ M @ Vout)
    else:
        Vout = np.zeros((M.shape[0], 0))
        lam_out, Q_out = np.zeros(0), np.zeros((0, 0))
    Qt = np.hstack([V @ U / Dt[None, :], Vout @ Q_out])
    lamt = np.concatenate([lam_reg, lam_out])
    return AxisSplit(n, p, D, M, K, V, Vout, U, Dt, lam_reg, Q_out, lam_out, Qt, lamt)


def ktilde_basis_free(M: np.ndarray, K: np.ndarray, V_reg: np.ndarray) -> np.ndarray:
    """K~ from the subspace S^reg alone (proof of the Corollary, Section 4):
    P_r = V_reg (V_reg^T M V_reg)^{-1} V_reg^T M is the M-orthogonal projector
    onto S^reg, P_o = I - P_r, and K~ = P_r^T K P_r + P_o^T K P_o."""
    Pr = V_reg @ np.linalg.solve(V_reg.T @ M @ V_reg, V_reg.T @ M)
    Po = np.eye(M.shape[0]) - Pr
    return Pr.T @ K @ Pr + Po.T @ K @ Po


# ------------------------------------------------------- closed forms
def cardinal_symbol(q: int, kmax: int, theta) -> np.ndarray:
    """sum_{k=-kmax}^{kmax} B~_q(k) cos(k theta)."""
    theta = np.asarray(theta, dtype=np.float64)
    ks = np.arange(-kmax, kmax + 1)
    vals = cardinal_bspline(q, ks.astype(np.float64))
    return np.cos(np.multiply.outer(theta, ks)) @ vals


def theta_closed_form(n: int, p: int, dirichlet) -> np.ndarray:
    """Diagonal of Theta in Theorem 3."""
    _, alpha, _ = table1(n, p, dirichlet)
    return cardinal_symbol(p, p // 2, alpha / n)


def lambda_reg_closed_form(n: int, p: int, dirichlet) -> np.ndarray:
    """Lambda_reg of Lemma 3 with the factor read as (2 - 2 cos h alpha)/h^2."""
    _, alpha, _ = table1(n, p, dirichlet)
    h = 1.0 / n
    t = h * alpha
    sk = cardinal_symbol(2 * p - 1, p - 1, t)
    sm = cardinal_symbol(2 * p + 1, p, t)
    # 2 - 2 cos t written as 4 sin^2(t/2): the same number without cancellation
    return 4.0 * np.sin(0.5 * t) ** 2 / h ** 2 * sk / sm


def dtilde_closed_form(n: int, p: int, dirichlet) -> np.ndarray:
    """D~_reg = D_reg Theta derived from the periodic symbols.

    With q_i = sin(x_i alpha_j + beta) on the 4n periodic nodes, the periodic
    mass matrix has symbol h * sigma_M(h alpha_j), sigma_M(t) = sum_{|k|<=p}
    B~_{2p+1}(k) cos(k t), and collocation has symbol Theta_jj. Hence
    ||F_j||^2_{L2(0,1)} = (h/4) sigma_M ||q||^2 / Theta_jj^2 and
    D~_jj^2 = sigma_M(h alpha_j) * mean_i q_i^2 (the mean over the 4n nodes is
    1/2 except for modes with h alpha_j in {0, pi})."""
    x, alpha, beta = table1(n, p, dirichlet)
    h = 1.0 / n
    sm = cardinal_symbol(2 * p + 1, p, h * alpha)
    per = node(np.arange(-2 * n + 1, 2 * n + 1), n, p)
    mean_q2 = np.mean(np.sin(np.outer(per, alpha) + beta) ** 2, axis=0)
    return np.sqrt(sm * mean_q2)


def collocation_matrix(n: int, p: int, dirichlet) -> np.ndarray:
    """C_reg[i, j] = B^_j(x_i) with the row nodes of Table 1 (Theorem 3)."""
    x, _, _ = table1(n, p, dirichlet)
    h = 1.0 / n
    combos = special_basis_combinations(n, p, dirichlet)
    C = np.zeros((len(x), len(combos)))
    for j, c in enumerate(combos):
        for v, k in c:
            C[:, j] += v * cardinal_bspline(p, (x - node(k, n, p)) / h)
    return C
