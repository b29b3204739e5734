// Host-side univariate IFFD setup (Sections 2, 4, 5 and 6 of the paper).
//
// Builds, for one parametric direction with Dirichlet set D (any subset of
// {0, 1}; the eight (parity of p, D) cases of Table 1):
//   * banded M and K of S_{p,h,D} by Cox-de Boor + (p+1)-point Gauss (Section 2);
//   * the edge blocks of V_reg in the special basis of Section 6 (eq.
//     "special_basis"), obtained exactly by Boehm knot insertion: inserting the
//     knot 0 p times into the uniform (cardinal) knot vector turns every cardinal
//     B-spline into a combination of the open-knot B-splines;
//   * V_out = M^{-1} G^T, G the derivative functionals of eq. "reg_space" (its
//     columns span the L2-orthogonal complement of S^reg), and Q_out, Lambda_out
//     of eq. "eigendecomposition_out" by Cholesky + cyclic Jacobi;
//   * Lambda_reg from Lemma 3 (with the factor (2 - 2cos t)/h^2 written as
//     4 sin^2(t/2)/h^2) and D~_reg = D_reg Theta from the periodic symbols:
//     D~_jj^2 = sigma_M(h alpha_j) * mean_i sin^2(x_i alpha_j + beta), which
//     equals the paper's numeric definition (U^T V_reg^T M V_reg U)^{1/2};
//   * the parameters of the generic transform of the six cases other than
//     D = {0,1}: U_ij = sin(pi (i - c)(j - e) / n + beta) (Table 1), evaluated
//     through a zero-padded DFT of length 2n (c, e integers) or 4n.
#include "host_setup.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <sstream>

namespace iffd {

namespace {

const double kPi = 3.14159265358979323846264338327950288;

// Gauss-Legendre nodes/weights on [-1,1] by Newton's method on P_q.
void gauss_legendre(int q, std::vector<double>* x, std::vector<double>* w) {
  x->assign(q, 0.0);
  w->assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    double t = std::cos(kPi * (i + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= q; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (q == 1) { p1 = t; p0 = 1.0; }
      dp = q * (t * p1 - p0) / (t * t - 1.0);
      double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double p0 = 1.0, p1 = t;
    for (int k = 2; k <= q; ++k) {
      double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    if (q == 1) { p1 = t; p0 = 1.0; }
    dp = q * (t * p1 - p0) / (t * t - 1.0);
    (*x)[i] = t;
    (*w)[i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

// Open uniform knot vector xi_0..xi_{n+2p} on [0,1].
std::vector<double> open_knots(int n, int p) {
  std::vector<double> k;
  for (int i = 0; i <= p; ++i) k.push_back(0.0);
  for (int i = 1; i < n; ++i) k.push_back(double(i) / n);
  for (int i = 0; i <= p; ++i) k.push_back(1.0);
  return k;
}

// Values (order 0) or derivatives (order r) of B_{p,e..e+p} at x on element e.
// Cox-de Boor for degree p-r, then r steps of the derivative recursion.
void bspline_local(const std::vector<double>& kn, int p, int e, double x, int r, double* out) {
  const int s = p + e;
  std::vector<double> cur(p + 2, 0.0), nxt(p + 2, 0.0);
  // cur[t] holds B_{d, s-d+t}, t = 0..d
  cur[0] = 1.0;
  int q = p - r;
  if (q < 0) {
    for (int t = 0; t <= p; ++t) out[t] = 0.0;
    return;
  }
  for (int d = 1; d <= q; ++d) {
    for (int t = 0; t <= d; ++t) {
      const int i = s - d + t;
      double acc = 0.0;
      // B_{d-1,i} is cur[t-1] (index i = s-(d-1)+(t-1)), B_{d-1,i+1} is cur[t]
      if (t - 1 >= 0) {
        const double den = kn[i + d] - kn[i];
        if (den != 0.0) acc += (x - kn[i]) / den * cur[t - 1];
      }
      if (t <= d - 1) {
        const double den = kn[i + d + 1] - kn[i + 1];
        if (den != 0.0) acc += (kn[i + d + 1] - x) / den * cur[t];
      }
      nxt[t] = acc;
    }
    std::swap(cur, nxt);
  }
  for (int d = q + 1; d <= p; ++d) {
    for (int t = 0; t <= d; ++t) {
      const int i = s - d + t;
      double acc = 0.0;
      if (t - 1 >= 0) {
        const double den = kn[i + d] - kn[i];
        if (den != 0.0) acc += d * cur[t - 1] / den;
      }
      if (t <= d - 1) {
        const double den = kn[i + d + 1] - kn[i + 1];
        if (den != 0.0) acc -= d * cur[t] / den;
      }
      nxt[t] = acc;
    }
    std::swap(cur, nxt);
  }
  for (int t = 0; t <= p; ++t) out[t] = cur[t];
}

// Banded Cholesky of an SPD band matrix (half bandwidth b, band layout
// A[i*(2b+1) + (j-i+b)]); L stored as L[i*(b+1) + (i-j)] for j = i-b..i.
bool band_cholesky(const std::vector<double>& A, int m, int b, std::vector<double>* L) {
  L->assign((size_t)m * (b + 1), 0.0);
  auto Lat = [&](int i, int j) -> double& { return (*L)[(size_t)i * (b + 1) + (i - j)]; };
  for (int i = 0; i < m; ++i) {
    for (int j = std::max(0, i - b); j <= i; ++j) {
      double s = A[(size_t)i * (2 * b + 1) + (j - i + b)];
      for (int k = std::max(0, i - b); k < j; ++k) {
        if (j - k > b) continue;
        s -= Lat(i, k) * Lat(j, k);
      }
      if (i == j) {
        if (s <= 0.0) return false;
        Lat(i, i) = std::sqrt(s);
      } else {
        Lat(i, j) = s / Lat(j, j);
      }
    }
  }
  return true;
}

void band_solve(const std::vector<double>& L, int m, int b, double* x) {
  auto Lat = [&](int i, int j) { return L[(size_t)i * (b + 1) + (i - j)]; };
  for (int i = 0; i < m; ++i) {
    double s = x[i];
    for (int k = std::max(0, i - b); k < i; ++k) s -= Lat(i, k) * x[k];
    x[i] = s / Lat(i, i);
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = x[i];
    for (int k = i + 1; k <= std::min(m - 1, i + b); ++k) s -= Lat(k, i) * x[k];
    x[i] = s / Lat(i, i);
  }
}

void band_matvec(const std::vector<double>& A, int m, int b, const double* x, double* y) {
  for (int i = 0; i < m; ++i) {
    double s = 0.0;
    for (int j = std::max(0, i - b); j <= std::min(m - 1, i + b); ++j)
      s += A[(size_t)i * (2 * b + 1) + (j - i + b)] * x[j];
    y[i] = s;
  }
}

// Cyclic Jacobi eigendecomposition of a dense symmetric n x n matrix (row-major).
// On return A's diagonal holds the eigenvalues and V (row-major, columns =
// eigenvectors) the orthonormal eigenvectors.
void jacobi_eig(std::vector<double>& A, int n, std::vector<double>* V) {
  V->assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) (*V)[(size_t)i * n + i] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  auto v = [&](int i, int j) -> double& { return (*V)[(size_t)i * n + j]; };
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += a(i, j) * a(i, j);
        if (i != j) off += a(i, j) * a(i, j);
      }
    if (off <= 1e-32 * tot) break;
    for (int pp = 0; pp < n - 1; ++pp) {
      for (int qq = pp + 1; qq < n; ++qq) {
        const double apq = a(pp, qq);
        if (apq == 0.0) continue;
        const double theta = (a(qq, qq) - a(pp, pp)) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
          const double akp = a(k, pp), akq = a(k, qq);
          a(k, pp) = c * akp - s * akq;
          a(k, qq) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
          const double apk = a(pp, k), aqk = a(qq, k);
          a(pp, k) = c * apk - s * aqk;
          a(qq, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = v(k, pp), vkq = v(k, qq);
          v(k, pp) = c * vkp - s * vkq;
          v(k, qq) = s * vkp + c * vkq;
        }
      }
    }
  }
}

// Generalized symmetric-definite eigenproblem Ka q = lambda Ma q (dense,
// row-major n x n): Ma = L L^T, C = L^{-1} Ka L^{-T}, C = Y diag Y^T,
// Q = L^{-T} Y (Q^T Ma Q = I). Eigenpairs sorted ascending.
bool gen_eig(const std::vector<double>& Ka, const std::vector<double>& Ma, int n,
             std::vector<double>* Q, std::vector<double>* lam) {
  std::vector<double> L((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = Ma[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      if (i == j) {
        if (s <= 0) return false;
        L[(size_t)i * n + i] = std::sqrt(s);
      } else {
        L[(size_t)i * n + j] = s / L[(size_t)j * n + j];
      }
    }
  // X = L^{-1} Ka  (forward substitution on columns)
  std::vector<double> X(Ka);
  for (int c = 0; c < n; ++c)
    for (int i = 0; i < n; ++i) {
      double s = X[(size_t)i * n + c];
      for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * X[(size_t)k * n + c];
      X[(size_t)i * n + c] = s / L[(size_t)i * n + i];
    }
  // C = X L^{-T}: C^T = L^{-1} X^T
  std::vector<double> C((size_t)n * n);
  for (int r = 0; r < n; ++r)
    for (int i = 0; i < n; ++i) {
      double s = X[(size_t)r * n + i];
      for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * C[(size_t)r * n + k];
      C[(size_t)r * n + i] = s / L[(size_t)i * n + i];
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      const double sym = 0.5 * (C[(size_t)i * n + j] + C[(size_t)j * n + i]);
      C[(size_t)i * n + j] = C[(size_t)j * n + i] = sym;
    }
  std::vector<double> Y;
  jacobi_eig(C, n, &Y);
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(),
            [&](int a, int b) { return C[(size_t)a * n + a] < C[(size_t)b * n + b]; });
  lam->assign(n, 0.0);
  Q->assign((size_t)n * n, 0.0);
  for (int jj = 0; jj < n; ++jj) {
    const int j = order[jj];
    (*lam)[jj] = C[(size_t)j * n + j];
    // q = L^{-T} y  (back substitution)
    std::vector<double> q(n);
    for (int i = n - 1; i >= 0; --i) {
      double s = Y[(size_t)i * n + j];
      for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * q[k];
      q[i] = s / L[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) (*Q)[(size_t)i * n + jj] = q[i];
  }
  return true;
}

// Boehm insertion of knot t into (kn, c): c[i] is the coefficient of the
// degree-p B-spline on kn[i..i+p+1].
void insert_knot(std::vector<double>* kn, std::vector<double>* c, int p, double t) {
  const std::vector<double>& k = *kn;
  int s = -1;
  for (int i = 0; i + 1 < (int)k.size(); ++i)
    if (k[i] <= t && t < k[i + 1]) s = i;
  std::vector<double> nc(c->size() + 1, 0.0);
  for (int i = 0; i < (int)nc.size(); ++i) {
    if (i <= s - p) {
      nc[i] = (*c)[i];
    } else if (i >= s + 1) {
      nc[i] = (*c)[i - 1];
    } else {
      const double a = (t - k[i]) / (k[i + p] - k[i]);
      nc[i] = (1.0 - a) * (*c)[i - 1] + a * (*c)[i];
    }
  }
  kn->insert(kn->begin() + s + 1, t);
  *c = nc;
}

// Banded M and K of S_{p,h,D} (B-spline 0 removed if dir0, n+p-1 if dir1),
// with an optional weight w(x) under both integrals; (p+1)-point Gauss per element.
void assemble_bands(int n, int p, bool dir0, bool dir1, double (*w)(double), std::vector<double>* Mb,
                    std::vector<double>* Kb) {
  const int m = n + p - (dir0 ? 1 : 0) - (dir1 ? 1 : 0), bw = 2 * p + 1, F = n + p;
  const int s0 = dir0 ? 1 : 0;
  const std::vector<double> kn = open_knots(n, p);
  std::vector<double> gx, gw;
  gauss_legendre(p + 1, &gx, &gw);
  std::vector<double> Mf((size_t)F * bw, 0.0), Kf((size_t)F * bw, 0.0);
  std::vector<double> B(p + 1), dB(p + 1);
  for (int e = 0; e < n; ++e) {
    const double a = double(e) / n, b = double(e + 1) / n;
    for (int g = 0; g <= p; ++g) {
      const double x = 0.5 * (b - a) * gx[g] + 0.5 * (a + b);
      double wt = 0.5 * (b - a) * gw[g];
      if (w) wt *= w(x);
      bspline_local(kn, p, e, x, 0, B.data());
      bspline_local(kn, p, e, x, 1, dB.data());
      for (int s = 0; s <= p; ++s)
        for (int t = 0; t <= p; ++t) {
          const int i = e + s, j = e + t;
          Mf[(size_t)i * bw + (j - i + p)] += wt * B[s] * B[t];
          Kf[(size_t)i * bw + (j - i + p)] += wt * dB[s] * dB[t];
        }
    }
  }
  Mb->assign((size_t)m * bw, 0.0);
  Kb->assign((size_t)m * bw, 0.0);
  for (int i = 0; i < m; ++i)
    for (int d = 0; d < bw; ++d) {
      const int j = i + d - p;
      if (j < 0 || j >= m) continue;
      (*Mb)[(size_t)i * bw + d] = Mf[(size_t)(i + s0) * bw + d];
      (*Kb)[(size_t)i * bw + d] = Kf[(size_t)(i + s0) * bw + d];
    }
}

double sin_2pi(double x) { return std::sin(2.0 * kPi * x); }

}  // namespace

double cardinal_half(int q, int twice_x) {
  // T_d[k] = B~_d(k/2); recurrence of Lemma 3 (eq. "cardinal") in half-units:
  // B~_d(k/2) = (d+1+k)/(2d) B~_{d-1}((k+1)/2) + (d+1-k)/(2d) B~_{d-1}((k-1)/2).
  static std::map<std::pair<int, int>, double> memo;
  const int K = q + 3;
  if (twice_x < -K || twice_x > K) return 0.0;
  auto key = std::make_pair(q, twice_x);
  auto it = memo.find(key);
  if (it != memo.end()) return it->second;
  std::vector<double> cur(2 * K + 3, 0.0), nxt(2 * K + 3, 0.0);
  auto at = [&](std::vector<double>& v, int k) -> double& { return v[k + K + 1]; };
  at(cur, -1) = 1.0;  // B~_0 = 1 on [-1/2, 1/2)
  at(cur, 0) = 1.0;
  for (int d = 1; d <= q; ++d) {
    for (int k = -K; k <= K; ++k) {
      const double left = (k + 1 <= K + 1) ? at(cur, k + 1) : 0.0;
      const double right = (k - 1 >= -K - 1) ? at(cur, k - 1) : 0.0;
      at(nxt, k) = (d + 1.0 + k) / (2.0 * d) * left + (d + 1.0 - k) / (2.0 * d) * right;
    }
    std::swap(cur, nxt);
  }
  const double r = at(cur, twice_x);
  memo[key] = r;
  return r;
}

bool fft_factor(int L, std::vector<int>* radices) {
  radices->clear();
  if (L < 1) return false;
  int x = L;
  while (x % 8 == 0) { radices->push_back(8); x /= 8; }
  while (x % 4 == 0) { radices->push_back(4); x /= 4; }
  while (x % 2 == 0) { radices->push_back(2); x /= 2; }
  for (int r = 3; r * r <= x || (x > 1 && r <= x); r += 2) {
    while (x % r == 0) { radices->push_back(r); x /= r; }
    if (x == 1) break;
  }
  if (x > 1) radices->push_back(x);
  return true;
}

namespace {

// Edge block of the special basis at the end x = 0 for one end type (Section
// 6, eq. "special_basis"): Dirichlet (dir) B~_i - B~_{dp-i}, i = 1..floor(p/2);
// otherwise, p even, B~_i + B~_{1-i}, i = 1..p/2, and p odd, B~_0 and
// B~_i + B~_{-i}, i = 1..(p-1)/2. Each combination of cardinal B-splines is
// written in the open-knot basis exactly by inserting the knot 0 p times into
// the uniform knot vector (Boehm). V[r * nfun + c]: coefficient of function c
// on the reduced basis function r counted from the end (the B-spline at the
// end itself is removed when dir). The right end is the mirror image.
std::string edge_block(int p, bool dir, int* nfun, int* rows, std::vector<double>* V) {
  const int half = p / 2;
  const int dp = (p % 2 == 1) ? 0 : 1;
  std::vector<std::vector<std::pair<double, int>>> combos;
  if (dir) {
    for (int i = 1; i <= half; ++i) combos.push_back({{1.0, i}, {-1.0, dp - i}});
  } else if (p % 2 == 0) {
    for (int i = 1; i <= half; ++i) combos.push_back({{1.0, i}, {1.0, 1 - i}});
  } else {
    combos.push_back({{1.0, 0}});
    for (int i = 1; i <= (p - 1) / 2; ++i) combos.push_back({{1.0, i}, {1.0, -i}});
  }
  *nfun = (int)combos.size();
  const int J0 = -3 * p - 4, J1 = 3 * p + 4;
  const int s0 = dir ? 1 : 0;
  std::vector<std::vector<double>> cols;
  int maxrow = -1;
  for (const auto& cb : combos) {
    std::vector<double> knots;
    for (int j = J0; j <= J1; ++j) knots.push_back(double(j));
    std::vector<double> coef(knots.size() - p - 1, 0.0);
    // B~_k is the uniform B-spline starting at knot k - floor(p/2) - 1
    for (const auto& t : cb) coef[(t.second - half - 1) - J0] += t.first;
    for (int r = 0; r < p; ++r) insert_knot(&knots, &coef, p, 0.0);
    int z = 0;
    while (knots[z] != 0.0) ++z;
    // open B-spline with full index jf (counted from x = 0) <-> coef[z + jf]
    if (dir && std::fabs(coef[z]) > 1e-13) return "special basis function does not vanish at a Dirichlet end";
    std::vector<double> col;
    for (int jf = s0; jf <= 2 * p + 2; ++jf) col.push_back(coef[z + jf]);
    for (int r = 0; r < (int)col.size(); ++r)
      if (std::fabs(col[r]) > 1e-13) maxrow = std::max(maxrow, r);
    cols.push_back(col);
  }
  *rows = maxrow + 1;
  if (*rows > 2 * p) return "special basis edge function is not local";
  V->assign((size_t)(*rows) * (*nfun), 0.0);
  for (int c = 0; c < *nfun; ++c)
    for (int r = 0; r < *rows; ++r) (*V)[(size_t)r * (*nfun) + c] = cols[c][r];
  return "";
}

// Rows of the constraint matrix G of eq. "reg_space" for the end x = 0 on the
// reduced basis (counted from the end): derivatives of orders 2, 4, .. (Dirichlet
// end) or 1, 3, .. (otherwise) up to p - 1 of the open B-splines at 0.
void end_constraints(const std::vector<double>& kn, int p, bool dir, int m, std::vector<std::vector<double>>* G) {
  std::vector<double> d(p + 1);
  const int s0 = dir ? 1 : 0;
  for (int ord = dir ? 2 : 1; ord <= p - 1; ord += 2) {
    bspline_local(kn, p, 0, 0.0, ord, d.data());
    std::vector<double> row(m, 0.0);
    for (int jf = s0; jf <= p && jf - s0 < m; ++jf) row[jf - s0] = d[jf];
    G->push_back(row);
  }
}

}  // namespace

std::string build_axis(int n, int p, bool dir0, bool dir1, Axis1D* A) {
  std::ostringstream err;
  if (p < 1 || p > 16) { err << "degree p=" << p << " outside 1..16"; return err.str(); }
  if (n <= p) { err << "n=" << n << " must exceed p=" << p; return err.str(); }
  A->n = n;
  A->p = p;
  A->dir0 = dir0;
  A->dir1 = dir1;
  A->m = n + p - (dir0 ? 1 : 0) - (dir1 ? 1 : 0);
  const int m = A->m;

  // ---- banded M, K of S_{p,h,D}
  assemble_bands(n, p, dir0, dir1, nullptr, &A->Mband, &A->Kband);
  const std::vector<double> kn = open_knots(n, p);

  // ---- special basis: edge blocks (knot insertion) and the interior functions
  std::string e = edge_block(p, dir0, &A->nL, &A->rowsL, &A->VL);
  if (!e.empty()) return e;
  e = edge_block(p, dir1, &A->nR, &A->rowsR, &A->VR);
  if (!e.empty()) return e;
  // interior special function i = floor(p/2)+1 .. n-ceil(p/2) is the open
  // B-spline with full index i + floor((p-1)/2) (p odd) or i + p/2 - 1 (p even)
  const int n_int = n - p;
  A->n_reg = A->nL + n_int + A->nR;
  A->n_out = m - A->n_reg;
  const int first_full = (p / 2 + 1) + ((p % 2 == 1) ? (p - 1) / 2 : p / 2 - 1);
  A->o = first_full - (dir0 ? 1 : 0) - A->nL;
  // the device passes give every row of V_reg to one region: left block,
  // interior, or right block
  if (A->rowsL > A->nL + A->o || m - A->rowsR < A->nL + A->o + n_int || A->rowsL > m - A->rowsR)
    return "n too small for the device layout of the special basis";

  // ---- Table 1: nodes x_i = (i - c) h, alpha_j = (j - e) pi, beta
  const bool odd = (p % 2 == 1);
  double c, ee, beta;
  if (odd) c = dir0 ? 0.0 : 1.0;
  else c = 0.5;
  if (dir0 && dir1) ee = 0.0;
  else if (dir0 || dir1) ee = 0.5;
  else ee = 1.0;
  beta = (dir1 && !dir0) || (!dir0 && !dir1) ? 0.5 * kPi : 0.0;
  if (dir0 && dir1) A->kind = odd ? TK_DST1 : TK_DST23;
  else A->kind = TK_GEN;
  A->gq = (c != std::floor(c) || ee != std::floor(ee)) ? 2 : 1;
  A->gqc = (int)std::lround(A->gq * c);
  A->gqe = (int)std::lround(A->gq * ee);

  // ---- Lambda_reg (Lemma 3) and D~_reg (periodic symbols)
  const double h = 1.0 / n;
  A->lam.assign(m, 0.0);
  A->dtilde.assign(A->n_reg, 0.0);
  for (int j = 0; j < A->n_reg; ++j) {
    const double alpha = (j + 1 - ee) * kPi;
    const double t = h * alpha;
    double sM = cardinal_half(2 * p + 1, 0), sK = cardinal_half(2 * p - 1, 0);
    for (int k = 1; k <= p; ++k) sM += 2.0 * cardinal_half(2 * p + 1, 2 * k) * std::cos(k * t);
    for (int k = 1; k <= p - 1; ++k) sK += 2.0 * cardinal_half(2 * p - 1, 2 * k) * std::cos(k * t);
    const double s2 = std::sin(0.5 * t);
    A->lam[j] = 4.0 * s2 * s2 / (h * h) * sK / sM;
    // mean of sin^2(x_i alpha_j + beta) over the 4n periodic nodes x_i = (i - c') h,
    // i = -2n+1..2n (c' = 0 for odd p, 1/2 for even p): 1/2 unless h alpha_j is a
    // multiple of pi, where the sum is taken exactly
    double meanq2 = 0.5;
    const double jm = j + 1 - ee;
    if (std::fabs(jm) < 1e-12 || std::fabs(jm - n) < 1e-12) {
      double acc = 0.0;
      for (int i = -2 * n + 1; i <= 2 * n; ++i) {
        const double x = (i - (odd ? 0.0 : 0.5)) * h;
        const double q = std::sin(x * alpha + beta);
        acc += q * q;
      }
      meanq2 = acc / (4.0 * n);
    }
    A->dtilde[j] = std::sqrt(sM * meanq2);
    if (!(A->dtilde[j] > 0.0)) return "degenerate regular mode (D~ = 0)";
  }
  // generic transform (Table 1 cases other than D = {0,1}): with
  // T(k) = sum_l s_l exp(+2 pi i l k / L), L = 2 n q, of the zero-padded real
  // sequence s (entries l = 1..n_reg), sin(theta (i - c)(j - e) + beta) gives
  //   FWD  y_j = Im(w_j T(q (j - e))) / D~_j,  w_j = exp(i (beta - pi c (j - e) / n)),
  //   BWD  x_i = Im(v_i T(q (i - c))),         v_i = exp(i (beta - pi e (i - c) / n)),
  // and the BWD input is pre-scaled by 1 / D~_j. Two real pencils share one
  // complex sequence; separating them costs a factor 1/2, folded in here.
  A->gpost.clear();
  if (A->kind == TK_GEN) {
    const int N = A->n_reg;
    for (int j = 1; j <= N; ++j) {
      const double ang = beta - kPi * c * (j - ee) / n;
      A->gpost.push_back(0.5 * std::cos(ang) / A->dtilde[j - 1]);
      A->gpost.push_back(0.5 * std::sin(ang) / A->dtilde[j - 1]);
    }
    for (int i = 1; i <= N; ++i) {
      const double ang = beta - kPi * ee * (i - c) / n;
      A->gpost.push_back(0.5 * std::cos(ang));
      A->gpost.push_back(0.5 * std::sin(ang));
    }
    for (int j = 1; j <= N; ++j) A->gpost.push_back(1.0 / A->dtilde[j - 1]);
  }

  // ---- remainder space: V_out = M^{-1} G^T, then Q_out, Lambda_out
  const int no = A->n_out;
  A->W.assign((size_t)m * no, 0.0);
  A->wlo = 0;
  A->whi = m;
  if (no > 0) {
    std::vector<std::vector<double>> G, GR;  // rows over the reduced basis
    end_constraints(kn, p, dir0, m, &G);
    end_constraints(kn, p, dir1, m, &GR);
    // orthonormalise each end's rows (modified Gram-Schmidt; derivative values
    // scale like h^-k), mirror the right end's rows
    auto orthonormalise = [&](std::vector<std::vector<double>>& R) {
      for (size_t a = 0; a < R.size(); ++a) {
        for (size_t b = 0; b < a; ++b) {
          double dot = 0;
          for (int i = 0; i < m; ++i) dot += R[a][i] * R[b][i];
          for (int i = 0; i < m; ++i) R[a][i] -= dot * R[b][i];
        }
        double nr = 0;
        for (int i = 0; i < m; ++i) nr += R[a][i] * R[a][i];
        nr = std::sqrt(nr);
        for (int i = 0; i < m; ++i) R[a][i] /= nr;
      }
    };
    orthonormalise(G);
    orthonormalise(GR);
    for (const auto& r : GR) {
      std::vector<double> row(m, 0.0);
      for (int i = 0; i < m; ++i) row[m - 1 - i] = r[i];
      G.push_back(row);
    }
    if ((int)G.size() != no) return "constraint count differs from n_out";
    std::vector<double> Lm;
    if (!band_cholesky(A->Mband, m, p, &Lm)) return "mass matrix is not positive definite";
    std::vector<double> Vout((size_t)m * no);  // column-major: Vout[i + k*m]
    for (int k = 0; k < no; ++k) {
      std::vector<double> x(G[k]);
      band_solve(Lm, m, p, x.data());
      for (int i = 0; i < m; ++i) Vout[i + (size_t)k * m] = x[i];
    }
    std::vector<double> Mo((size_t)no * no), Ko((size_t)no * no), tmp(m);
    for (int b = 0; b < no; ++b) {
      band_matvec(A->Kband, m, p, &Vout[(size_t)b * m], tmp.data());
      for (int a = 0; a < no; ++a) {
        double sm = 0, sk = 0;
        for (int i = 0; i < m; ++i) {
          sm += G[a][i] * Vout[i + (size_t)b * m];
          sk += Vout[i + (size_t)a * m] * tmp[i];
        }
        Mo[(size_t)a * no + b] = sm;
        Ko[(size_t)a * no + b] = sk;
      }
    }
    for (int a = 0; a < no; ++a)
      for (int b = 0; b < a; ++b) {
        const double s1 = 0.5 * (Mo[(size_t)a * no + b] + Mo[(size_t)b * no + a]);
        const double s2 = 0.5 * (Ko[(size_t)a * no + b] + Ko[(size_t)b * no + a]);
        Mo[(size_t)a * no + b] = Mo[(size_t)b * no + a] = s1;
        Ko[(size_t)a * no + b] = Ko[(size_t)b * no + a] = s2;
      }
    std::vector<double> Qo, lo;
    if (!gen_eig(Ko, Mo, no, &Qo, &lo)) return "remainder mass matrix is not positive definite";
    double wmax = 0.0;
    for (int i = 0; i < m; ++i)
      for (int k = 0; k < no; ++k) {
        double s = 0;
        for (int a = 0; a < no; ++a) s += Vout[i + (size_t)a * m] * Qo[(size_t)a * no + k];
        A->W[(size_t)i * no + k] = s;
        wmax = std::max(wmax, std::fabs(s));
      }
    for (int k = 0; k < no; ++k) A->lam[A->n_reg + k] = lo[k];
    // support: the maximal block of rows around the middle whose entries are all
    // below 1e-17 max|W| is dropped (W decays geometrically away from both ends)
    auto small = [&](int i) {
      for (int k = 0; k < no; ++k)
        if (std::fabs(A->W[(size_t)i * no + k]) > 1e-17 * wmax) return false;
      return true;
    };
    const int mid = m / 2;
    if (small(mid)) {
      int lo_i = mid, hi_i = mid;
      while (lo_i > 0 && small(lo_i - 1)) --lo_i;
      while (hi_i < m && small(hi_i)) ++hi_i;
      A->wlo = lo_i;
      A->whi = hi_i;
    } else {
      A->wlo = m;
      A->whi = m;
    }
  }
  return "";
}

void build_weighted_bands(Axis1D* A) {
  assemble_bands(A->n, A->p, A->dir0, A->dir1, sin_2pi, &A->Msband, &A->Ksband);
}

std::string exact_fd_axis(const Axis1D& ax, std::vector<double>* Q, std::vector<double>* lam) {
  const int m = ax.m, p = ax.p, bw = 2 * p + 1;
  std::vector<double> Md((size_t)m * m, 0.0), Kd((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i)
    for (int d = 0; d < bw; ++d) {
      const int j = i + d - p;
      if (j < 0 || j >= m) continue;
      Md[(size_t)i * m + j] = ax.Mband[(size_t)i * bw + d];
      Kd[(size_t)i * m + j] = ax.Kband[(size_t)i * bw + d];
    }
  std::vector<double> Qr;
  if (!gen_eig(Kd, Md, m, &Qr, lam)) return "exact FD: mass matrix is not positive definite";
  Q->assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) (*Q)[i + (size_t)j * m] = Qr[(size_t)i * m + j];
  return "";
}

}  // namespace iffd
