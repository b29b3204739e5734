// Host-side univariate IFFD setup (Sections 2, 4, 5 and 6 of the paper).
//
// Builds, for one parametric direction with Dirichlet set D (any subset of
// {0, 1}; the eight (parity of p, D) cases of Table 1):
//   * banded M and K of S_{p,h,D} by Cox-de Boor + (p+1)-point Gauss (Section 2);
//   * V_reg in the special basis of Section 6 (eq. "special_basis"), obtained
//     exactly by Boehm knot insertion: inserting the knots 0 and 1 p times (and
//     every repeated interior knot its extra times) into the uniform (cardinal)
//     knot vector turns every cardinal B-spline into a combination of the
//     open-knot B-splines; stored as edge blocks, identity runs and, around
//     repeated knots (Remark "reduced_regularity"), small dense blocks;
//   * V_out = M^{-1} G^T, G the derivative functionals of eq. "reg_space" and,
//     at repeated knots, the derivative jumps that S^reg forbids (its columns
//     span the L2-orthogonal complement of S^reg), and Q_out, Lambda_out
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

// p-open knot vector on the uniform grid z_k = k/n (Section 2): p+1 copies
// of 0, the interior breakpoints, p+1 copies of 1. A breakpoint k listed in
// `reps` as (k, e) appears 1 + e times (reduced regularity C^{p-1-e} there,
// Remark "reduced_regularity").
// With unit_h the knots are given in units of h (the integers 0..n).
std::vector<double> open_knots(int n, int p, const std::vector<std::pair<int, int>>& reps = {},
                               bool unit_h = false) {
  const double scale = unit_h ? 1.0 : double(n);
  std::vector<double> k;
  for (int i = 0; i <= p; ++i) k.push_back(0.0);
  size_t r = 0;
  for (int i = 1; i < n; ++i) {
    int copies = 1;
    while (r < reps.size() && reps[r].first < i) ++r;
    if (r < reps.size() && reps[r].first == i) copies += reps[r].second;
    for (int c = 0; c < copies; ++c) k.push_back(double(i) / scale);
  }
  for (int i = 0; i <= p; ++i) k.push_back(double(n) / scale);
  return k;
}

// Span of element e: the last index s with xi_s = e/n, so that xi_s <= x <
// xi_{s+1} on the element and B_{p,s-p..s} are the B-splines nonzero there
// (s = p + e without repeated knots).
int element_span(const std::vector<double>& kn, int n, int e) {
  const double z = double(e) / n;
  return int(std::upper_bound(kn.begin(), kn.end(), z) - kn.begin()) - 1;
}

// Values (order 0) or derivatives (order r) of B_{p,s-p..s} at x on the
// element of span s. Cox-de Boor for degree p-r, then r steps of the
// derivative recursion; terms with a vanishing knot difference are dropped.
void bspline_local(const std::vector<double>& kn, int p, int s, double x, int r, double* out) {
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

// Banded M and K of S_{p,h,D} on the knot vector kn (B-spline 0 removed if
// dir0, the last one if dir1), with an optional weight w(x) under both
// integrals; (p+1)-point Gauss per element. B_i and B_j share an element only
// if |i - j| <= p, also with repeated knots, so the half bandwidth is p.
void assemble_bands(int n, int p, const std::vector<double>& kn, bool dir0, bool dir1, double (*w)(double),
                    std::vector<double>* Mb, std::vector<double>* Kb) {
  const int F = (int)kn.size() - p - 1, bw = 2 * p + 1;
  const int m = F - (dir0 ? 1 : 0) - (dir1 ? 1 : 0);
  const int s0 = dir0 ? 1 : 0;
  std::vector<double> gx, gw;
  gauss_legendre(p + 1, &gx, &gw);
  std::vector<double> Mf((size_t)F * bw, 0.0), Kf((size_t)F * bw, 0.0);
  std::vector<double> B(p + 1), dB(p + 1);
  for (int e = 0; e < n; ++e) {
    const double a = double(e) / n, b = double(e + 1) / n;
    const int sp = element_span(kn, n, e);
    for (int g = 0; g <= p; ++g) {
      const double x = 0.5 * (b - a) * gx[g] + 0.5 * (a + b);
      double wt = 0.5 * (b - a) * gw[g];
      if (w) wt *= w(x);
      bspline_local(kn, p, sp, x, 0, B.data());
      bspline_local(kn, p, sp, x, 1, dB.data());
      for (int s = 0; s <= p; ++s)
        for (int t = 0; t <= p; ++t) {
          const int i = sp - p + s, j = sp - p + t;
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

// A combination sum_t c_t N_{a_t} of uniform B-splines of degree p; N_a has
// the knots a, a+1, .., a+p+1 (units of h). The cardinal B-spline B~_k of
// eq. "Btilde" is N_{k - floor(p/2) - 1}.
using Combo = std::vector<std::pair<double, int>>;
using SparseCol = std::vector<std::pair<int, double>>;  // (index, value), increasing index

// Edge functions of the special basis at the end x = 0 (Section 6, eq.
// "special_basis"), counted from the end: at a Dirichlet end B~_i - B~_{dp-i},
// i = 1..floor(p/2); at a natural end, p even, B~_i + B~_{1-i}, i = 1..p/2,
// and p odd, B~_0 and B~_i + B~_{-i}, i = 1..(p-1)/2. The functions at x = 1
// are their mirror images.
std::vector<Combo> edge_combos(int p, bool dir) {
  const int half = p / 2;
  const int dp = (p % 2 == 1) ? 0 : 1;
  std::vector<std::vector<std::pair<double, int>>> card;
  if (dir) {
    for (int i = 1; i <= half; ++i) card.push_back({{1.0, i}, {-1.0, dp - i}});
  } else if (p % 2 == 0) {
    for (int i = 1; i <= half; ++i) card.push_back({{1.0, i}, {1.0, 1 - i}});
  } else {
    card.push_back({{1.0, 0}});
    for (int i = 1; i <= (p - 1) / 2; ++i) card.push_back({{1.0, i}, {1.0, -i}});
  }
  std::vector<Combo> out;
  for (auto& c : card) {
    Combo cb;
    for (auto& t : c) cb.push_back({t.first, t.second - half - 1});
    out.push_back(cb);
  }
  return out;
}

// Coefficients of the restriction to [0, 1] of the combination cb in the
// open-knot basis whose knot vector, in units of h, is G (repeated interior
// breakpoints `reps`). Exact up to rounding by Boehm insertion: inserting the
// breakpoints 0 and n p times each and every repeated breakpoint k e_k times
// into the uniform knots turns cb into a combination of B-splines that are,
// inside [0, n], those of G (outside they vanish on [0, n]). Breakpoints
// outside the support change no coefficient; the ones in it, its ends
// included, are inserted so that the multiplicities match those of G. The
// uniform knots are padded by p + 2 on each side so that every insertion
// stays inside them. Returns (full B-spline index, coefficient), entries below
// 1e-13 of the largest dropped.
std::string restrict_combo(int n, int p, const Combo& cb, const std::vector<double>& G,
                           const std::vector<std::pair<int, int>>& reps, SparseCol* col) {
  int lo = cb[0].second, hi = cb[0].second + p + 1;
  for (const auto& t : cb) {
    lo = std::min(lo, t.second);
    hi = std::max(hi, t.second + p + 1);
  }
  const int J0 = lo - p - 2, J1 = hi + p + 2;
  std::vector<double> knots;
  for (int j = J0; j <= J1; ++j) knots.push_back(double(j));
  std::vector<double> coef(knots.size() - p - 1, 0.0);
  for (const auto& t : cb) coef[t.second - J0] += t.first;
  auto ins = [&](int t, int times) {
    if (t < lo || t > hi) return;
    for (int r = 0; r < times; ++r) insert_knot(&knots, &coef, p, double(t));
  };
  ins(0, p);
  ins(n, p);
  for (const auto& r : reps) ins(r.first, r.second);
  double cmax = 0.0;
  for (double c : coef) cmax = std::max(cmax, std::fabs(c));
  col->clear();
  for (int w = 0; w < (int)coef.size(); ++w) {
    if (!(std::fabs(coef[w]) > 1e-13 * cmax)) continue;
    const double a = knots[w], b = knots[w + p + 1];
    if (b <= 0.0 || a >= double(n)) continue;  // vanishes on [0, n]
    if (a < 0.0 || b > double(n)) return "special function does not restrict to the open-knot basis";
    const int w0 = int(std::lower_bound(knots.begin(), knots.end(), a) - knots.begin());
    const int j = int(std::lower_bound(G.begin(), G.end(), a) - G.begin()) + (w - w0);
    if (j + p + 1 >= (int)G.size()) return "special function outside the open-knot basis";
    for (int q = 0; q <= p + 1; ++q)
      if (G[j + q] != knots[w + q]) return "special function: knot sequences do not match";
    col->push_back({j, coef[w]});
  }
  return "";
}

// Derivative of order ord at x of the B-splines of the element of span sp, as a
// row over the reduced basis (full index - s0; removed functions skipped),
// scaled by sign and added to row.
void add_functional(const std::vector<double>& kn, int p, int sp, double x, int ord, int s0, int m, double sign,
                    std::vector<double>* row) {
  std::vector<double> d(p + 1);
  bspline_local(kn, p, sp, x, ord, d.data());
  for (int t = 0; t <= p; ++t) {
    const int r = sp - p + t - s0;
    if (r >= 0 && r < m) (*row)[r] += sign * d[t];
  }
}

// The transform passes apply V_reg through the compressed form of Axis1D:
// gather (y_j = sum_i V_reg[i][j] r_i, one output per column) and scatter
// (x_i = sum_j V_reg[i][j] w_j, one output per row). These two functions
// restate the kernels' column and row rules on the host.
void device_col(const Axis1D& A, int j, SparseCol* out) {
  out->clear();
  if (j < A.nL) {
    for (int r = 0; r < A.rowsL; ++r) out->push_back({r, A.VL[(size_t)r * A.nL + j]});
    return;
  }
  if (j >= A.n_reg - A.nR) {
    const int c = A.n_reg - 1 - j;
    for (int r = A.rowsR - 1; r >= 0; --r) out->push_back({A.m - 1 - r, A.VR[(size_t)r * A.nR + c]});
    return;
  }
  int o = A.o;
  for (size_t b = 0; b < A.blk.size(); b += 6) {
    const int c0 = A.blk[b], c1 = A.blk[b + 1], r0 = A.blk[b + 2], r1 = A.blk[b + 3], vo = A.blk[b + 5];
    if (j < c0) break;
    if (j < c1) {
      for (int r = r0; r < r1; ++r) out->push_back({r, A.VB[(size_t)vo + (size_t)(r - r0) * (c1 - c0) + (j - c0)]});
      return;
    }
    o = A.blk[b + 4];
  }
  out->push_back({j + o, 1.0});
}

void device_row(const Axis1D& A, int i, SparseCol* out) {
  out->clear();
  if (i < A.rowsL) {
    for (int c = 0; c < A.nL; ++c) out->push_back({c, A.VL[(size_t)i * A.nL + c]});
    return;
  }
  if (i >= A.m - A.rowsR) {
    const int r = A.m - 1 - i;
    for (int c = A.nR - 1; c >= 0; --c) out->push_back({A.n_reg - 1 - c, A.VR[(size_t)r * A.nR + c]});
    return;
  }
  int o = A.o;
  for (size_t b = 0; b < A.blk.size(); b += 6) {
    const int c0 = A.blk[b], c1 = A.blk[b + 1], r0 = A.blk[b + 2], r1 = A.blk[b + 3], vo = A.blk[b + 5];
    if (i < r0) break;
    if (i < r1) {
      for (int c = c0; c < c1; ++c) out->push_back({c, A.VB[(size_t)vo + (size_t)(i - r0) * (c1 - c0) + (c - c0)]});
      return;
    }
    o = A.blk[b + 4];
  }
  out->push_back({i - o, 1.0});
}

// Two sparse vectors agree to 1e-13 (entries missing in one count as 0).
bool same_sparse(const SparseCol& a, const SparseCol& b) {
  size_t x = 0, y = 0;
  while (x < a.size() || y < b.size()) {
    double d;
    if (y >= b.size() || (x < a.size() && a[x].first < b[y].first)) d = a[x++].second;
    else if (x >= a.size() || b[y].first < a[x].first) d = b[y++].second;
    else d = a[x++].second - b[y++].second;
    if (!(std::fabs(d) <= 1e-13)) return false;
  }
  return true;
}

}  // namespace

std::string build_axis(int n, int p, bool dir0, bool dir1, Axis1D* A,
                       const std::vector<std::pair<int, int>>& reps_in) {
  std::ostringstream err;
  if (p < 1 || p > 16) { err << "degree p=" << p << " outside 1..16"; return err.str(); }
  if (n <= p) { err << "n=" << n << " must exceed p=" << p; return err.str(); }
  std::vector<std::pair<int, int>> reps(reps_in);
  std::sort(reps.begin(), reps.end());
  int extra = 0;
  for (size_t r = 0; r < reps.size(); ++r) {
    if (reps[r].first < 1 || reps[r].first > n - 1) { err << "repeated knot " << reps[r].first << " outside 1..n-1"; return err.str(); }
    if (reps[r].second < 1 || reps[r].second > p - 1) {
      err << "extra multiplicity " << reps[r].second << " outside 1..p-1"; return err.str();
    }
    if (r > 0 && reps[r].first == reps[r - 1].first) { err << "knot " << reps[r].first << " repeated twice"; return err.str(); }
    extra += reps[r].second;
  }
  A->n = n;
  A->p = p;
  A->dir0 = dir0;
  A->dir1 = dir1;
  A->reps = reps;
  A->m = n + p + extra - (dir0 ? 1 : 0) - (dir1 ? 1 : 0);
  const int m = A->m;
  const int s0 = dir0 ? 1 : 0;

  // ---- banded M, K of S_{p,h,D}
  const std::vector<double> kn = open_knots(n, p, reps);
  assemble_bands(n, p, kn, dir0, dir1, nullptr, &A->Mband, &A->Kband);

  // ---- special basis (Section 6) in the open-knot basis. With repeated knots
  // the regular space is the same (Remark "reduced_regularity"); only the
  // coordinates of its functions change. Column j of V_reg: the left edge
  // functions, the interior cardinal B-splines N_0 .. N_{n-p-1}, and the right
  // edge functions (mirror images: computed at x = 0 on the mirrored knots).
  const std::vector<double> kh = open_knots(n, p, reps, true);  // knots in units of h
  std::vector<std::pair<int, int>> mreps;
  for (auto it = reps.rbegin(); it != reps.rend(); ++it) mreps.push_back({n - it->first, it->second});
  const std::vector<double> khm = open_knots(n, p, mreps, true);
  const int F = (int)kh.size() - p - 1;
  const std::vector<Combo> left = edge_combos(p, dir0), right = edge_combos(p, dir1);
  A->nL = (int)left.size();
  A->nR = (int)right.size();
  const int n_int = n - p;
  A->n_reg = A->nL + n_int + A->nR;
  A->n_out = m - A->n_reg;
  const int nr = A->n_reg;
  std::vector<SparseCol> cols(nr);  // V_reg by columns, reduced row indices
  SparseCol full;
  for (int j = 0; j < nr; ++j) {
    const bool is_right = j >= nr - A->nR;
    std::string e;
    if (j < A->nL) e = restrict_combo(n, p, left[j], kh, reps, &full);
    else if (is_right) e = restrict_combo(n, p, right[nr - 1 - j], khm, mreps, &full);
    else e = restrict_combo(n, p, Combo{{1.0, j - A->nL}}, kh, reps, &full);
    if (!e.empty()) return e;
    for (const auto& t : full) {
      const int jf = is_right ? F - 1 - t.first : t.first;  // full index on kh
      if ((dir0 && jf == 0) || (dir1 && jf == F - 1)) return "special basis function does not vanish at a Dirichlet end";
      cols[j].push_back({jf - s0, t.second});
    }
    std::sort(cols[j].begin(), cols[j].end());
  }
  // compressed form used by the device passes: edge blocks, identity runs
  // (column j is the B-spline with reduced index j + offset) and dense blocks
  // over the runs of other interior columns (around repeated knots). A run
  // that touches an edge block (no identity column between them, or shared
  // rows) joins it; if the two edge blocks then overlap, the left block takes
  // all of V_reg (small n only).
  struct Run { int c0, c1, r0, r1; };
  std::vector<Run> runs;
  for (int j = A->nL; j < nr - A->nR; ++j) {
    if (cols[j].empty()) return "special basis function vanishes";
    const bool unit = cols[j].size() == 1 && cols[j][0].second == 1.0;
    if (unit) continue;
    if (runs.empty() || runs.back().c1 != j) runs.push_back({j, j + 1, cols[j].front().first, cols[j].back().first + 1});
    Run& r = runs.back();
    r.c1 = j + 1;
    r.r0 = std::min(r.r0, cols[j].front().first);
    r.r1 = std::max(r.r1, cols[j].back().first + 1);
  }
  A->rowsL = 0;
  for (int j = 0; j < A->nL; ++j)
    for (const auto& t : cols[j]) A->rowsL = std::max(A->rowsL, t.first + 1);
  A->rowsR = 0;
  for (int j = nr - A->nR; j < nr; ++j)
    for (const auto& t : cols[j]) A->rowsR = std::max(A->rowsR, m - t.first);
  size_t first = 0, last = runs.size();
  while (first < last && (runs[first].c0 == A->nL || runs[first].r0 < A->rowsL)) {
    A->nL = runs[first].c1;
    A->rowsL = std::max(A->rowsL, runs[first].r1);
    ++first;
  }
  while (last > first && (runs[last - 1].c1 == nr - A->nR || runs[last - 1].r1 > m - A->rowsR)) {
    A->nR = nr - runs[last - 1].c0;
    A->rowsR = std::max(A->rowsR, m - runs[last - 1].r0);
    --last;
  }
  if (A->rowsL > m - A->rowsR || A->nL > nr - A->nR) {
    A->nL = nr;
    A->rowsL = m;
    A->nR = 0;
    A->rowsR = 0;
    first = last = runs.size();
  }
  A->VL.assign((size_t)A->rowsL * A->nL, 0.0);
  for (int j = 0; j < A->nL; ++j)
    for (const auto& t : cols[j]) {
      if (t.first >= A->rowsL) return "unexpected structure of V_reg";
      A->VL[(size_t)t.first * A->nL + j] = t.second;
    }
  A->VR.assign((size_t)A->rowsR * A->nR, 0.0);
  for (int j = nr - A->nR; j < nr; ++j)
    for (const auto& t : cols[j]) {
      if (m - 1 - t.first >= A->rowsR) return "unexpected structure of V_reg";
      A->VR[(size_t)(m - 1 - t.first) * A->nR + (nr - 1 - j)] = t.second;
    }
  // identity offsets: o before the first block, then the offset after each block
  A->blk.clear();
  A->VB.clear();
  A->o = 0;
  bool have_o = false;
  int cur = 0;
  size_t next = first;
  for (int j = A->nL; j < nr - A->nR; ++j) {
    if (next < last && j == runs[next].c0) {
      const Run& r = runs[next];
      const int vo = (int)A->VB.size();
      A->VB.resize(A->VB.size() + (size_t)(r.r1 - r.r0) * (r.c1 - r.c0), 0.0);
      for (int c = r.c0; c < r.c1; ++c)
        for (const auto& t : cols[c]) A->VB[(size_t)vo + (size_t)(t.first - r.r0) * (r.c1 - r.c0) + (c - r.c0)] = t.second;
      // offset of the identity columns after the block (the block's own if none follow)
      int after = cur;
      if (r.c1 < nr - A->nR) after = cols[r.c1][0].first - r.c1;
      A->blk.insert(A->blk.end(), {r.c0, r.c1, r.r0, r.r1, after, vo});
      cur = after;
      have_o = true;
      j = r.c1 - 1;
      ++next;
      continue;
    }
    const int off = cols[j][0].first - j;
    if (!have_o) {
      A->o = cur = off;
      have_o = true;
    } else if (off != cur) {
      return "unexpected structure of V_reg";
    }
  }
  // the device rules must reproduce V_reg column by column and row by row
  std::vector<SparseCol> rows(m);
  for (int j = 0; j < nr; ++j)
    for (const auto& t : cols[j]) rows[t.first].push_back({j, t.second});
  SparseCol dv;
  for (int j = 0; j < nr; ++j) {
    device_col(*A, j, &dv);
    for (const auto& t : dv)
      if (t.first < 0 || t.first >= m) return "n too small for the device layout of the special basis";
    if (!same_sparse(dv, cols[j])) return "n too small for the device layout of the special basis";
  }
  for (int i = 0; i < m; ++i) {
    device_row(*A, i, &dv);
    for (const auto& t : dv)
      if (t.first < 0 || t.first >= nr) return "n too small for the device layout of the special basis";
    if (!same_sparse(dv, rows[i])) return "n too small for the device layout of the special basis";
  }

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
  A->wlo = A->wlo_f = 0;
  A->whi = A->whi_f = m;
  if (no > 0) {
    // rows of G over the reduced basis (eq. "reg_space"): derivatives of the
    // even orders 2, 4, .. (Dirichlet end) or the odd orders 1, 3, .. (natural
    // end) up to p - 1 at each end, and, at a breakpoint k repeated e times,
    // the jumps of the derivatives of orders p - e .. p - 1 (functions of
    // S^reg are C^{p-1} there). Each group is orthonormalised (modified
    // Gram-Schmidt; derivative values scale like h^-k).
    std::vector<std::vector<double>> G;
    auto orthonormalise_into = [&](std::vector<std::vector<double>> R) {
      for (size_t a = 0; a < R.size(); ++a) {
        for (size_t b = 0; b < a; ++b) {
          double dot = 0;
          for (int i = 0; i < m; ++i) dot += R[a][i] * R[b][i];
          for (int i = 0; i < m; ++i) R[a][i] -= dot * R[b][i];
        }
        double nr2 = 0;
        for (int i = 0; i < m; ++i) nr2 += R[a][i] * R[a][i];
        const double nrm = std::sqrt(nr2);
        for (int i = 0; i < m; ++i) R[a][i] /= nrm;
        G.push_back(R[a]);
      }
    };
    const int sp0 = element_span(kn, n, 0), sp1 = element_span(kn, n, n - 1);
    for (int end = 0; end < 2; ++end) {
      const bool dir = end == 0 ? dir0 : dir1;
      std::vector<std::vector<double>> R;
      for (int ord = dir ? 2 : 1; ord <= p - 1; ord += 2) {
        std::vector<double> row(m, 0.0);
        add_functional(kn, p, end == 0 ? sp0 : sp1, end == 0 ? 0.0 : 1.0, ord, s0, m, 1.0, &row);
        R.push_back(row);
      }
      orthonormalise_into(R);
    }
    for (const auto& rk : reps) {
      std::vector<std::vector<double>> R;
      const double x = double(rk.first) / n;
      for (int ord = p - rk.second; ord <= p - 1; ++ord) {
        std::vector<double> row(m, 0.0);
        add_functional(kn, p, element_span(kn, n, rk.first), x, ord, s0, m, 1.0, &row);
        add_functional(kn, p, element_span(kn, n, rk.first - 1), x, ord, s0, m, -1.0, &row);
        R.push_back(row);
      }
      orthonormalise_into(R);
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
    // support: the longest run of rows whose entries are all below tol max|W|
    // is skipped by the passes (W decays geometrically away from both ends and
    // from repeated knots); tol = 1e-17 for FP64 passes, 1e-10 for FP32 ones
    // (far below FP32 rounding: at most m 1e-10 of the result's scale)
    auto support = [&](double tol, int* wlo, int* whi) {
      auto small = [&](int i) {
        for (int k = 0; k < no; ++k)
          if (std::fabs(A->W[(size_t)i * no + k]) > tol * wmax) return false;
        return true;
      };
      int best_lo = m, best_len = 0;
      for (int i = 0; i < m;) {
        if (!small(i)) { ++i; continue; }
        int k = i;
        while (k < m && small(k)) ++k;
        if (k - i > best_len) { best_len = k - i; best_lo = i; }
        i = k;
      }
      *wlo = best_lo;
      *whi = best_lo + best_len;
    };
    support(1e-17, &A->wlo, &A->whi);
    support(1e-10, &A->wlo_f, &A->whi_f);
  }
  return "";
}

void expand_vreg(const Axis1D& A, double* V) {
  std::fill(V, V + (size_t)A.m * A.n_reg, 0.0);
  SparseCol c;
  for (int j = 0; j < A.n_reg; ++j) {
    device_col(A, j, &c);
    for (const auto& t : c) V[(size_t)t.first * A.n_reg + j] = t.second;
  }
}

void build_quad_axis(const Axis1D& A, QuadAxis* Q) {
  const int n = A.n, p = A.p, m = A.m, s0 = A.dir0 ? 1 : 0;
  const std::vector<double> kn = open_knots(n, p, A.reps);
  std::vector<double> gx, gw, B(p + 1), dB(p + 1);
  gauss_legendre(p + 1, &gx, &gw);
  std::vector<int> ord(p + 1);  // nodes in increasing order
  for (int g = 0; g <= p; ++g) ord[g] = g;
  std::sort(ord.begin(), ord.end(), [&](int i, int j) { return gx[i] < gx[j]; });
  Q->nq = n * (p + 1);
  Q->m = m;
  Q->x.clear(); Q->w.clear(); Q->col.clear(); Q->bv.clear(); Q->dv.clear();
  Q->rp.assign(1, 0);
  for (int e = 0; e < n; ++e) {
    const double a = double(e) / n, b = double(e + 1) / n;
    const int sp = element_span(kn, n, e);
    for (int gi = 0; gi <= p; ++gi) {
      const int g = ord[gi];
      const double x = 0.5 * (b - a) * gx[g] + 0.5 * (a + b);
      Q->x.push_back(x);
      Q->w.push_back(0.5 * (b - a) * gw[g]);
      bspline_local(kn, p, sp, x, 0, B.data());
      bspline_local(kn, p, sp, x, 1, dB.data());
      for (int t = 0; t <= p; ++t) {
        const int j = sp - p + t - s0;  // index among the kept functions
        if (j < 0 || j >= m) continue;
        Q->col.push_back(j);
        Q->bv.push_back(B[t]);
        Q->dv.push_back(dB[t]);
      }
      Q->rp.push_back((int)Q->col.size());
    }
  }
  // transpose (counting sort by column; points stay increasing within a row)
  Q->trp.assign(m + 1, 0);
  for (int c : Q->col) ++Q->trp[c + 1];
  for (int j = 0; j < m; ++j) Q->trp[j + 1] += Q->trp[j];
  Q->tcol.assign(Q->col.size(), 0);
  Q->tbv.assign(Q->col.size(), 0.0);
  Q->tdv.assign(Q->col.size(), 0.0);
  std::vector<int> next(Q->trp.begin(), Q->trp.end() - 1);
  for (int q = 0; q < Q->nq; ++q)
    for (int k = Q->rp[q]; k < Q->rp[q + 1]; ++k) {
      const int t = next[Q->col[k]]++;
      Q->tcol[t] = q;
      Q->tbv[t] = Q->bv[k];
      Q->tdv[t] = Q->dv[k];
    }
}

void build_weighted_bands(Axis1D* A) {
  assemble_bands(A->n, A->p, open_knots(A->n, A->p, A->reps), A->dir0, A->dir1, sin_2pi, &A->Msband, &A->Ksband);
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
