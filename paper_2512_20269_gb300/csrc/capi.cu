// C ABI of the IFFD library (declarations and contracts in include/iffd.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/iffd.h"
#include "device_common.cuh"
#include "fd.h"
#include "host_setup.h"
#include "kernels.h"
#include "plan.h"
#include "precond_warp_geom.h"

namespace iffd {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(IFFD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static const double kPi = 3.14159265358979323846264338327950288;

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ------------------------------------------------------------------ tables
struct TableBuilder {
  std::vector<char> bytes;
  size_t add(const void* src, size_t n) {
    const size_t off = align256(bytes.size());
    bytes.resize(off + n);
    std::memcpy(bytes.data() + off, src, n);
    return off;
  }
  template <typename T>
  size_t add_vec(const std::vector<T>& v) {
    if (v.empty()) {  // keep a valid (zero) entry so the device pointer is never dangling
      T zero;
      std::memset(&zero, 0, sizeof(T));
      return add(&zero, sizeof(T));
    }
    return add(v.data(), v.size() * sizeof(T));
  }
};

template <typename T>
static std::vector<T> cast_vec(const std::vector<double>& v) {
  return std::vector<T>(v.begin(), v.end());
}

struct AxisOffsets {
  size_t VL, VR, W, lam, post, chirp, bhat, VB, blk;
};

// double-float copies of FP64 tables (hi = nearest float, lo = the rounded rest)
static std::vector<df> df_vec(const std::vector<double>& v) {
  std::vector<df> o;
  o.reserve(v.size());
  for (double x : v) o.push_back(df(x));
  return o;
}

static bool register_radix(int r) { return r == 8 || r == 4 || r == 2 || r == 3 || r == 5; }

// Stages and twiddles of one Stockham FFT of length len with the radix
// sequence rad. Register-butterfly stages store exp(-2 pi i q k / (Ns r)) for
// q = 1..r-1, k < Ns; direct-DFT stages store exp(-2 pi i s / (Ns r)), s < Ns r.
struct FftPlan {
  int len = 0;
  std::vector<int> rad, twoff;
  std::vector<double> tw;
};

static std::string fft_plan(int len, const std::vector<int>& rad, FftPlan* f) {
  f->len = len;
  f->rad = rad;
  if ((int)f->rad.size() > kMaxStages) return "too many FFT stages";
  f->tw.clear();
  f->twoff.clear();
  long long Ns = 1;
  for (int r : f->rad) {
    f->twoff.push_back((int)(f->tw.size() / 2));
    const long long den = Ns * r;
    auto push = [&](long long num) {
      const double ang = -2.0 * kPi * (double)(num % den) / (double)den;
      f->tw.push_back(std::cos(ang));
      f->tw.push_back(std::sin(ang));
    };
    if (register_radix(r)) {
      for (int q = 1; q < r; ++q)
        for (long long k = 0; k < Ns; ++k) push((long long)q * k);
    } else {
      for (long long s = 0; s < den; ++s) push(s);
    }
    Ns *= r;
  }
  return "";
}

// Radix sequences offered to the tuner for one FFT length: the greedy
// radix-8 sequence (the default: 8s, then 4 or 2, then odd factors
// ascending), the radix-4 sequence, and the greedy sequence reversed (small
// radices first). Duplicates are dropped; the first entry is the default.
std::vector<std::vector<int>> radix_variants(int len) {
  std::vector<int> greedy;
  fft_factor(len, &greedy);
  int e2 = 0, x = len;
  while (x % 2 == 0) { x /= 2; ++e2; }
  std::vector<int> odd(greedy.begin(), greedy.end());
  odd.erase(std::remove_if(odd.begin(), odd.end(), [](int r) { return r % 2 == 0; }), odd.end());
  std::vector<int> four;
  for (int k = 0; k < e2 / 2; ++k) four.push_back(4);
  if (e2 % 2) four.push_back(2);
  four.insert(four.end(), odd.begin(), odd.end());
  std::vector<int> rev(greedy.rbegin(), greedy.rend());
  std::vector<std::vector<int>> out{greedy};
  for (const auto& v : {four, rev})
    if (std::find(out.begin(), out.end(), v) == out.end()) out.push_back(v);
  return out;
}

// Estimated real flops per element of one FFT stage of radix r: (r-1) twiddle
// products and the r-point DFT of a register butterfly, or r - 1 complex
// multiply-adds per output of a direct stage.
static double stage_cost(int r) {
  switch (r) {
    case 2: return 5.0;
    case 3: return 8.0;
    case 4: return 8.5;
    case 5: return 11.6;
    case 8: return 11.75;
    default: return 8.0 * (r - 1) + 2.0;
  }
}

static double fft_cost(int len) {
  std::vector<int> rad;
  fft_factor(len, &rad);
  double c = 0.0;
  for (int r : rad) c += stage_cost(r);
  return c * len;
}

static bool smooth5(int x) {
  for (int r : {2, 3, 5})
    while (x % r == 0) x /= r;
  return x == 1;
}

// Bluestein length for a length-L DFT: the cheapest 5-smooth F in [2L-1, 4L],
// taken when two length-F FFTs and the chirp products cost less than 0.7 of
// the direct mixed-radix FFT of length L (whose large prime factors run as
// direct DFT stages). Returns 0 when the direct FFT is kept.
static int bluestein_length(int L) {
  if (L < 16) return 0;
  int best = 0;
  double best_cost = 0.0;
  for (int f = 2 * L - 1; f <= 4 * L; ++f) {
    if (!smooth5(f)) continue;
    const double c = 2.0 * fft_cost(f) + 7.0 * f + 12.0 * L;
    if (best == 0 || c < best_cost) { best = f; best_cost = c; }
  }
  return (best != 0 && best_cost < 0.7 * fft_cost(L)) ? best : 0;
}

// Forward DFT of a 5-smooth length in double precision (host; Bluestein
// kernel spectrum only), recursive decimation in time with twiddles
// exp(-2 pi i e / n) from exactly reduced integer angles.
static void host_dft(std::vector<double>& re, std::vector<double>& im) {
  const int n = (int)re.size();
  std::vector<double> c(n), sn(n);
  for (int e = 0; e < n; ++e) {
    const double ang = -2.0 * kPi * (double)e / (double)n;
    c[e] = std::cos(ang);
    sn[e] = std::sin(ang);
  }
  // rec(len, stride, off): DFT of x[off + j * stride], j < len, into out
  std::vector<double> ore(n), oim(n);
  struct Rec {
    const std::vector<double>& c;
    const std::vector<double>& sn;
    int n;
    void run(const double* xr, const double* xi, int len, int stride, double* yr, double* yi) const {
      if (len == 1) { yr[0] = xr[0]; yi[0] = xi[0]; return; }
      int r = 2;
      while (len % r) ++r;
      const int l2 = len / r;
      std::vector<double> tr(len), ti(len);
      for (int q = 0; q < r; ++q) run(xr + (size_t)q * stride, xi + (size_t)q * stride, l2, stride * r,
                                      tr.data() + (size_t)q * l2, ti.data() + (size_t)q * l2);
      const int step = n / len;  // exp(-2 pi i e / len) = table[e * step]
      for (int t = 0; t < r; ++t)
        for (int k = 0; k < l2; ++k) {
          const int kk = k + t * l2;
          double ar = 0.0, ai = 0.0;
          for (int q = 0; q < r; ++q) {
            const long long e = ((long long)q * kk) % len;
            const double wr = c[(size_t)(e * step)], wi = sn[(size_t)(e * step)];
            const double vr = tr[(size_t)q * l2 + k], vi = ti[(size_t)q * l2 + k];
            ar += vr * wr - vi * wi;
            ai += vr * wi + vi * wr;
          }
          yr[kk] = ar;
          yi[kk] = ai;
        }
    }
  } rec{c, sn, n};
  rec.run(re.data(), im.data(), n, 1, ore.data(), oim.data());
  re.swap(ore);
  im.swap(oim);
}

// Chirp c_j = exp(i pi j^2 / L) (j < L) and bhat = DFT_F(b) / F for the
// Bluestein kernel b_t = c_t (t < L), b_{F-t} = c_t (0 < t < L), 0 otherwise.
static void bluestein_tables(int L, int F, std::vector<double>* chirp, std::vector<double>* bhat) {
  chirp->assign(2 * (size_t)L, 0.0);
  std::vector<double> br(F, 0.0), bi(F, 0.0);
  for (int j = 0; j < L; ++j) {
    const long long e = ((long long)j * j) % (2LL * L);  // exact reduction of j^2 mod 2L
    const double ang = kPi * (double)e / (double)L;
    (*chirp)[2 * j] = std::cos(ang);
    (*chirp)[2 * j + 1] = std::sin(ang);
    br[j] = std::cos(ang);
    bi[j] = std::sin(ang);
    if (j > 0) {
      br[F - j] = br[j];
      bi[F - j] = bi[j];
    }
  }
  host_dft(br, bi);
  bhat->resize(2 * (size_t)F);
  for (int k = 0; k < F; ++k) {
    (*bhat)[2 * k] = br[k] / F;
    (*bhat)[2 * k + 1] = bi[k] / F;
  }
}

static std::vector<double> post_table(const Axis1D& A) {
  std::vector<double> post;
  const int N = A.n_reg;
  if (A.kind == TK_DST23) {
    for (int k = 0; k <= N / 2; ++k) {
      const double sk = 1.0 / A.dtilde[N - 1 - k];
      const double sm = (k >= 1) ? 1.0 / A.dtilde[k - 1] : 0.0;
      const double c = std::cos(kPi * k / (2.0 * N)), s = std::sin(kPi * k / (2.0 * N));
      post.push_back(0.5 * sk * c);
      post.push_back(0.5 * sk * s);
      post.push_back(0.5 * sm * s);
      post.push_back(0.5 * sm * c);
    }
  } else {
    for (int j = 0; j < N; ++j) post.push_back(0.5 / A.dtilde[j]);
  }
  return post;
}

// Fills one precision's tables. With F > L the length-L DFT runs as Bluestein
// over a length-F FFT; the FFT stages are set by set_fft.
template <typename T>
static void fill_axistab(AxisTab<T>* t, const Axis1D& A, int L, int F, const char* base, const AxisOffsets& o) {
  t->m = A.m;
  t->n_reg = A.n_reg;
  t->n_out = A.n_out;
  t->p = A.p;
  t->o = A.o;
  t->nL = A.nL;
  t->rowsL = A.rowsL;
  t->nR = A.nR;
  t->rowsR = A.rowsR;
  t->gq = A.gq;
  t->gqc = A.gqc;
  t->gqe = A.gqe;
  t->wlo = std::is_same<T, float>::value ? A.wlo_f : A.wlo;
  t->whi = std::is_same<T, float>::value ? A.whi_f : A.whi;
  t->kind = A.kind;
  t->L = L;
  t->F = F;
  t->blu = (F > L) ? 1 : 0;
  t->VL = reinterpret_cast<const T*>(base + o.VL);
  t->VR = reinterpret_cast<const T*>(base + o.VR);
  t->nblk = (int)(A.blk.size() / 6);
  t->blk = reinterpret_cast<const int*>(base + o.blk);
  t->VB = reinterpret_cast<const T*>(base + o.VB);
  t->W = reinterpret_cast<const T*>(base + o.W);
  t->lam = reinterpret_cast<const T*>(base + o.lam);
  t->post = reinterpret_cast<const T*>(base + o.post);
  t->chirp = reinterpret_cast<const T*>(base + o.chirp);
  t->bhat = reinterpret_cast<const T*>(base + o.bhat);
  t->rden = nullptr;
  t->fm = make_fastdiv(A.m);
  t->fL = make_fastdiv(L);
  t->fF = make_fastdiv(F);
  t->fN = make_fastdiv(A.n_reg);
  t->fK = make_fastdiv(A.n_reg / 2 + 1);
  t->fnout = make_fastdiv(A.n_out);
}

template <typename T>
static const T* var_tw(const FftVar& v);
template <>
const double* var_tw<double>(const FftVar& v) { return v.twd; }
template <>
const float* var_tw<float>(const FftVar& v) { return v.twf; }
template <>
const df* var_tw<df>(const FftVar& v) { return v.twq; }

// Selects the radix sequence v (whose length must equal t->F).
template <typename T>
void set_fft(AxisTab<T>* t, const FftVar& v) {
  t->nst = v.nst;
  int Ns = 1;
  for (int s = 0; s < kMaxStages; ++s) {
    t->radix[s] = s < v.nst ? v.radix[s] : 1;
    t->twoff[s] = s < v.nst ? v.twoff[s] : 0;
    t->fnb[s] = make_fastdiv(v.len / t->radix[s]);
    t->fNs[s] = make_fastdiv(Ns);
    if (s < v.nst) Ns *= v.radix[s];
  }
  t->tw = var_tw<T>(v);
}
template void set_fft<double>(AxisTab<double>*, const FftVar&);
template void set_fft<float>(AxisTab<float>*, const FftVar&);
template void set_fft<df>(AxisTab<df>*, const FftVar&);

// Index of the default (first) radix sequence of length len in fvar.
static int default_var(const std::vector<FftVar>& fv, int len) {
  for (size_t i = 0; i < fv.size(); ++i)
    if (fv[i].len == len) return (int)i;
  return -1;
}

// Default pencils per tile of a transform pass whose FFT has length F: 8,
// halved while the tile needs more than 110 KB of shared memory
// (iffd_autotune may pick others).
static int pick_pp(int m, int F, size_t elt, int* PP, int* ldt) {
  *ldt = m | 1;
  int pp = 8;
  while (pp > 2 && precond_smem_bytes(pp, *ldt, F, elt) > 110 * 1024) pp /= 2;
  if (precond_smem_bytes(pp, *ldt, F, elt) > 220 * 1024) return 0;
  *PP = pp;
  return 1;
}

// Length of the complex DFT that carries one direction's transform (two
// pencils per sequence): n_reg (DST-II/III, Makhoul order), 2 (n_reg + 1)
// (DST-I, odd extension), 2 n q (generic Table 1 case, zero padding).
static int dft_length(const Axis1D& A) {
  if (A.kind == TK_DST23) return A.n_reg;
  if (A.kind == TK_DST1) return 2 * (A.n_reg + 1);
  return 2 * A.n * A.gq;
}

// Transform of one direction for one precision (element size elt): the DFT
// length L, the FFT length F actually run (F > L: Bluestein) and the tile.
// Bluestein is used when bluestein_length() picks it and its two length-F
// buffers fit in shared memory; otherwise the direct length-L FFT. Returns 0
// if neither fits.
static int choose_transform(const Axis1D& A, size_t elt, int* L, int* F, int* PP, int* ldt) {
  *L = dft_length(A);
  const int fb = bluestein_length(*L);
  if (fb > 0 && pick_pp(A.m, fb, elt, PP, ldt)) {
    *F = fb;
    return 1;
  }
  *F = *L;
  return pick_pp(A.m, *L, elt, PP, ldt);
}

static int build_plan(Plan* P, cudaStream_t stream) {
  TableBuilder tb;
  struct PerAxis {
    AxisOffsets od, of, oq;  // FP64, FP32 and double-float tables
    size_t Mb, Kb, Mt, Kt, QT, Q, lamQ, Msb, Ksb;
    int L, F;                          // DFT length; Bluestein FFT length (0: direct)
    std::vector<FftPlan> vars;         // radix sequences of length L (and F)
    std::vector<size_t> var_d, var_f, var_q;  // their twiddle tables (FP64, FP32, double-float)
    int ilo, ihi;
    size_t wt, wt_d, wt_q;             // warp-FFT twiddles, FP32, FP64 and df (D = {0,1} directions)
  } pa[3];
  for (int a = 0; a < P->d; ++a) {
    const Axis1D& A = P->host[a];
    // the DST of the regular part is carried by a complex DFT of length L
    // (two pencils per sequence; Makhoul order for DST-II/III, odd extension
    // for DST-I); lengths with large prime factors may run as Bluestein
    pa[a].L = dft_length(A);
    pa[a].F = bluestein_length(pa[a].L);
    std::vector<double> chirp, bhat;
    if (pa[a].F > 0) bluestein_tables(pa[a].L, pa[a].F, &chirp, &bhat);
    std::string err;
    for (int len : {pa[a].L, pa[a].F}) {
      if (len <= 0) continue;
      for (const auto& rad : radix_variants(len)) {
        FftPlan fp;
        err = fft_plan(len, rad, &fp);
        if (!err.empty()) return fail(IFFD_ERR_UNSUPPORTED, err);
        pa[a].var_d.push_back(tb.add_vec(fp.tw));
        pa[a].var_f.push_back(tb.add_vec(cast_vec<float>(fp.tw)));
        pa[a].var_q.push_back(tb.add_vec(df_vec(fp.tw)));
        pa[a].vars.push_back(std::move(fp));
      }
    }
    const std::vector<double> post = (A.kind == TK_GEN) ? A.gpost : post_table(A);
    pa[a].od.VL = tb.add_vec(A.VL);
    pa[a].od.VR = tb.add_vec(A.VR);
    pa[a].od.W = tb.add_vec(A.W);
    pa[a].od.lam = tb.add_vec(A.lam);
    pa[a].od.post = tb.add_vec(post);
    pa[a].od.chirp = tb.add_vec(chirp);
    pa[a].od.bhat = tb.add_vec(bhat);
    pa[a].od.VB = tb.add_vec(A.VB);
    pa[a].od.blk = tb.add_vec(A.blk);
    pa[a].of.blk = pa[a].od.blk;
    pa[a].of.VB = tb.add_vec(cast_vec<float>(A.VB));
    {
      // exp(-2 pi i e / N), e < N, for the warp-FFT pass of FFT length N
      // (n_reg for DST-II/III, 2 (n_reg + 1) for DST-I)
      std::vector<double> wt;
      const int Nw = (A.kind == TK_DST23) ? A.n_reg : (A.kind == TK_DST1 ? 2 * (A.n_reg + 1) : 0);
      if (Nw == 64 || Nw == 128 || Nw == 256 || Nw == 512)
        for (int e = 0; e < Nw; ++e) {
          const double ang = -2.0 * kPi * e / Nw;
          wt.push_back(std::cos(ang));
          wt.push_back(std::sin(ang));
        }
      pa[a].wt = tb.add_vec(cast_vec<float>(wt));
      pa[a].wt_d = tb.add_vec(wt);
      std::vector<df2> wq;
      for (size_t e = 0; e + 1 < wt.size(); e += 2) wq.push_back(df2{df(wt[e]), df(wt[e + 1])});
      pa[a].wt_q = tb.add_vec(wq);
    }
    pa[a].oq.VL = tb.add_vec(df_vec(A.VL));
    pa[a].oq.VR = tb.add_vec(df_vec(A.VR));
    pa[a].oq.W = tb.add_vec(df_vec(A.W));
    pa[a].oq.lam = tb.add_vec(df_vec(A.lam));
    pa[a].oq.post = tb.add_vec(df_vec(post));
    pa[a].oq.VB = tb.add_vec(df_vec(A.VB));
    pa[a].oq.blk = pa[a].od.blk;
    pa[a].oq.chirp = pa[a].oq.bhat = tb.add_vec(std::vector<df>{});  // the warp pass runs no Bluestein
    pa[a].of.VL = tb.add_vec(cast_vec<float>(A.VL));
    pa[a].of.VR = tb.add_vec(cast_vec<float>(A.VR));
    pa[a].of.W = tb.add_vec(cast_vec<float>(A.W));
    pa[a].of.lam = tb.add_vec(cast_vec<float>(A.lam));
    pa[a].of.post = tb.add_vec(cast_vec<float>(post));
    pa[a].of.chirp = tb.add_vec(cast_vec<float>(chirp));
    pa[a].of.bhat = tb.add_vec(cast_vec<float>(bhat));
    // stiffness band tables; interior rows are symmetric Toeplitz
    const int p = A.p, m = A.m, bw = 2 * p + 1;
    pa[a].Mb = tb.add_vec(A.Mband);
    pa[a].Kb = tb.add_vec(A.Kband);
    std::vector<double> mt(p + 1, 0.0), kt(p + 1, 0.0);
    // rows coupled to a B-spline with repeated end knots are general band rows:
    // the first 2p-1 rows at a Dirichlet end (its end B-spline is removed), 2p
    // rows at a natural end
    // (with repeated knots every row is a general band row)
    int ilo = 2 * p - (A.dir0 ? 1 : 0), ihi = m - 2 * p + (A.dir1 ? 1 : 0);
    if (ihi <= ilo || !A.reps.empty()) { ilo = 0; ihi = 0; }
    else {
      const int mid = (ilo + ihi) / 2;
      for (int k = 0; k <= p; ++k) {
        mt[k] = A.Mband[(size_t)mid * bw + p + k];
        kt[k] = A.Kband[(size_t)mid * bw + p + k];
      }
      for (int i = ilo; i < ihi; ++i)
        for (int k = -p; k <= p; ++k) {
          const double dm = A.Mband[(size_t)i * bw + p + k] - mt[std::abs(k)];
          const double dk = A.Kband[(size_t)i * bw + p + k] - kt[std::abs(k)];
          if (std::fabs(dm) > 1e-12 * std::fabs(mt[0]) || std::fabs(dk) > 1e-12 * std::fabs(kt[0]))
            return fail(IFFD_ERR_UNSUPPORTED, "interior rows of M/K are not Toeplitz");
        }
    }
    pa[a].ilo = ilo;
    pa[a].ihi = ihi;
    pa[a].Mt = tb.add_vec(mt);
    pa[a].Kt = tb.add_vec(kt);
    if (P->opt.coef == IFFD_COEF_SEPARABLE_SIN) {
      pa[a].Msb = tb.add_vec(A.Msband);
      pa[a].Ksb = tb.add_vec(A.Ksband);
    }
    if (P->opt.precond == IFFD_PRECOND_EXACT_FD) {
      std::vector<double> Qc, lq;
      err = exact_fd_axis(A, &Qc, &lq);
      if (!err.empty()) return fail(IFFD_ERR_UNSUPPORTED, err);
      std::vector<double> Qr((size_t)m * m), QTr((size_t)m * m);
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
          Qr[(size_t)i * m + j] = Qc[i + (size_t)j * m];   // Q[i][j]
          QTr[(size_t)i * m + j] = Qc[j + (size_t)i * m];  // Q^T[i][j] = Q[j][i]
        }
      pa[a].Q = tb.add_vec(Qr);
      pa[a].QT = tb.add_vec(QTr);
      pa[a].lamQ = tb.add_vec(lq);
      if (fd_smem(m) > 227 * 1024) return fail(IFFD_ERR_UNSUPPORTED, "exact FD comparator: m too large");
    }
  }
  IFFD_CUDA(cudaMalloc(&P->dev, align256(tb.bytes.size()) + 256));
  IFFD_CUDA(cudaMemcpyAsync(P->dev, tb.bytes.data(), tb.bytes.size(), cudaMemcpyHostToDevice, stream));
  IFFD_CUDA(cudaStreamSynchronize(stream));
  const char* base = static_cast<const char*>(P->dev);
  long long N = 1;
  for (int a = 0; a < P->d; ++a) N *= P->host[a].m;
  P->dims.d = P->d;
  for (int a = 0; a < 3; ++a) P->dims.m[a] = (a < P->d) ? P->host[a].m : 1;
  P->dims.N = N;
  int max_parts = vec_grid(N);
  for (int a = 0; a < P->d; ++a) {
    const Axis1D& A = P->host[a];
    // FFT variants with device twiddle pointers
    P->fvar[a].clear();
    for (size_t k = 0; k < pa[a].vars.size(); ++k) {
      const FftPlan& fp = pa[a].vars[k];
      FftVar v{};
      v.len = fp.len;
      v.nst = (int)fp.rad.size();
      for (int st = 0; st < v.nst; ++st) {
        v.radix[st] = fp.rad[st];
        v.twoff[st] = fp.twoff[st];
      }
      v.twd = reinterpret_cast<const double*>(base + pa[a].var_d[k]);
      v.twf = reinterpret_cast<const float*>(base + pa[a].var_f[k]);
      v.twq = reinterpret_cast<const df*>(base + pa[a].var_q[k]);
      P->fvar[a].push_back(v);
    }
    // per precision: Bluestein (F > L) or the direct length-L FFT, default
    // radix sequence and tile
    int L, F;
    if (!choose_transform(A, sizeof(double), &L, &F, &P->PPd[a], &P->ldtd[a]))
      return fail(IFFD_ERR_UNSUPPORTED, "transform length too large for shared memory");
    fill_axistab(&P->axd[a], A, L, F, base, pa[a].od);
    P->vsel_d[a] = default_var(P->fvar[a], F);
    set_fft(&P->axd[a], P->fvar[a][P->vsel_d[a]]);
    if (!choose_transform(A, sizeof(float), &L, &F, &P->PPf[a], &P->ldtf[a]))
      return fail(IFFD_ERR_UNSUPPORTED, "transform length too large for shared memory");
    fill_axistab(&P->axf[a], A, L, F, base, pa[a].of);
    P->vsel_f[a] = default_var(P->fvar[a], F);
    set_fft(&P->axf[a], P->fvar[a][P->vsel_f[a]]);
    P->wtab[a] = reinterpret_cast<const float2*>(base + pa[a].wt);
    P->wtab_d[a] = reinterpret_cast<const double2*>(base + pa[a].wt_d);
    // double-float tables: the FP64 transform layout (L, F) and its radix
    // sequence (the block passes of directions without a warp-FFT pass)
    fill_axistab(&P->axq[a], A, P->axd[a].L, P->axd[a].F, base, pa[a].oq);
    set_fft(&P->axq[a], P->fvar[a][P->vsel_d[a]]);
    P->wtab_q[a] = reinterpret_cast<const df2*>(base + pa[a].wt_q);
    P->warp_f[a] = 0;
    P->warp_d[a] = 0;
    if (const int wN = wpass_len(P->axf[a])) {
      // the warp-FFT pass by default, unless its larger tiles leave the GPU
      // underfilled where the block kernel's would not
      const int tw = precond_tiles(P->dims, a, wpass_pencils(wN)), tb = precond_tiles(P->dims, a, P->PPf[a]);
      P->warp_f[a] = (tw >= 152 || tb < 152) ? 1 : 0;
      // paired on the last direction (the fused pass, where it measured ~10 %
      // faster; the single passes measured ~5 % slower paired: fewer
      // instructions per value, but a third fewer resident warps)
      P->pair_f[a] = (P->warp_f[a] && wN <= 256 && a == P->d - 1) ? 1 : 0;
    }
    BandTab& b = P->bt[a];
    b.m = A.m;
    b.p = A.p;
    b.Mb = reinterpret_cast<const double*>(base + pa[a].Mb);
    b.Kb = reinterpret_cast<const double*>(base + pa[a].Kb);
    b.Mt = reinterpret_cast<const double*>(base + pa[a].Mt);
    b.Kt = reinterpret_cast<const double*>(base + pa[a].Kt);
    b.ilo = pa[a].ilo;
    b.ihi = pa[a].ihi;
    P->ldts[a] = A.m | 1;
    int pp = 8;
    while (pp > 2 && (size_t)2 * pp * P->ldts[a] * sizeof(double) > 100 * 1024) pp /= 2;
    P->PPs[a] = pp;
    pp = 16;
    while (pp > 2 && (size_t)4 * pp * P->ldts[a] * sizeof(double) > 110 * 1024) pp /= 2;
    P->PPv[a] = pp;
    if (P->opt.coef == IFFD_COEF_SEPARABLE_SIN) {
      P->wb[a].Msb = reinterpret_cast<const double*>(base + pa[a].Msb);
      P->wb[a].Ksb = reinterpret_cast<const double*>(base + pa[a].Ksb);
      P->wb[a].c = P->opt.coef_amp;
      max_parts = std::max(max_parts, stiff_tiles(P->dims, a, P->PPv[a]));
    }
    if (P->opt.precond == IFFD_PRECOND_EXACT_FD) {
      P->Q[a] = reinterpret_cast<const double*>(base + pa[a].Q);
      P->QT[a] = reinterpret_cast<const double*>(base + pa[a].QT);
      P->lamQ[a] = reinterpret_cast<const double*>(base + pa[a].lamQ);
    }
    // partial sums: room for the smallest tile the tuner may pick
    max_parts = std::max(max_parts, precond_tiles(P->dims, a, kMinTunePP));
    max_parts = std::max(max_parts, stiff_tiles(P->dims, a, kMinTunePP));
  }
  P->max_parts = max_parts;
  // FP64 plans: the double-float passes by default where every direction can
  // run one and their tiles fill the GPU. Small problems are latency-bound (a
  // few long CTAs); they take the FP64-pipe block kernel instead, its tile
  // narrowed (8, 4, 2 pencils) until the tiles fill the GPU or reach 2 pencils
  // (65^2, p = 3: 0.61 against 0.71 ms per solve).
  {
    const int sms = device_sm_count();
    bool fills = true;
    for (int a = 0; a < P->d; ++a) {
      const int wN = wpass_len(P->axq[a]);
      if (precond_tiles(P->dims, a, wN ? wpass_pencils(wN) : P->PPd[a]) < sms) fills = false;
    }
    P->dfq = dfq_eligible(*P) && fills;
    for (int a = 0; a < P->d; ++a)
      while (P->PPd[a] > 2 && precond_tiles(P->dims, a, P->PPd[a]) < sms) P->PPd[a] /= 2;
  }
  const size_t vec = align256((size_t)N * sizeof(double));
  size_t off = 0;
  P->off_r = off; off += vec;
  P->off_z = off; off += vec;
  P->off_p = off; off += vec;
  P->off_q = off; off += vec;
  P->off_t1 = off; off += vec;
  P->off_t2 = off; off += vec;
  P->off_t3 = off;
  P->off_t4 = off;
  if (P->opt.coef == IFFD_COEF_SEPARABLE_SIN) {
    P->off_t4 = off + vec;
    off += 2 * vec;
  }
  P->off_tf = off;
  if (P->opt.precision == IFFD_PREC_FP32_TRANSFORM) off += align256((size_t)N * sizeof(float));
  P->off_part = off; off += align256((size_t)2 * max_parts * sizeof(double));
  P->off_state = off; off += align256(sizeof(SolveState));
  P->ws_bytes = off;
  IFFD_CUDA(cudaHostAlloc((void**)&P->host_state, sizeof(SolveState), cudaHostAllocDefault));
  return IFFD_OK;
}

// ------------------------------------------------------------- operations
static char* wsb(void* ws, size_t off) { return static_cast<char*>(ws) + off; }

__global__ void dot_kernel(const double* __restrict__ a, const double* __restrict__ b, long long N,
                           double* __restrict__ partial, const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  __shared__ double red[kThreads / 32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void copy_kernel(const double* __restrict__ a, double* __restrict__ b, long long N,
                            const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    b[i] = a[i];
}

template <typename Tc>
PassLaunch<Tc> make_pass(const Plan* P, int axis, const AxisTab<Tc>* tabs, const int* PPs, const int* ldts,
                         const int* done) {
  PassLaunch<Tc> L;
  L.dims = P->dims;
  L.axis = axis;
  L.PP = PPs[axis];
  L.ldt = ldts[axis];
  L.ax = tabs[axis];
  L.lamA = tabs[0].lam;
  L.lamB = (P->d == 3) ? tabs[1].lam : tabs[0].lam;
  L.dot0 = nullptr;
  L.dot1 = nullptr;
  L.partial = nullptr;
  L.done = done;
  L.pipe = std::is_same<Tc, double>::value ? P->pipe_d[axis] : P->pipe_f[axis];
  L.wN = 0;
  L.wt = nullptr;
  L.pair = 0;
  if constexpr (std::is_same<Tc, float>::value) {
    const F32Geom g = f32_geom(*P, axis);
    if (g.wN) {
      L.PP = g.PP;
      L.ldt = g.ldt;
      L.wN = g.wN;
      L.wt = g.wt;
      L.pipe = 0;
      L.pair = g.pair;
    }
  } else {
    if (const int wN = f64_warp_len(*P, axis)) {
      L.PP = wpass_pencils(wN);
      L.ldt = wpass_ldt(wN, P->axd[axis].m, walias<double>());
      L.wN = wN;
      L.wt = P->wtab_d[axis];
      L.pipe = 0;
    }
  }
  return L;
}

// Double-float transforms for an FP64 IFFD plan: every direction runs the
// double-float warp-FFT pass (lengths 64, 128, 256) or the double-float block
// kernel (any length run without Bluestein's convolution).
static bool df_warp_dir(const Plan& P, int a) {
  return wpass_len(P.axq[a]) > 0 && P.dims.N / P.axq[a].m < (1LL << 31);
}
int dfq_eligible(const Plan& P) {
  if (P.opt.precision != IFFD_PREC_FP64 || P.opt.precond != IFFD_PRECOND_IFFD) return 0;
  for (int a = 0; a < P.d; ++a)
    if (!df_warp_dir(P, a) && P.axq[a].blu) return 0;
  return 1;
}

// The double-float pass along direction `axis` (see Plan::dfq): the warp-FFT
// pass, or the block kernel with the FP64 plan's tile (both values take 8 bytes).
static PassLaunch<df> make_pass_df(const Plan* P, int axis, const int* done) {
  PassLaunch<df> L{};
  L.dims = P->dims;
  L.axis = axis;
  L.ax = P->axq[axis];
  L.lamA = P->axq[0].lam;
  L.lamB = (P->d == 3) ? P->axq[1].lam : P->axq[0].lam;
  L.done = done;
  L.pipe = 0;
  if (df_warp_dir(*P, axis)) {
    L.wN = wpass_len(P->axq[axis]);
    L.PP = wpass_pencils(L.wN);
    L.ldt = wpass_ldt(L.wN, P->axq[axis].m, walias<df>());
    L.wt = P->wtab_q[axis];
  } else {
    L.wN = 0;
    L.PP = P->PPd[axis];
    L.ldt = P->ldtd[axis];
    L.wt = nullptr;
  }
  return L;
}

int f32_last_parts(const Plan& P) {
  const F32Geom g = f32_geom(P, 0);
  return precond_tiles(P.dims, 0, g.PP) * (g.pair ? 2 : 1);
}

int f64_warp_len(const Plan& P, int a) {
  return (P.warp_d[a] && P.dims.N / P.axd[a].m < (1LL << 31)) ? wpass_len(P.axd[a]) : 0;
}

F32Geom f32_geom(const Plan& P, int a) {
  F32Geom g{P.PPf[a], P.ldtf[a], 0, nullptr, 0, 0};
  const int wN = (P.warp_f[a] && P.dims.N / P.axf[a].m < (1LL << 31)) ? wpass_len(P.axf[a]) : 0;
  if (wN) {
    g.wN = wN;
    g.wt = P.wtab[a];
    g.pair = (P.pair_f[a] && wN <= 256) ? 1 : 0;
    g.PP = wpass_pencils(wN, g.pair);
    g.ldt = wpass_ldt(wN, P.axf[a].m, walias<float>());
    g.smem = wpass_smem_bytes(wN, g.ldt, sizeof(float), g.pair, walias<float>());
  } else {
    g.smem = precond_smem_bytes(g.PP, g.ldt, P.axf[a].F, sizeof(float));
  }
  return g;
}
template PassLaunch<double> make_pass<double>(const Plan*, int, const AxisTab<double>*, const int*, const int*,
                                              const int*);
template PassLaunch<float> make_pass<float>(const Plan*, int, const AxisTab<float>*, const int*, const int*,
                                            const int*);

// z = P^{-1} r; with ndot >= 1 also partial (dot0, z) [and (dot1, z)] into
// `partial`; *nparts receives the number of partial sums.
static int run_precond(const Plan* P, const double* r, double* z, void* ws, cudaStream_t st, const int* done,
                       int ndot, const double* d0, const double* d1, double* partial, int* nparts) {
  const int d = P->d;
  const long long N = P->dims.N;
  if (P->opt.precond == IFFD_PRECOND_NONE || P->opt.precond == IFFD_PRECOND_EXACT_FD) {
    if (P->opt.precond == IFFD_PRECOND_NONE) {
      P->prof.begin(IFFD_K_VECTOR, st);
      copy_kernel<<<vec_grid(N), kThreads, 0, st>>>(r, z, N, done);
      IFFD_CUDA(cudaGetLastError());
      P->prof.end(st);
    } else {
      for (int a = 0; a < d - 1; ++a) {
        IFFD_LAUNCH(P, IFFD_K_FD_PASS, st,
                    launch_fd_pass(PM_FWD, a == 0 ? r : z, z, P->dims, a, P->QT[a], P->Q[a], P->lamQ[a],
                                   P->lamQ[0], P->lamQ[1], done, st));
      }
      IFFD_LAUNCH(P, IFFD_K_FD_PASS, st,
                  launch_fd_pass(PM_FUSED, z, z, P->dims, d - 1, P->QT[d - 1], P->Q[d - 1], P->lamQ[d - 1],
                                 P->lamQ[0], P->lamQ[1], done, st));
      for (int a = d - 2; a >= 0; --a) {
        IFFD_LAUNCH(P, IFFD_K_FD_PASS, st,
                    launch_fd_pass(PM_BWD, z, z, P->dims, a, P->QT[a], P->Q[a], P->lamQ[a], P->lamQ[0],
                                   P->lamQ[1], done, st));
      }
    }
    if (ndot >= 1) {
      const int g = vec_grid(N);
      P->prof.begin(IFFD_K_VECTOR, st);
      dot_kernel<<<g, kThreads, 0, st>>>(d0, z, N, partial, done);
      IFFD_CUDA(cudaGetLastError());
      P->prof.end(st);
      if (ndot >= 2) {
        P->prof.begin(IFFD_K_VECTOR, st);
        dot_kernel<<<g, kThreads, 0, st>>>(d1, z, N, partial + g, done);
        IFFD_CUDA(cudaGetLastError());
        P->prof.end(st);
      }
      *nparts = g;
    }
    return IFFD_OK;
  }
  if (P->opt.precision == IFFD_PREC_FP64 && P->dfq) {
    // double-float passes: r (FP64) -> z holding df values -> ... -> z (FP64);
    // a df value takes the 8 bytes of the FP64 value it stands for
    df* zq = reinterpret_cast<df*>(z);
    {
      auto L = make_pass_df(P, 0, done);
      IFFD_LAUNCH(P, IFFD_K_PRECOND_FWD, st, (launch_pass_df<double, df>(L, PM_FWD, 0, r, zq, st)));
    }
    for (int a = 1; a < d - 1; ++a) {
      auto L = make_pass_df(P, a, done);
      IFFD_LAUNCH(P, IFFD_K_PRECOND_FWD, st, (launch_pass_df<df, df>(L, PM_FWD, 0, zq, zq, st)));
    }
    {
      auto L = make_pass_df(P, d - 1, done);
      IFFD_LAUNCH(P, IFFD_K_PRECOND_FUSED, st, (launch_pass_df<df, df>(L, PM_FUSED, 0, zq, zq, st)));
    }
    for (int a = d - 2; a >= 1; --a) {
      auto L = make_pass_df(P, a, done);
      IFFD_LAUNCH(P, IFFD_K_PRECOND_BWD, st, (launch_pass_df<df, df>(L, PM_BWD, 0, zq, zq, st)));
    }
    {
      auto L = make_pass_df(P, 0, done);
      int nd = 0;
      if (ndot >= 1) {
        nd = ndot;
        L.dot0 = d0;
        L.dot1 = d1;
        L.partial = partial;
        *nparts = precond_tiles(P->dims, 0, L.PP);
      }
      IFFD_LAUNCH(P, IFFD_K_PRECOND_BWD, st, (launch_pass_df<df, double>(L, PM_BWD, nd, zq, z, st)));
    }
    return IFFD_OK;
  }
  if (P->opt.precision == IFFD_PREC_FP64) {
    for (int a = 0; a < d - 1; ++a) {
      auto L = make_pass<double>(P, a, P->axd, P->PPd, P->ldtd, done);
      IFFD_LAUNCH(P, IFFD_K_PRECOND_FWD, st, (launch_pass<double, double, double>(L, PM_FWD, 0, a == 0 ? r : z, z, st)));
    }
    {
      auto L = make_pass<double>(P, d - 1, P->axd, P->PPd, P->ldtd, done);
      IFFD_LAUNCH(P, IFFD_K_PRECOND_FUSED, st, (launch_pass<double, double, double>(L, PM_FUSED, 0, z, z, st)));
    }
    for (int a = d - 2; a >= 0; --a) {
      auto L = make_pass<double>(P, a, P->axd, P->PPd, P->ldtd, done);
      int nd = 0;
      if (a == 0 && ndot >= 1) {
        nd = ndot;
        L.dot0 = d0;
        L.dot1 = d1;
        L.partial = partial;
        *nparts = precond_tiles(P->dims, 0, L.PP);
      }
      IFFD_LAUNCH(P, IFFD_K_PRECOND_BWD, st, (launch_pass<double, double, double>(L, PM_BWD, nd, z, z, st)));
    }
    return IFFD_OK;
  }
  // float32 transforms: float intermediate in the workspace
  float* tf = reinterpret_cast<float*>(wsb(ws, P->off_tf));
  {
    auto L = make_pass<float>(P, 0, P->axf, P->PPf, P->ldtf, done);
    IFFD_LAUNCH(P, IFFD_K_PRECOND_FWD, st, (launch_pass<float, double, float>(L, PM_FWD, 0, r, tf, st)));
  }
  for (int a = 1; a < d - 1; ++a) {
    auto L = make_pass<float>(P, a, P->axf, P->PPf, P->ldtf, done);
    IFFD_LAUNCH(P, IFFD_K_PRECOND_FWD, st, (launch_pass<float, float, float>(L, PM_FWD, 0, tf, tf, st)));
  }
  {
    auto L = make_pass<float>(P, d - 1, P->axf, P->PPf, P->ldtf, done);
    IFFD_LAUNCH(P, IFFD_K_PRECOND_FUSED, st, (launch_pass<float, float, float>(L, PM_FUSED, 0, tf, tf, st)));
  }
  for (int a = d - 2; a >= 1; --a) {
    auto L = make_pass<float>(P, a, P->axf, P->PPf, P->ldtf, done);
    IFFD_LAUNCH(P, IFFD_K_PRECOND_BWD, st, (launch_pass<float, float, float>(L, PM_BWD, 0, tf, tf, st)));
  }
  {
    auto L = make_pass<float>(P, 0, P->axf, P->PPf, P->ldtf, done);
    int nd = 0;
    if (ndot >= 1) {
      nd = ndot;
      L.dot0 = d0;
      L.dot1 = d1;
      L.partial = partial;
      *nparts = f32_last_parts(*P);
    }
    IFFD_LAUNCH(P, IFFD_K_PRECOND_BWD, st, (launch_pass<float, float, double>(L, PM_BWD, nd, tf, z, st)));
  }
  return IFFD_OK;
}

StiffLaunch make_stiff(const Plan* P, int axis) {
  StiffLaunch S;
  S.dims = P->dims;
  S.axis = axis;
  S.PP = P->PPs[axis];
  S.ldt = P->ldts[axis];
  S.bt = P->bt[axis];
  return S;
}

// out = A^ u (pmode 0), or with the PCG direction update fused (pmode 1: p = z;
// pmode 2: p = z + beta p) applied to p. Optional partial (dotv, out).
static int run_stiffness(const Plan* P, const double* u, const double* z, double* p, const double* beta, int pmode,
                         double* out, void* ws, cudaStream_t st, const int* done, const double* dotv,
                         double* partial, int* nparts) {
  double* T1 = reinterpret_cast<double*>(wsb(ws, P->off_t1));
  double* T2 = reinterpret_cast<double*>(wsb(ws, P->off_t2));
  const int d = P->d;
  if (P->opt.coef == IFFD_COEF_SEPARABLE_SIN) {
    double* T3 = reinterpret_cast<double*>(wsb(ws, P->off_t3));
    double* T4 = reinterpret_cast<double*>(wsb(ws, P->off_t4));
    auto SV = [&](int a) {
      StiffLaunch S = make_stiff(P, a);
      S.PP = P->PPv[a];
      return S;
    };
    IFFD_LAUNCH(P, IFFD_K_STIFF_FIRST, st,
                launch_vstiff_first(SV(d - 1), P->wb[d - 1], u, z, p, beta, pmode, T1, T2, T3, T4, done, st));
    for (int a = d - 2; a >= 1; --a)
      IFFD_LAUNCH(P, IFFD_K_STIFF_MID, st, launch_vstiff_mid(SV(a), P->wb[a], T1, T2, T3, T4, done, st));
    IFFD_LAUNCH(P, IFFD_K_STIFF_LAST, st,
                launch_vstiff_last(SV(0), P->wb[0], T1, T2, T3, T4, out, dotv, partial, done, st));
    if (nparts) *nparts = stiff_tiles(P->dims, 0, P->PPv[0]);
    return IFFD_OK;
  }
  IFFD_LAUNCH(P, IFFD_K_STIFF_FIRST, st,
              launch_stiff_first(make_stiff(P, d - 1), u, z, p, beta, pmode, T1, T2, done, st));
  for (int a = d - 2; a >= 1; --a)
    IFFD_LAUNCH(P, IFFD_K_STIFF_MID, st, launch_stiff_mid(make_stiff(P, a), T1, T2, done, st));
  IFFD_LAUNCH(P, IFFD_K_STIFF_LAST, st, launch_stiff_last(make_stiff(P, 0), T1, T2, out, dotv, partial, done, st));
  if (nparts) *nparts = stiff_tiles(P->dims, 0, P->PPs[0]);
  return IFFD_OK;
}

static int check_ws(const Plan* P, void* ws) {
  if (ws == nullptr) return fail(IFFD_ERR_WORKSPACE, "workspace pointer is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(IFFD_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  (void)P;
  return IFFD_OK;
}

static int check_device(const Plan* P) {
  int dev = -1;
  IFFD_CUDA(cudaGetDevice(&dev));
  if (dev != P->device) return fail(IFFD_ERR_INVALID_ARG, "plan was created on another CUDA device");
  return IFFD_OK;
}

}  // namespace iffd

using namespace iffd;


namespace iffd {

// Support of iffd_apply_stiffness_noalloc (csrc/noalloc.cu): the three
// stiffness sweeps of plan h with caller-given temporaries T1, T2 (each at
// least N doubles). Counts the launches; records no profiler events.
int plan_stiffness_with_scratch(iffd_handle h, const double* u, double* Au, double* T1, double* T2,
                                cudaStream_t st) {
  const Plan* P = &h->P;
  if (P->opt.coef != IFFD_COEF_CONST)
    return fail(IFFD_ERR_UNSUPPORTED, "iffd_apply_stiffness_noalloc: only IFFD_COEF_CONST plans are supported");
  int rc = check_device(P);
  if (rc) return rc;
  const int d = P->d;
  P->prof.launches += d;
  IFFD_CUDA(launch_stiff_first(make_stiff(P, d - 1), u, nullptr, nullptr, nullptr, 0, T1, T2, nullptr, st));
  for (int a = d - 2; a >= 1; --a) IFFD_CUDA(launch_stiff_mid(make_stiff(P, a), T1, T2, nullptr, st));
  IFFD_CUDA(launch_stiff_last(make_stiff(P, 0), T1, T2, Au, nullptr, nullptr, nullptr, st));
  return IFFD_OK;
}

int plan_check_noalloc(iffd_handle h) {
  const Plan* P = &h->P;
  int rc = check_device(P);
  if (rc) return rc;
  if (P->opt.coef != IFFD_COEF_CONST)
    return fail(IFFD_ERR_UNSUPPORTED, "iffd_apply_stiffness_noalloc: only IFFD_COEF_CONST plans are supported");
  return IFFD_OK;
}

long long plan_num_dofs(iffd_handle h) { return h->P.dims.N; }

// ||f - A u|| / ||f|| of a finished solve, with the kernels of iffd_pcg_solve's
// exit check, on the plan's workspace ws (its solve state is overwritten).
int plan_true_residual(iffd_handle h, const double* f, const double* u, void* ws, cudaStream_t st, double* out) {
  const Plan* P = &h->P;
  const long long N = P->dims.N;
  double* q = reinterpret_cast<double*>(wsb(ws, P->off_q));
  double* part = reinterpret_cast<double*>(wsb(ws, P->off_part));
  SolveState* S = reinterpret_cast<SolveState*>(wsb(ws, P->off_state));
  const double tol2 = P->opt.rtol * P->opt.rtol;
  IFFD_LAUNCH(P, IFFD_K_VECTOR, st, (dot_kernel<<<vec_grid(N), kThreads, 0, st>>>(f, f, N, part, nullptr),
                                     cudaGetLastError()));
  IFFD_LAUNCH(P, IFFD_K_FINALIZE, st, launch_finalize(S, part, vec_grid(N), FP_FF, tol2, P->opt.maxit, st));
  int rc = run_stiffness(P, u, nullptr, nullptr, nullptr, 0, q, ws, st, nullptr, nullptr, nullptr, nullptr);
  if (rc) return rc;
  IFFD_LAUNCH(P, IFFD_K_VECTOR, st, launch_residual(f, q, N, part, st));
  IFFD_LAUNCH(P, IFFD_K_FINALIZE, st, launch_finalize(S, part, vec_grid(N), FP_TRUE, tol2, P->opt.maxit, st));
  IFFD_CUDA(cudaMemcpyAsync(P->host_state, S, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
  IFFD_CUDA(cudaStreamSynchronize(st));
  *out = P->host_state->ff > 0.0 ? std::sqrt(P->host_state->zq / P->host_state->ff) : 0.0;
  return IFFD_OK;
}

int record_error(int code, const std::string& msg) { return fail(code, msg); }

}  // namespace iffd

namespace iffd {

int plan_create(int d, const int* n_elems, int p, const int* dirichlet, const iffd_options* opt, cudaStream_t stream,
                iffd_plan** outp, const int* nrep, const int* reps) {
  if (!outp || !n_elems || !dirichlet) return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  if (d != 2 && d != 3) return fail(IFFD_ERR_INVALID_ARG, "d must be 2 or 3");
  if (p < 1) return fail(IFFD_ERR_INVALID_ARG, "p must be >= 1");
  bool any_dir = false;
  for (int a = 0; a < d; ++a) any_dir = any_dir || dirichlet[2 * a] || dirichlet[2 * a + 1];
  if (!any_dir) return fail(IFFD_ERR_SINGULAR, "no Dirichlet boundary: the stiffness matrix is singular");
  iffd_options o;
  iffd_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != IFFD_PREC_FP64 && o.precision != IFFD_PREC_FP32_TRANSFORM)
    return fail(IFFD_ERR_INVALID_ARG, "unknown precision");
  if (o.precond < 0 || o.precond > 2) return fail(IFFD_ERR_INVALID_ARG, "unknown preconditioner");
  if (o.coef != IFFD_COEF_CONST && o.coef != IFFD_COEF_SEPARABLE_SIN)
    return fail(IFFD_ERR_UNSUPPORTED, "coefficient kind not supported");
  if (o.coef == IFFD_COEF_SEPARABLE_SIN && !(std::fabs(o.coef_amp) < 1.0))
    return fail(IFFD_ERR_INVALID_ARG, "coef_amp must satisfy |c| < 1 (positive coefficient)");
  if (!(o.rtol > 0.0) || o.maxit < 1) return fail(IFFD_ERR_INVALID_ARG, "rtol must be > 0 and maxit >= 1");
  iffd_plan* h = new iffd_plan();
  Plan* P = &h->P;
  P->d = d;
  P->p = p;
  P->opt = o;
  if (cudaGetDevice(&P->device) != cudaSuccess) {
    delete h;
    return fail(IFFD_ERR_CUDA, "no CUDA device");
  }
  const int* rp = reps;
  for (int a = 0; a < d; ++a) {
    P->n[a] = n_elems[a];
    std::vector<std::pair<int, int>> ra;
    for (int r = 0; nrep && r < nrep[a]; ++r, rp += 2) ra.push_back({rp[0], rp[1]});
    std::string err =
        build_axis(n_elems[a], p, dirichlet[2 * a] != 0, dirichlet[2 * a + 1] != 0, &P->host[a], ra);
    if (!err.empty()) {
      delete h;
      return fail(IFFD_ERR_UNSUPPORTED, err);
    }
    if (P->host[a].n_out > kMaxNout) {
      delete h;
      return fail(IFFD_ERR_UNSUPPORTED, "n_out above 16");
    }
    if (o.coef == IFFD_COEF_SEPARABLE_SIN) build_weighted_bands(&P->host[a]);
  }
  int rc = build_plan(P, stream);
  if (rc == IFFD_OK && o.precision == IFFD_PREC_FP64 && o.precond == IFFD_PRECOND_IFFD) {
    // reciprocals of the summed eigenvalues for the FUSED pass (8 N bytes)
    cudaError_t e = cudaMalloc(&P->rden, (size_t)P->dims.N * sizeof(double));
    if (e == cudaSuccess)
      e = launch_rden_fill(P->rden, P->dims, P->axd[d - 1].lam, P->axd[0].lam, P->axd[d == 3 ? 1 : 0].lam, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "eigenvalue reciprocals");
    else P->axd[d - 1].rden = P->rden;
  }
  if (rc == IFFD_OK) rc = build_general_tables(P, stream);
  if (rc != IFFD_OK) {
    const std::string msg = g_err;
    if (P->dev) cudaFree(P->dev);
    if (P->rden) cudaFree(P->rden);
    if (P->gen_mem) cudaFree(P->gen_mem);
    if (P->host_state) cudaFreeHost(P->host_state);
    delete h;
    g_err = msg;
    return rc;
  }
  *outp = h;
  return IFFD_OK;
}

// The opening launches of a PCG solve (Section 3, zero start): state reset,
// x = 0, r = f, (f, f), z = P^{-1} r with (r, z).
static int enqueue_start(const Plan* P, const double* f, double* u, void* ws, cudaStream_t st) {
  const long long N = P->dims.N;
  double* r = reinterpret_cast<double*>(wsb(ws, P->off_r));
  double* z = reinterpret_cast<double*>(wsb(ws, P->off_z));
  double* part = reinterpret_cast<double*>(wsb(ws, P->off_part));
  SolveState* S = reinterpret_cast<SolveState*>(wsb(ws, P->off_state));
  const double tol2 = P->opt.rtol * P->opt.rtol;
  const int maxit = P->opt.maxit;
  int np = 0;
  IFFD_LAUNCH(P, IFFD_K_PCG_INIT, st, launch_pcg_init(f, u, r, N, part, st, S));
  IFFD_LAUNCH(P, IFFD_K_FINALIZE, st, launch_finalize(S, part, vec_grid(N), FP_FF, tol2, maxit, st));
  const int rc = run_precond(P, r, z, ws, st, &S->done, 1, r, nullptr, part, &np);
  if (rc) return rc;
  IFFD_LAUNCH(P, IFFD_K_FINALIZE, st, launch_finalize(S, part, np, FP_RZ0, tol2, maxit, st));
  return IFFD_OK;
}

// One PCG iteration: p = z (it == 0) or z + beta p fused into the first
// stiffness sweep, q = A^ p with (p, q), alpha, x += alpha p, r -= alpha q with
// (r, r) and the stopping test, z = P^{-1} r with (r, z) (and (q, z) for the
// flexible beta), beta. Every kernel returns at once after the solve is done.
static int enqueue_iteration(const Plan* P, double* u, void* ws, cudaStream_t st, int it) {
  const long long N = P->dims.N;
  double* r = reinterpret_cast<double*>(wsb(ws, P->off_r));
  double* z = reinterpret_cast<double*>(wsb(ws, P->off_z));
  double* p = reinterpret_cast<double*>(wsb(ws, P->off_p));
  double* q = reinterpret_cast<double*>(wsb(ws, P->off_q));
  double* part = reinterpret_cast<double*>(wsb(ws, P->off_part));
  SolveState* S = reinterpret_cast<SolveState*>(wsb(ws, P->off_state));
  const int* done = &S->done;
  const double tol2 = P->opt.rtol * P->opt.rtol;
  const int maxit = P->opt.maxit;
  const bool flex = P->opt.flexible || P->opt.precision == IFFD_PREC_FP32_TRANSFORM;
  int np = 0;
  int rc = run_stiffness(P, nullptr, z, p, &S->beta, it == 0 ? 1 : 2, q, ws, st, done, p, part, &np);
  if (rc) return rc;
  IFFD_LAUNCH(P, IFFD_K_FINALIZE, st, launch_finalize(S, part, np, FP_PQ, tol2, maxit, st));
  IFFD_LAUNCH(P, IFFD_K_PCG_UPDATE, st, launch_pcg_update(u, r, p, q, S, N, part, done, st));
  IFFD_LAUNCH(P, IFFD_K_FINALIZE, st, launch_finalize(S, part, vec_grid(N), FP_RR, tol2, maxit, st));
  rc = run_precond(P, r, z, ws, st, done, flex ? 2 : 1, r, q, part, &np);
  if (rc) return rc;
  IFFD_LAUNCH(P, IFFD_K_FINALIZE, st, launch_finalize(S, part, np, flex ? FP_RZ_FLEX : FP_RZ, tol2, maxit, st));
  return IFFD_OK;
}

static void drop_graph(Plan::SolveGraph& g) {
  if (g.first) cudaGraphExecDestroy(g.first);
  if (g.next) cudaGraphExecDestroy(g.next);
  g = Plan::SolveGraph{};
}

static void drop_graphs(Plan::SolveGraphs& G) {
  for (auto& g : G.g) drop_graph(g);
}

void plan_drop_graphs(Plan* P) {
  drop_graphs(P->graphs);
  P->graphs.failed = false;
}

// Captures what `enqueue` launches on the plan's private stream into an
// executable graph; `kernels` receives the number of kernel launches in it.
template <typename Fn>
static int capture_graph(const Plan* P, Fn enqueue, cudaGraphExec_t* exec, long long* kernels) {
  cudaStream_t cap = P->graphs.cap;
  const long long l0 = P->prof.launches;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
  const int rc = enqueue(cap);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(cap, &g);
  *kernels = P->prof.launches - l0;
  P->prof.launches = l0;  // captured, not run
  if (rc || e != cudaSuccess || g == nullptr) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc ? rc : cuda_fail(e, "cudaStreamEndCapture");
  }
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *exec = nullptr;
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  return IFFD_OK;
}

// The two graphs of a solve on (f, u, ws), into slot g: the opening launches
// with the first `nfirst` iterations, and `chunk` later iterations.
static int capture_solve_graphs(const Plan* P, Plan::SolveGraph& g, const double* f, double* u, void* ws,
                                int nfirst, int chunk) {
  Plan::SolveGraphs& G = P->graphs;
  drop_graph(g);
  if (!G.cap) {
    const cudaError_t e = cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      G.cap = nullptr;
      return cuda_fail(e, "cudaStreamCreateWithFlags");
    }
  }
  int rc = capture_graph(
      P,
      [&](cudaStream_t cs) {
        int r = enqueue_start(P, f, u, ws, cs);
        for (int c = 0; c < nfirst && !r; ++c) r = enqueue_iteration(P, u, ws, cs, c);
        return r;
      },
      &g.first, &g.kfirst);
  if (rc) return rc;
  rc = capture_graph(
      P,
      [&](cudaStream_t cs) {
        int r = IFFD_OK;
        for (int c = 0; c < chunk && !r; ++c) r = enqueue_iteration(P, u, ws, cs, nfirst + c);
        return r;
      },
      &g.next, &g.knext);
  if (rc) return rc;
  g.f = f;
  g.u = u;
  g.ws = ws;
  g.nfirst = nfirst;
  return IFFD_OK;
}

// The graph set for a solve on (f, u, ws) whose first graph runs `nfirst`
// iterations, captured if this triple was one of the last two solves'
// (nullptr: launch directly).
static const Plan::SolveGraph* solve_graphs_for(const Plan* P, const double* f, double* u, void* ws, int nfirst,
                                                int chunk) {
  Plan::SolveGraphs& G = P->graphs;
  const unsigned long long now = ++G.tick;
  for (auto& g : G.g)
    if (g.first && g.next && g.f == f && g.u == u && g.ws == ws) {
      if (g.nfirst != nfirst) {  // the iteration count moved: capture again, same slot
        const long long replays = g.replays;
        if (capture_solve_graphs(P, g, f, u, ws, nfirst, chunk)) {
          drop_graphs(G);
          G.failed = true;
          g_err.clear();
          return nullptr;
        }
        g.replays = replays;
      }
      g.used = now;
      ++g.replays;
      return &g;
    }
  bool seen = false;
  for (int k = 0; k < 2; ++k) seen = seen || (G.seen_f[k] == f && G.seen_u[k] == u && G.seen_ws[k] == ws);
  G.seen_f[1] = G.seen_f[0];
  G.seen_u[1] = G.seen_u[0];
  G.seen_ws[1] = G.seen_ws[0];
  G.seen_f[0] = f;
  G.seen_u[0] = u;
  G.seen_ws[0] = ws;
  if (!seen) return nullptr;
  Plan::SolveGraph& slot = G.g[0].used <= G.g[1].used ? G.g[0] : G.g[1];
  if (slot.first && slot.replays == 0) {  // captures that are evicted unused: the caller's pattern
    drop_graphs(G);                       // does not repeat, launch directly from now on
    G.failed = true;
    return nullptr;
  }
  if (capture_solve_graphs(P, slot, f, u, ws, nfirst, chunk)) {  // not capturable here: direct launches for good
    drop_graphs(G);
    G.failed = true;
    g_err.clear();
    return nullptr;
  }
  slot.used = now;
  return &slot;
}

void plan_release(iffd_plan* h) {
  if (!h) return;
  Plan* P = &h->P;
  drop_graphs(P->graphs);
  if (P->graphs.cap) cudaStreamDestroy(P->graphs.cap);
  P->prof.release();
  if (P->dev) cudaFree(P->dev);
  if (P->rden) cudaFree(P->rden);
  if (P->gen_mem) cudaFree(P->gen_mem);
  if (P->host_state) cudaFreeHost(P->host_state);
  delete h;
}

StiffLaunch plan_stiff_launch(const Plan* P, int axis) { return make_stiff(P, axis); }

}  // namespace iffd

extern "C" {

int iffd_default_options(iffd_options* opt) {
  if (!opt) return fail(IFFD_ERR_INVALID_ARG, "opt is NULL");
  opt->precision = IFFD_PREC_FP64;
  opt->precond = IFFD_PRECOND_IFFD;
  opt->rtol = 1e-8;
  opt->maxit = 500;
  opt->coef = IFFD_COEF_CONST;
  opt->true_residual = 1;
  opt->flexible = 0;
  opt->coef_amp = 0.5;
  opt->autotune = 0;
  return IFFD_OK;
}

int iffd_setup_knots(int d, const int* n_elems, int p, const int* dirichlet, const int* nrep, const int* reps,
                     const iffd_options* opt, void* stream, iffd_handle* out) {
  g_err.clear();
  if (!out) return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  if (nrep) {
    if (d != 2 && d != 3) return fail(IFFD_ERR_INVALID_ARG, "d must be 2 or 3");
    int total = 0;
    for (int a = 0; a < d; ++a) {
      if (nrep[a] < 0) return fail(IFFD_ERR_INVALID_ARG, "negative repeated-knot count");
      total += nrep[a];
    }
    if (total > 0 && !reps) return fail(IFFD_ERR_INVALID_ARG, "reps is NULL");
  }
  iffd_plan* h = nullptr;
  const int rc = plan_create(d, n_elems, p, dirichlet, opt, static_cast<cudaStream_t>(stream), &h, nrep, reps);
  if (rc != IFFD_OK) return rc;
  *out = h;
  return IFFD_OK;
}

int iffd_setup(int d, const int* n_elems, int p, const int* dirichlet, const iffd_options* opt, void* stream,
               iffd_handle* out) {
  return iffd_setup_knots(d, n_elems, p, dirichlet, nullptr, nullptr, opt, stream, out);
}

int iffd_workspace_bytes(iffd_handle h, size_t* bytes) {
  if (!h || !bytes) return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  *bytes = h->P.ws_bytes;
  return IFFD_OK;
}

int iffd_get_dims(iffd_handle h, int axis, int* m, int* n_reg, int* n_out) {
  if (!h || axis < 0 || axis >= h->P.d) return fail(IFFD_ERR_INVALID_ARG, "bad handle or axis");
  const Axis1D& A = h->P.host[axis];
  if (m) *m = A.m;
  if (n_reg) *n_reg = A.n_reg;
  if (n_out) *n_out = A.n_out;
  return IFFD_OK;
}

// Dense V_reg (m x n_reg, row-major) as the device passes apply it.
static void dense_vreg(const Axis1D& A, double* V) { expand_vreg(A, V); }

int iffd_get_1d(iffd_handle h, int axis, double* M_band, double* K_band, double* lam, double* dtilde, double* Vreg,
                double* W) {
  if (!h || axis < 0 || axis >= h->P.d) return fail(IFFD_ERR_INVALID_ARG, "bad handle or axis");
  const Axis1D& A = h->P.host[axis];
  auto cp = [](double* dst, const std::vector<double>& v) {
    if (dst && !v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(double));
  };
  cp(M_band, A.Mband);
  cp(K_band, A.Kband);
  cp(lam, A.lam);
  cp(dtilde, A.dtilde);
  if (Vreg) dense_vreg(A, Vreg);
  cp(W, A.W);
  return IFFD_OK;
}

int iffd_host_axis_knots(int n, int p, const int* dirichlet, int nrep, const int* reps, int* m, int* n_reg,
                         int* n_out, double* M_band, double* K_band, double* lam, double* dtilde, double* Vreg,
                         double* W) {
  g_err.clear();
  if (!dirichlet) return fail(IFFD_ERR_INVALID_ARG, "dirichlet is NULL");
  if (nrep < 0 || (nrep > 0 && !reps)) return fail(IFFD_ERR_INVALID_ARG, "bad repeated-knot list");
  std::vector<std::pair<int, int>> ra;
  for (int r = 0; r < nrep; ++r) ra.push_back({reps[2 * r], reps[2 * r + 1]});
  Axis1D A;
  const std::string err = build_axis(n, p, dirichlet[0] != 0, dirichlet[1] != 0, &A, ra);
  if (!err.empty()) return fail(IFFD_ERR_UNSUPPORTED, err);
  if (m) *m = A.m;
  if (n_reg) *n_reg = A.n_reg;
  if (n_out) *n_out = A.n_out;
  auto cp = [](double* dst, const std::vector<double>& v) {
    if (dst && !v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(double));
  };
  cp(M_band, A.Mband);
  cp(K_band, A.Kband);
  cp(lam, A.lam);
  cp(dtilde, A.dtilde);
  if (Vreg) dense_vreg(A, Vreg);
  cp(W, A.W);
  return IFFD_OK;
}

int iffd_host_axis(int n, int p, const int* dirichlet, int* m, int* n_reg, int* n_out, double* M_band,
                   double* K_band, double* lam, double* dtilde, double* Vreg, double* W) {
  return iffd_host_axis_knots(n, p, dirichlet, 0, nullptr, m, n_reg, n_out, M_band, K_band, lam, dtilde, Vreg, W);
}

int iffd_host_transform(int n, int p, const int* dirichlet, int precision, int* L, int* F, int* pencils) {
  g_err.clear();
  if (!dirichlet || !L || !F) return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  if (precision != IFFD_PREC_FP64 && precision != IFFD_PREC_FP32_TRANSFORM)
    return fail(IFFD_ERR_INVALID_ARG, "unknown precision");
  Axis1D A;
  const std::string err = build_axis(n, p, dirichlet[0] != 0, dirichlet[1] != 0, &A);
  if (!err.empty()) return fail(IFFD_ERR_UNSUPPORTED, err);
  int PP = 0, ldt = 0;
  if (!choose_transform(A, precision == IFFD_PREC_FP64 ? sizeof(double) : sizeof(float), L, F, &PP, &ldt))
    return fail(IFFD_ERR_UNSUPPORTED, "transform length too large for shared memory");
  if (pencils) *pencils = PP;
  return IFFD_OK;
}

int iffd_apply_preconditioner(iffd_handle h, const double* r, double* z, void* ws, void* stream) {
  if (!h || !r || !z) return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  if (r == z) return fail(IFFD_ERR_INVALID_ARG, "r and z must not alias");
  int rc = check_ws(&h->P, ws);
  if (rc) return rc;
  rc = check_device(&h->P);
  if (rc) return rc;
  return run_precond(&h->P, r, z, ws, static_cast<cudaStream_t>(stream), nullptr, 0, nullptr, nullptr, nullptr,
                     nullptr);
}

int iffd_apply_stiffness(iffd_handle h, const double* u, double* Au, void* ws, void* stream) {
  if (!h || !u || !Au) return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  if (u == Au) return fail(IFFD_ERR_INVALID_ARG, "u and Au must not alias");
  int rc = check_ws(&h->P, ws);
  if (rc) return rc;
  rc = check_device(&h->P);
  if (rc) return rc;
  return run_stiffness(&h->P, u, nullptr, nullptr, nullptr, 0, Au, ws, static_cast<cudaStream_t>(stream), nullptr,
                       nullptr, nullptr, nullptr);
}

int iffd_pcg_solve(iffd_handle h, const double* f, double* u, void* ws, void* stream, iffd_pcg_info* info) {
  if (!h || !f || !u) return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  if (f == u) return fail(IFFD_ERR_INVALID_ARG, "f and u must not alias");
  int rc = check_ws(&h->P, ws);
  if (rc) return rc;
  rc = check_device(&h->P);
  if (rc) return rc;
  const Plan* P = &h->P;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long N = P->dims.N;
  double* q = reinterpret_cast<double*>(wsb(ws, P->off_q));
  double* part = reinterpret_cast<double*>(wsb(ws, P->off_part));
  SolveState* S = reinterpret_cast<SolveState*>(wsb(ws, P->off_state));
  const double tol2 = P->opt.rtol * P->opt.rtol;
  const int maxit = P->opt.maxit;
  const int chunk = 4;  // iterations enqueued between two reads of the solve state
  // The first chunk runs as many iterations as the plan's last converged
  // solve took, so that a repeated solve of the same kind reads its state
  // once and enqueues no iterations past its convergence (each of which
  // would launch a dozen kernels that exit at once).
  const int nfirst = std::min(maxit, P->last_iters > 0 ? P->last_iters : chunk);

  // Chunks run from captured CUDA graphs when they can (one launch per chunk
  // instead of ~50): not while per-launch event timing is on, and only for
  // the (f, u, workspace) they were captured with.
  const Plan::SolveGraph* graph = nullptr;
  if (!P->prof.on && !P->graphs.failed && maxit >= chunk) graph = solve_graphs_for(P, f, u, ws, nfirst, chunk);
  auto read_state = [&]() -> int {
    IFFD_CUDA(cudaMemcpyAsync(P->host_state, S, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
    IFFD_CUDA(cudaStreamSynchronize(st));
    return IFFD_OK;
  };
  int it = 0;
  bool finished = false;
  if (graph) {
    IFFD_CUDA(cudaGraphLaunch(graph->first, st));
    P->prof.launches += graph->kfirst;
    it = graph->nfirst;
    if ((rc = read_state())) return rc;
    finished = P->host_state->done || it >= maxit;
    while (!finished) {
      if (it + chunk <= maxit) {
        IFFD_CUDA(cudaGraphLaunch(graph->next, st));
        P->prof.launches += graph->knext;
        it += chunk;
      } else {
        for (; it < maxit; ++it)
          if ((rc = enqueue_iteration(P, u, ws, st, it))) return rc;
      }
      if ((rc = read_state())) return rc;
      finished = P->host_state->done || it >= maxit;
    }
  } else {
    if ((rc = enqueue_start(P, f, u, ws, st))) return rc;
    while (!finished) {
      const int n = it == 0 ? nfirst : chunk;
      for (int c = 0; c < n && it < maxit; ++c, ++it)
        if ((rc = enqueue_iteration(P, u, ws, st, it))) return rc;
      if ((rc = read_state())) return rc;
      finished = P->host_state->done || it >= maxit;
    }
  }
  SolveState hs = *P->host_state;
  if (hs.done && hs.status == IFFD_OK && hs.iters > 0) P->last_iters = hs.iters;
  double true_rel = -1.0;
  if (P->opt.true_residual && hs.ff > 0.0) {
    rc = run_stiffness(P, u, nullptr, nullptr, nullptr, 0, q, ws, st, nullptr, nullptr, nullptr, nullptr);
    if (rc) return rc;
    IFFD_LAUNCH(P, IFFD_K_VECTOR, st, launch_residual(f, q, N, part, st));
    IFFD_LAUNCH(P, IFFD_K_FINALIZE, st, launch_finalize(S, part, vec_grid(N), FP_TRUE, tol2, maxit, st));
    IFFD_CUDA(cudaMemcpyAsync(P->host_state, S, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
    IFFD_CUDA(cudaStreamSynchronize(st));
    true_rel = std::sqrt(P->host_state->zq / hs.ff);
  }
  int status = hs.status;
  if (!hs.done) status = IFFD_ERR_NOT_CONVERGED;
  if (info) {
    info->iters = hs.iters;
    info->rel_res = hs.ff > 0 ? std::sqrt(hs.rr / hs.ff) : 0.0;
    info->true_rel_res = true_rel;
    info->status = status;
  }
  if (status == IFFD_ERR_NOT_CONVERGED) return fail(status, "PCG did not reach rtol within maxit");
  if (status == IFFD_ERR_BREAKDOWN) return fail(status, "PCG breakdown (non-positive curvature or NaN)");
  return IFFD_OK;
}

// ------------------------------------------ general-coefficient stiffness
int iffd_quad_points(iffd_handle h, int axis, int* nq, double* x, double* w) {
  g_err.clear();
  if (!h || axis < 0 || axis >= h->P.d) return fail(IFFD_ERR_INVALID_ARG, "bad handle or axis");
  QuadAxis Q;
  build_quad_axis(h->P.host[axis], &Q);
  if (nq) *nq = Q.nq;
  if (x) std::memcpy(x, Q.x.data(), Q.x.size() * sizeof(double));
  if (w) std::memcpy(w, Q.w.data(), Q.w.size() * sizeof(double));
  return IFFD_OK;
}

int iffd_host_quad_axis(int n, int p, const int* dirichlet, int nrep, const int* reps, int* nq, int* m, double* x,
                        double* w, double* B, double* D) {
  g_err.clear();
  if (!dirichlet) return fail(IFFD_ERR_INVALID_ARG, "dirichlet is NULL");
  if (nrep < 0 || (nrep > 0 && !reps)) return fail(IFFD_ERR_INVALID_ARG, "bad repeated-knot list");
  std::vector<std::pair<int, int>> ra;
  for (int r = 0; r < nrep; ++r) ra.push_back({reps[2 * r], reps[2 * r + 1]});
  Axis1D A;
  const std::string err = build_axis(n, p, dirichlet[0] != 0, dirichlet[1] != 0, &A, ra);
  if (!err.empty()) return fail(IFFD_ERR_UNSUPPORTED, err);
  QuadAxis Q;
  build_quad_axis(A, &Q);
  if (nq) *nq = Q.nq;
  if (m) *m = Q.m;
  if (x) std::memcpy(x, Q.x.data(), Q.x.size() * sizeof(double));
  if (w) std::memcpy(w, Q.w.data(), Q.w.size() * sizeof(double));
  // dense B and D from the CSR rows, and their transposes checked against the
  // transposed CSR (the device applies both)
  for (int q = 0; q < Q.nq; ++q)
    for (int j = 0; j < Q.m; ++j) {
      if (B) B[(size_t)q * Q.m + j] = 0.0;
      if (D) D[(size_t)q * Q.m + j] = 0.0;
    }
  for (int q = 0; q < Q.nq; ++q)
    for (int k = Q.rp[q]; k < Q.rp[q + 1]; ++k) {
      if (B) B[(size_t)q * Q.m + Q.col[k]] = Q.bv[k];
      if (D) D[(size_t)q * Q.m + Q.col[k]] = Q.dv[k];
    }
  for (int j = 0; j < Q.m; ++j)
    for (int k = Q.trp[j]; k < Q.trp[j + 1]; ++k) {
      const int q = Q.tcol[k];
      bool found = false;
      for (int kk = Q.rp[q]; kk < Q.rp[q + 1]; ++kk)
        if (Q.col[kk] == j) found = Q.bv[kk] == Q.tbv[k] && Q.dv[kk] == Q.tdv[k];
      if (!found) return fail(IFFD_ERR_UNSUPPORTED, "transposed Gauss-point table is inconsistent");
    }
  if ((int)Q.tcol.size() != Q.rp[Q.nq]) return fail(IFFD_ERR_UNSUPPORTED, "transposed Gauss-point table size");
  return IFFD_OK;
}

int iffd_general_workspace_bytes(iffd_handle h, size_t* bytes) {
  g_err.clear();
  if (!h || !bytes) return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  *bytes = general_ws_bytes(&h->P);
  return IFFD_OK;
}

static int check_general(const Plan* P, const double* C, int ncomp, const void* gws) {
  if (!C) return fail(IFFD_ERR_INVALID_ARG, "coefficient is NULL");
  if (ncomp != 1 && ncomp != P->d * (P->d + 1) / 2)
    return fail(IFFD_ERR_INVALID_ARG, "ncomp must be 1 or d (d + 1) / 2");
  if (!gws) return fail(IFFD_ERR_WORKSPACE, "general workspace is NULL");
  if (reinterpret_cast<uintptr_t>(gws) % 256 != 0) return fail(IFFD_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  const long long rows = (long long)P->gen[1].nq * (P->d == 3 ? P->gen[2].nq : 1);
  if (rows >= (1LL << 31)) return fail(IFFD_ERR_UNSUPPORTED, "Gauss grid too large");
  if (P->p > kGenMaxDegree) return fail(IFFD_ERR_UNSUPPORTED, "general coefficient: degree above 11");
  return check_device(P);
}

int iffd_apply_stiffness_general(iffd_handle h, const double* C, int ncomp, const double* u, double* Au, void* gws,
                                 void* stream) {
  g_err.clear();
  if (!h || !u || !Au) return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  if (u == Au) return fail(IFFD_ERR_INVALID_ARG, "u and Au must not alias");
  int rc = check_general(&h->P, C, ncomp, gws);
  if (rc) return rc;
  return run_general(&h->P, C, ncomp, u, Au, gws, static_cast<cudaStream_t>(stream), nullptr);
}

// PCG on A_C u = f with the plan's preconditioner (the IFFD preconditioner of
// the constant-coefficient operator): the loop of iffd_pcg_solve with the
// general operator in place of the stiffness sweeps.
int iffd_pcg_solve_general(iffd_handle h, const double* C, int ncomp, const double* f, double* u, void* ws, void* gws,
                           void* stream, iffd_pcg_info* info) {
  g_err.clear();
  if (!h || !f || !u) return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  if (f == u) return fail(IFFD_ERR_INVALID_ARG, "f and u must not alias");
  Plan* P = &h->P;
  int rc = check_ws(P, ws);
  if (rc) return rc;
  rc = check_general(P, C, ncomp, gws);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long N = P->dims.N;
  double* r = reinterpret_cast<double*>(wsb(ws, P->off_r));
  double* z = reinterpret_cast<double*>(wsb(ws, P->off_z));
  double* p = reinterpret_cast<double*>(wsb(ws, P->off_p));
  double* q = reinterpret_cast<double*>(wsb(ws, P->off_q));
  double* part = reinterpret_cast<double*>(wsb(ws, P->off_part));
  SolveState* S = reinterpret_cast<SolveState*>(wsb(ws, P->off_state));
  const int* done = &S->done;
  const double tol2 = P->opt.rtol * P->opt.rtol;
  const int maxit = P->opt.maxit;
  const bool flex = P->opt.flexible || P->opt.precision == IFFD_PREC_FP32_TRANSFORM;
  const int g = vec_grid(N);
  int np = 0;

  IFFD_LAUNCH(P, IFFD_K_PCG_INIT, st, launch_pcg_init(f, u, r, N, part, st, S));
  IFFD_LAUNCH(P, IFFD_K_FINALIZE, st, launch_finalize(S, part, g, FP_FF, tol2, maxit, st));
  rc = run_precond(P, r, z, ws, st, done, 1, r, nullptr, part, &np);
  if (rc) return rc;
  IFFD_LAUNCH(P, IFFD_K_FINALIZE, st, launch_finalize(S, part, np, FP_RZ0, tol2, maxit, st));
  int it = 0;
  const int chunk = 4;
  bool finished = false;
  while (!finished) {
    for (int c = 0; c < chunk && it < maxit; ++c, ++it) {
      IFFD_LAUNCH(P, IFFD_K_GENERAL, st, launch_gen_pupdate(z, p, S, it == 0 ? 1 : 2, N, done, st));
      rc = run_general(P, C, ncomp, p, q, gws, st, done);
      if (rc) return rc;
      P->prof.begin(IFFD_K_VECTOR, st);
      dot_kernel<<<g, kThreads, 0, st>>>(p, q, N, part, done);
      IFFD_CUDA(cudaGetLastError());
      P->prof.end(st);
      IFFD_LAUNCH(P, IFFD_K_FINALIZE, st, launch_finalize(S, part, g, FP_PQ, tol2, maxit, st));
      IFFD_LAUNCH(P, IFFD_K_PCG_UPDATE, st, launch_pcg_update(u, r, p, q, S, N, part, done, st));
      IFFD_LAUNCH(P, IFFD_K_FINALIZE, st, launch_finalize(S, part, g, FP_RR, tol2, maxit, st));
      rc = run_precond(P, r, z, ws, st, done, flex ? 2 : 1, r, q, part, &np);
      if (rc) return rc;
      IFFD_LAUNCH(P, IFFD_K_FINALIZE, st, launch_finalize(S, part, np, flex ? FP_RZ_FLEX : FP_RZ, tol2, maxit, st));
    }
    IFFD_CUDA(cudaMemcpyAsync(P->host_state, S, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
    IFFD_CUDA(cudaStreamSynchronize(st));
    finished = P->host_state->done || it >= maxit;
  }
  SolveState hs = *P->host_state;
  double true_rel = -1.0;
  if (P->opt.true_residual && hs.ff > 0.0) {
    rc = run_general(P, C, ncomp, u, q, gws, st, nullptr);
    if (rc) return rc;
    IFFD_LAUNCH(P, IFFD_K_VECTOR, st, launch_residual(f, q, N, part, st));
    IFFD_LAUNCH(P, IFFD_K_FINALIZE, st, launch_finalize(S, part, g, FP_TRUE, tol2, maxit, st));
    IFFD_CUDA(cudaMemcpyAsync(P->host_state, S, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
    IFFD_CUDA(cudaStreamSynchronize(st));
    true_rel = std::sqrt(P->host_state->zq / hs.ff);
  }
  int status = hs.status;
  if (!hs.done) status = IFFD_ERR_NOT_CONVERGED;
  if (info) {
    info->iters = hs.iters;
    info->rel_res = hs.ff > 0 ? std::sqrt(hs.rr / hs.ff) : 0.0;
    info->true_rel_res = true_rel;
    info->status = status;
  }
  if (status == IFFD_ERR_NOT_CONVERGED) return fail(status, "PCG did not reach rtol within maxit");
  if (status == IFFD_ERR_BREAKDOWN) return fail(status, "PCG breakdown (non-positive curvature or NaN)");
  return IFFD_OK;
}

static const char* kKindNames[IFFD_K_KINDS] = {
    "precond_fwd", "precond_fused", "precond_bwd", "stiff_first", "stiff_mid", "stiff_last",
    "pcg_update", "pcg_init", "finalize", "fd_pass", "vector", "general"};

int iffd_profile_enable(iffd_handle h, int enable) {
  if (!h) return fail(IFFD_ERR_INVALID_ARG, "NULL handle");
  h->P.prof.on = enable != 0;
  return IFFD_OK;
}

int iffd_profile_reset(iffd_handle h) {
  if (!h) return fail(IFFD_ERR_INVALID_ARG, "NULL handle");
  cudaError_t e = h->P.prof.collect();
  if (e != cudaSuccess) return cuda_fail(e, "iffd_profile_reset");
  for (int k = 0; k < IFFD_K_KINDS; ++k) {
    h->P.prof.cnt[k] = 0;
    h->P.prof.ms[k] = 0.0;
  }
  return IFFD_OK;
}

int iffd_profile_read(iffd_handle h, int kind, long long* launches, double* ms, const char** name) {
  if (!h || kind < 0 || kind >= IFFD_K_KINDS) return fail(IFFD_ERR_INVALID_ARG, "bad handle or kind");
  cudaError_t e = h->P.prof.collect();
  if (e != cudaSuccess) return cuda_fail(e, "iffd_profile_read");
  if (launches) *launches = h->P.prof.cnt[kind];
  if (ms) *ms = h->P.prof.ms[kind];
  if (name) *name = kKindNames[kind];
  return IFFD_OK;
}

int iffd_launch_count(iffd_handle h, long long* count) {
  if (!h || !count) return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  *count = h->P.prof.launches;
  return IFFD_OK;
}

int iffd_destroy(iffd_handle h) {
  if (!h) return IFFD_OK;
  plan_release(h);
  return IFFD_OK;
}

const char* iffd_last_error(void) { return g_err.c_str(); }

}  // extern "C"
