// Transform passes with warp-local FFTs, FP32 or FP64 arithmetic T (one
// translation unit per FFT length includes this header).
//
// Same operator as precond_pass (Q~^T, Q~, or both with the eigenvalue scaling,
// eq. "preconditioner"), for the D = {0,1} directions of Table 1 whose FFT
// length N is 64, 128, 256 or 512: DST-II / DST-III (even p, N = n_reg, with
// Makhoul's reordering) and DST-I (odd p, N = 2 (n_reg + 1), odd extension). The block-wide
// kernel spends most of its instructions on run-time index arithmetic and on
// shared-memory round trips between its steps; with FP32 arithmetic that, not
// the FFT, limits it, and in FP64 its block-wide barriers between the steps
// leave part of the FP64 pipe idle. Here a pencil pair belongs to LS lanes of one warp from
// the edge gather to the output: the gather and Makhoul's reordering feed the
// first FFT stage directly, every stage reads its R = N / LS values per lane
// into registers, synchronises the warp and writes them back in place, and the
// separation / twiddle / D~^{-1} step writes the results into the tile. All
// sizes and the radix sequence (8, 8, then 8, 4 or 2) are compile-time
// constants; the only block-wide steps are the coalesced tile load and store.
#pragma once

#include <algorithm>
#include <type_traits>

#include "device_common.cuh"
#include "fpair.cuh"
#include "kernels.h"
#include "precond_dev.cuh"
#include "precond_warp_geom.h"

namespace iffd {

// Complex values in the sequence buffers are float2 / double2 (one 64- or
// 128-bit shared-memory access each).
template <typename T>
__device__ __forceinline__ Cplx<T> wld(const vec2_t<T>* b, int i) {
  const vec2_t<T> t = b[i];
  return {t.x, t.y};
}
template <typename T>
__device__ __forceinline__ void wst(vec2_t<T>* b, int i, Cplx<T> v) { b[i] = vec2_t<T>{v.x, v.y}; }

// The four post-processing factors of DST-II/III output pair k (AxisTab::post).
template <typename T>
struct Post4 {
  T x, y, z, w;
};
__device__ __forceinline__ Post4<float> ldpost(const float* p, int k) {
  const float4 t = ldg(reinterpret_cast<const float4*>(p) + k);
  return {t.x, t.y, t.z, t.w};
}
__device__ __forceinline__ Post4<double> ldpost(const double* p, int k) {
  const double2 a = ldg(reinterpret_cast<const double2*>(p) + 2 * k);
  const double2 b = ldg(reinterpret_cast<const double2*>(p) + 2 * k + 1);
  return {a.x, a.y, b.x, b.y};
}

__device__ __forceinline__ Post4<df> ldpost(const df* p, int k) {
  const float4 a = ldg(reinterpret_cast<const float4*>(p) + 2 * k);
  const float4 b = ldg(reinterpret_cast<const float4*>(p) + 2 * k + 1);
  return {{a.x, a.y}, {a.z, a.w}, {b.x, b.y}, {b.z, b.w}};
}

template <int r, typename T>
__device__ __forceinline__ void wdft(Cplx<T>* v) {
  if constexpr (r == 2) dft2(v);
  else if constexpr (r == 4) dft4(v);
  else dft8(v);
}

// One Stockham stage of radix r and span Ns on the sequence in buf (the same
// index map as fft_block): butterfly j takes in[j + q N/r], twiddles input q by
// exp(-2 pi i q k / (Ns r)), k = j mod Ns (table wt[e] = exp(-2 pi i e / N)),
// and writes out[(j - k) r + k + t Ns]. Lane ls runs butterflies ls + LS u.
template <typename T, int N, int r, int Ns>
__device__ __forceinline__ void wstage(vec2_t<T>* buf, int ls, const vec2_t<tab_t<T>>* __restrict__ wt) {
  constexpr int R = WarpFft<N>::R, LS = WarpFft<N>::LS, nb = N / r, BPL = R / r;
  static_assert(N % r == 0 && R % r == 0 && nb == LS * BPL, "stage does not tile the warp");
  // with nb and Ns multiples of 8 (Ns = 1 only with r = 8), the padded index
  // is linear in q and t: wpad(j + q nb) = wpad(j) + q (nb + nb / 8), and
  // wpad(base + t Ns) = wpad(base) + t (Ns + Ns / 8) (+ t when Ns = 1)
  static_assert(nb % 8 == 0 && (Ns % 8 == 0 || (Ns == 1 && r == 8)), "padded index not linear");
  constexpr int qstep = nb + nb / 8, tstep = (Ns == 1) ? 1 : Ns + Ns / 8;
  Cplx<T> v[BPL][r];
#pragma unroll
  for (int u = 0; u < BPL; ++u) {
    const vec2_t<T>* bj = buf + wpad(ls + LS * u);
#pragma unroll
    for (int q = 0; q < r; ++q) v[u][q] = wld<T>(bj, q * qstep);
  }
  __syncwarp();
#pragma unroll
  for (int u = 0; u < BPL; ++u) {
    const int j = ls + LS * u;
    const int k = j & (Ns - 1);
    if constexpr (Ns > 1) {
#pragma unroll
      for (int q = 1; q < r; ++q) {
        const vec2_t<tab_t<T>> w = ldg(wt + q * k * (N / (Ns * r)));
        v[u][q] = cmul(v[u][q], Cplx<tab_t<T>>{w.x, w.y});
      }
    }
    wdft<r>(v[u]);
    vec2_t<T>* bb = buf + wpad((j - k) * r + k);
#pragma unroll
    for (int t = 0; t < r; ++t) wst<T>(bb, t * tstep, v[u][t]);
  }
  __syncwarp();
}

// The stages after the first (span Ns = 8).
template <typename T, int N>
__device__ __forceinline__ void wfft_rest(vec2_t<T>* buf, int ls, const vec2_t<tab_t<T>>* __restrict__ wt) {
  wstage<T, N, 8, 8>(buf, ls, wt);
  if constexpr (N == 128) wstage<T, N, 2, 64>(buf, ls, wt);
  if constexpr (N == 256) wstage<T, N, 4, 64>(buf, ls, wt);
  if constexpr (N == 512) wstage<T, N, 8, 64>(buf, ls, wt);
}

// First stage (radix 8, span 1, no twiddles) with the inputs supplied by
// src(j, q) (sequence element j + q N/8; j < N/8, q a constant once unrolled).
template <typename T, int N, typename Src>
__device__ __forceinline__ void wstage_first(vec2_t<T>* buf, int ls, Src src) {
  constexpr int R = WarpFft<N>::R, LS = WarpFft<N>::LS, r = 8, nb = N / r, BPL = R / r;
  Cplx<T> v[BPL][r];
#pragma unroll
  for (int u = 0; u < BPL; ++u) {
    const int j = ls + LS * u;
#pragma unroll
    for (int q = 0; q < r; ++q) v[u][q] = src(j, q);
  }
  __syncwarp();
#pragma unroll
  for (int u = 0; u < BPL; ++u) {
    const int j = ls + LS * u;
    dft8(v[u]);
    vec2_t<T>* bb = buf + wpad(j * r);  // wpad(8 j + t) = wpad(8 j) + t
#pragma unroll
    for (int t = 0; t < r; ++t) wst<T>(bb, t, v[u][t]);
  }
  __syncwarp();
}

// Sum over the LS lanes of one sequence group (aligned, power of two).
template <int LS, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int off = LS / 2; off > 0; off >>= 1) v += shfl_xor(v, off);
  return v;
}

// Sums of V values (a power of two, V <= LS) of every lane over the LS lanes
// of its sequence group, scattered over the lanes: the halving rounds send
// half of a lane's values to its partner and keep the other half (V - 1
// exchanges instead of V log2(LS)), the remaining rounds exchange the single
// value left. Lane ls returns the group total of value ls / (LS / V).
template <int LS, int V, typename T>
__device__ __forceinline__ T group_sum_scatter(T (&v)[V], int ls) {
  static_assert(V >= 1 && V <= LS && (V & (V - 1)) == 0, "V: a power of two up to LS");
#pragma unroll
  for (int H = V / 2, off = LS / 2; H >= 1; H /= 2, off /= 2) {
    const bool upper = (ls & off) != 0;  // keeps the upper half of the values
#pragma unroll
    for (int i = 0; i < H; ++i) {
      const T keep = upper ? v[H + i] : v[i];
      const T send = upper ? v[i] : v[H + i];
      v[i] = keep + shfl_xor(send, off);
    }
  }
  T x = v[0];
#pragma unroll
  for (int off = LS / (2 * V); off > 0; off >>= 1) x += shfl_xor(x, off);
  return x;
}

// V_reg row rule of the scatter (x_i = sum_j V_reg[i][j] w_j): edge blocks,
// interior blocks, identity runs (see AxisTab).
template <typename T, typename TT, typename WReg>
__device__ __forceinline__ T wscatter_row(int i, const AxisTab<TT>& ax, WReg wreg) {
  const int m = ax.m, N = ax.n_reg;
  if (i < ax.rowsL) {
    T x = T(0);
    for (int c = 0; c < ax.nL; ++c) x = fma(ldg(ax.VL + i * ax.nL + c), wreg(c), x);
    return x;
  }
  if (i >= m - ax.rowsR) {
    const int r = m - 1 - i;
    T x = T(0);
    for (int c = 0; c < ax.nR; ++c) x = fma(ldg(ax.VR + r * ax.nR + c), wreg(N - 1 - c), x);
    return x;
  }
  int o = ax.o;
  for (int b = 0; b < ax.nblk; ++b) {
    const int* B = ax.blk + 6 * b;
    const int r0 = ldg(B + 2), r1 = ldg(B + 3);
    if (i < r0) break;
    if (i < r1) {
      const int c0 = ldg(B), c1 = ldg(B + 1);
      const TT* V = ax.VB + ldg(B + 5) + (i - r0) * (c1 - c0);
      T x = T(0);
      for (int c = c0; c < c1; ++c) x = fma(ldg(V + (c - c0)), wreg(c), x);
      return x;
    }
    o = ldg(B + 4);
  }
  return wreg(i - o);
}

// tile_setup with 32-bit quotients (the host limits these passes to fewer
// than 2^31 pencils per direction).
__device__ __forceinline__ TileInfo wtile_setup(const Dims& dims, int axis, int PP, long long tile, long long* pbase,
                                                int* pia, int* pib) {
  const unsigned m0 = dims.m[0], m1 = dims.m[1];
  const unsigned Q = (unsigned)(dims.N / dims.m[axis]);
  const unsigned q0 = (unsigned)tile * (unsigned)PP;
  TileInfo t;
  t.nvalid = (int)min((unsigned)PP, Q - q0);
  t.S = (axis == 0) ? 1 : ((axis == 1) ? (long long)m0 : (long long)m0 * m1);
  for (int pc = threadIdx.x; pc < PP; pc += blockDim.x) {
    unsigned q = q0 + pc;
    if (q >= Q) q = Q - 1;
    long long base;
    unsigned ia, ib;
    if (axis == 0) {
      base = (long long)q * m0;
      ib = q / m1;
      ia = q - ib * m1;
    } else {
      const unsigned rest = q / m0, x = q - rest * m0;
      ia = x;
      ib = rest;
      base = x + (long long)rest * ((axis == 1) ? (long long)m0 * m1 : (long long)m0);
    }
    pbase[pc] = base;
    pia[pc] = (int)ia;
    pib[pc] = (int)ib;
  }
  return t;
}

// The three steps of one tile: coalesced load into `tile` (row length ldt),
// warp-local transform, coalesced store. Each is called by the whole CTA.
template <int N, typename T, typename Tin>
__device__ __forceinline__ void wload_tile(const Tin* __restrict__ in, T* tile, int axis, int ldt,
                                           const AxisTab<T>& ax, const long long* pbase, const TileInfo& g) {
  constexpr int LS = WarpFft<N>::LS, PP = warp_pencils<N>(), G = 32 / LS;
  const int m = ax.m;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  (void)LS; (void)G; (void)tid; (void)warp; (void)lane;
  // ---- coalesced tile load (padding pencils are zero)
  constexpr int kW = kThreads / 32, kIPR = (N + kMaxNout + 31) / 32;  // rows of a warp: PP / kW
  constexpr bool kAll = std::is_same<T, df>::value && std::is_same<Tin, double>::value && (PP / kW) * kIPR <= 20;
  if (kAll && axis == 0) {
    // FP64 input of the double-float passes (lengths 128, 256): every value
    // of the warp's rows is loaded first (all in flight at once), then
    // converted and stored
    constexpr int RPW = PP / kW, IPR = kIPR;
    Tin v[RPW][IPR];
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      const int pc = warp + r * kW;
      const Tin* src = in + pbase[pc];
#pragma unroll
      for (int u = 0; u < IPR; ++u) {
        const int i = lane + 32 * u;
        v[r][u] = (pc < g.nvalid && i < m) ? src[i] : Tin(0);
      }
    }
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      T* row = tile + (warp + r * kW) * ldt;
#pragma unroll
      for (int u = 0; u < IPR; ++u) {
        const int i = lane + 32 * u;
        if (i < m) row[i] = cvt<T>(v[r][u]);
      }
    }
  } else if (axis == 0) {
    // two rows per warp at a time (rows pc and pc + 8): twice the loads in
    // flight of one row
    constexpr int W = kThreads / 32;
    static_assert(PP % (2 * W) == 0, "rows come in pairs per warp");
    for (int pc = warp; pc < PP; pc += 2 * W) {
      T* row0 = tile + pc * ldt;
      T* row1 = row0 + W * ldt;
      const bool v0 = pc < g.nvalid, v1 = pc + W < g.nvalid;
      const Tin* src0 = in + pbase[pc];
      const Tin* src1 = in + pbase[pc + W];
#pragma unroll 4
      for (int i = lane; i < m; i += 32) {
        const Tin a = v0 ? src0[i] : Tin(0);
        const Tin b = v1 ? src1[i] : Tin(0);
        row0[i] = cvt<T>(a);
        row1[i] = cvt<T>(b);
      }
    }
  } else {
    constexpr int RS = kThreads / PP;  // rows per sweep
    const int pc = tid & (PP - 1);
    const bool valid = pc < g.nvalid;
    const Tin* src = in + pbase[pc];
    const long long step = g.S * RS;
    int i = tid / PP;
    const Tin* p = src + i * g.S;
    for (; i + 3 * RS < m; i += 4 * RS, p += 4 * step) {
      Tin v0 = Tin(0), v1 = Tin(0), v2 = Tin(0), v3 = Tin(0);
      if (valid) {
        v0 = p[0];
        v1 = p[step];
        v2 = p[2 * step];
        v3 = p[3 * step];
      }
      tile[pc * ldt + i] = cvt<T>(v0);
      tile[pc * ldt + i + RS] = cvt<T>(v1);
      tile[pc * ldt + i + 2 * RS] = cvt<T>(v2);
      tile[pc * ldt + i + 3 * RS] = cvt<T>(v3);
    }
    for (; i < m; i += RS, p += step) tile[pc * ldt + i] = valid ? cvt<T>(p[0]) : T(0);
  }
}

// Pencils of tile row `row`: the row itself, or for a pair (f2 rows) the two
// pencils 4 (row / 2) + row % 2 and that + 2, so that the two sequences of a
// lane group combine the pencils (4 s, 4 s + 1) and (4 s + 2, 4 s + 3) as the
// unpaired pass combines (2 s, 2 s + 1).
template <typename T>
__device__ __forceinline__ int row_pencil(int row) {
  if constexpr (IsPair<T>::value) return 4 * (row >> 1) + (row & 1);
  else return row;
}
// A per-pencil table entry (eigenvalue of another direction) for tile row `row`.
template <typename T>
__device__ __forceinline__ T row_lam(const tab_t<T>* __restrict__ lam, const int* idx, int row) {
  const int p = row_pencil<T>(row);
  if constexpr (IsPair<T>::value) return f2{ldg(lam + idx[p]), ldg(lam + idx[p + 2])};
  else return ldg(lam + idx[p]);
}

// KIND 1: DST-II / DST-III (even p), FFT length N = n_reg in Makhoul's order;
// KIND 0: DST-I (odd p), FFT length N = 2 (n_reg + 1) of the odd extension.
// ALIAS: the sequence buffer of pencil pair pr occupies the pair's own two
// tile rows (ldt >= wbuf_len<N>(), see wpass_ldt; no separate buffer, so more
// CTAs fit on an SM): every step that moves values between the rows and the
// buffer reads all it needs into registers before the warp writes, and no
// other warp touches those rows. Otherwise the buffers follow the tile (wbuf).
template <typename T, int N, int KIND, int MODE, bool ALIAS>
__device__ __forceinline__ void wtransform(T* tile, vec2_t<T>* wbuf, T* outv, const Dims& dims, int ldt,
                                           const AxisTab<tab_t<T>>& ax, const vec2_t<tab_t<T>>* __restrict__ wt,
                                           const tab_t<T>* __restrict__ lamA, const tab_t<T>* __restrict__ lamB,
                                           const int* pia, const int* pib) {
  using TT = tab_t<T>;
  constexpr int LS = WarpFft<N>::LS, PP = warp_pencils<N>(), G = 32 / LS;
  const int m = ax.m;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  (void)LS; (void)G; (void)tid; (void)warp; (void)lane;
  // ---- warp-local transform of pencil pair pr (pencils 2 pr, 2 pr + 1)
  const int grp = lane / LS, ls = lane % LS;
  const int pr = warp * G + grp;
  T* ra = tile + (2 * pr) * ldt;
  T* rb = ra + ldt;
  T* ova = outv + (2 * pr) * kMaxNout;
  T* ovb = ova + kMaxNout;
  vec2_t<T>* buf = ALIAS ? reinterpret_cast<vec2_t<T>*>(ra)  // 2 ldt values >= wbuf_len<N>() complex
                         : wbuf + (size_t)pr * wbuf_len<N>();
  const int nw = ax.n_out;
  constexpr int NR = (KIND == 1) ? N : N / 2 - 1;  // n_reg

  if constexpr (MODE == PM_FWD || MODE == PM_FUSED) {
    // y_out = W^T r over the support rows of W, four columns per row read
    for (int k0 = 0; k0 < nw; k0 += 4) {
      T sa[4] = {T(0), T(0), T(0), T(0)}, sb[4] = {T(0), T(0), T(0), T(0)};
      auto rows = [&](int i0, int i1) {
        for (int i = i0 + ls; i < i1; i += LS) {
          const T xa = ra[i], xb = rb[i];
          const TT* w = ax.W + i * nw + k0;
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (k0 + k < nw) {
              const TT wk = ldg(w + k);
              sa[k] = fma(wk, xa, sa[k]);
              sb[k] = fma(wk, xb, sb[k]);
            }
        }
      };
      rows(0, ax.wlo);
      rows(ax.whi, m);
      // the lane sums of the (up to) 2 x 4 columns, reduced and scattered
      // over the group's lanes in one set of exchanges (double-float and
      // FP64, where an exchange and a sum cost several instructions); FP32,
      // paired or not, sums every column over the group (measured faster
      // there, and the paired pass keeps the unpaired order)
      if constexpr (std::is_same<TT, float>::value) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (k0 + k < nw) {
            const T ya = group_sum<LS>(sa[k]), yb = group_sum<LS>(sb[k]);
            if (ls == 0) {
              ova[k0 + k] = ya;
              ovb[k0 + k] = yb;
            }
          }
      } else if (nw - k0 <= 2) {
        T v[4] = {sa[0], sa[1], sb[0], sb[1]};
        const T y = group_sum_scatter<LS, 4>(v, ls);
        constexpr int S = LS / 4;
        const int j = ls / S, k = j & 1;
        if (ls % S == 0 && k0 + k < nw) (j < 2 ? ova : ovb)[k0 + k] = y;
      } else {
        T v[8] = {sa[0], sa[1], sa[2], sa[3], sb[0], sb[1], sb[2], sb[3]};
        const T y = group_sum_scatter<LS, 8>(v, ls);
        constexpr int S = LS / 8;
        const int j = ls / S, k = j & 3;
        if (ls % S == 0 && k0 + k < nw) (j < 4 ? ova : ovb)[k0 + k] = y;
      }
    }
    // Makhoul order of u_i = (-1)^i y_i, y = V_reg^T r, as the first stage's
    // input: element l = j + q N/8 lies in the first half exactly when q < 4.
    // Without interior blocks (and with at most 4 edge functions per lane) the
    // edge values y_i (i < nL, i >= N - nR) are computed first and stored
    // in the rows an identity column would use, row i + o: those rows belong to
    // no other column and have been read already (by the edge dot products and
    // W^T r), so the gather below is one branch-free read per element.
    const int ne = ax.nL + ax.nR;
    const bool uniform = ax.nblk == 0 && 2 * ne <= 4 * LS;
    if (uniform) {
      // every lane reads its (at most 4) edge values before any lane writes
      T ev[4];
      int slot[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int t = ls + r * LS;
        slot[r] = -1;
        ev[r] = T(0);
        if (t < 2 * ne) {
          const int c = t < ne ? t : t - ne;
          const int i = c < ax.nL ? c : NR - ax.nR + (c - ax.nL);
          ev[r] = reg_gather(t < ne ? ra : rb, i, ax);
          slot[r] = (t < ne ? 0 : ldt) + i + ax.o;
        }
      }
      __syncwarp();
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (slot[r] >= 0) ra[slot[r]] = ev[r];
      __syncwarp();
    }
    if constexpr (KIND == 1) {
      wstage_first<T, N>(buf, ls, [&](int j, int q) {
        const int l = j + q * (N / 8);
        const bool hi = q >= 4;
        const int i = hi ? 2 * (N - 1 - l) + 1 : 2 * l;
        T ya, yb;
        if (uniform) {
          ya = ra[i + ax.o];
          yb = rb[i + ax.o];
        } else {
          ya = reg_gather(ra, i, ax);
          yb = reg_gather(rb, i, ax);
        }
        return Cplx<T>{neg_if(ya, hi), neg_if(yb, hi)};
      });
      wfft_rest<T, N>(buf, ls, wt);
      // separation, twiddle and D~^{-1}: outputs N-1-k and k-1 from Z[k], Z[N-k]
      if constexpr (ALIAS) {
        constexpr int US = (N / 2 + LS) / LS;  // k = ls + LS u <= N / 2
        T o1a[US], o1b[US], o2a[US], o2b[US];
        auto put = [&](int u) {
          const int k = ls + LS * u;
          ra[N - 1 - k] = o1a[u];
          rb[N - 1 - k] = o1b[u];
          if (k > 0 && 2 * k != N) {
            ra[k - 1] = o2a[u];
            rb[k - 1] = o2b[u];
          }
        };
#pragma unroll
        for (int u = 0; u < US; ++u) {
          const int k = ls + LS * u;
          if (k <= N / 2) {
            const Cplx<T> zk = wld<T>(buf, wpad(k));
            const Cplx<T> zm = wld<T>(buf, wpad(k == 0 ? 0 : N - k));
            const T Ar = zk.x + zm.x, Ai = zk.y - zm.y;
            const T Br = zk.y + zm.y, Bi = zm.x - zk.x;
            const Post4<TT> t = ldpost(ax.post, k);
            o1a[u] = dot2(t.x, Ar, t.y, Ai);
            o1b[u] = dot2(t.x, Br, t.y, Bi);
            o2a[u] = dot2(t.z, Ar, -t.w, Ai);
            o2b[u] = dot2(t.z, Br, -t.w, Bi);
                    }
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < US; ++u)
          if (ls + LS * u <= N / 2) put(u);
      } else {
        for (int k = ls; k <= N / 2; k += LS) {
          const Cplx<T> zk = wld<T>(buf, wpad(k));
          const Cplx<T> zm = wld<T>(buf, wpad(k == 0 ? 0 : N - k));
          const T Ar = zk.x + zm.x, Ai = zk.y - zm.y;
          const T Br = zk.y + zm.y, Bi = zm.x - zk.x;
          const Post4<TT> t = ldpost(ax.post, k);
          ra[N - 1 - k] = dot2(t.x, Ar, t.y, Ai);
          rb[N - 1 - k] = dot2(t.x, Br, t.y, Bi);
          if (k > 0 && 2 * k != N) {
            ra[k - 1] = dot2(t.z, Ar, -t.w, Ai);
            rb[k - 1] = dot2(t.z, Br, -t.w, Bi);
          }
        }
      }
    } else {
      // odd extension of length N = 2n: 0, y_0 .. y_{n-2}, 0, -y_{n-2} .. -y_0;
      // element l = j + q N/8 is in the second half exactly when q >= 4, and
      // the zeros are l = 0 and l = n (j = 0 with q = 0 or 4)
      wstage_first<T, N>(buf, ls, [&](int j, int q) {
        const int l = j + q * (N / 8);
        const bool hi = q >= 4;
        const int i = hi ? N - 1 - l : l - 1;
        T ya = T(0), yb = T(0);
        if (!((q == 0 || q == 4) && j == 0)) {
          if (uniform) {
            ya = ra[i + ax.o];
            yb = rb[i + ax.o];
          } else {
            ya = reg_gather(ra, i, ax);
            yb = reg_gather(rb, i, ax);
          }
        }
        return Cplx<T>{neg_if(ya, hi), neg_if(yb, hi)};
      });
      wfft_rest<T, N>(buf, ls, wt);
      // DST-I output j is -Im Z[j+1] (pencil a) and Re Z[j+1] (pencil b), times 1/(2 D~_j)
      if constexpr (ALIAS) {
        constexpr int UJ = (NR + LS - 1) / LS;
        T oa[UJ], ob[UJ];
#pragma unroll
        for (int u = 0; u < UJ; ++u) {
          const int j = ls + LS * u;
          if (j < NR) {
            const Cplx<T> z = wld<T>(buf, wpad(j + 1));
            const TT sc = ldg(ax.post + j);
            oa[u] = -sc * z.y;
            ob[u] = sc * z.x;
          }
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < UJ; ++u) {
          const int j = ls + LS * u;
          if (j < NR) {
            ra[j] = oa[u];
            rb[j] = ob[u];
          }
        }
      } else {
        for (int j = ls; j < NR; j += LS) {
          const Cplx<T> z = wld<T>(buf, wpad(j + 1));
          const TT sc = ldg(ax.post + j);
          ra[j] = -sc * z.y;
          rb[j] = sc * z.x;
        }
      }
    }
    __syncwarp();
    for (int k = ls; k < nw; k += LS) {
      ra[NR + k] = ova[k];
      rb[NR + k] = ovb[k];
    }
    __syncwarp();
  }

  if constexpr (MODE == PM_FUSED) {
    // divide by the summed eigenvalues of all directions
    const int pa = 2 * pr, pb = pa + 1;  // rows of the tile
    const T la = row_lam<T>(lamA, pia, pa), lb = row_lam<T>(lamA, pia, pb);
    const T ma = (dims.d == 3) ? row_lam<T>(lamB, pib, pa) : T(0);
    const T mb = (dims.d == 3) ? row_lam<T>(lamB, pib, pb) : T(0);
    for (int i = ls; i < m; i += LS) {
      const TT li = ldg(ax.lam + i);
      T da = li + la, db = li + lb;
      if (dims.d == 3) {
        da += ma;
        db += mb;
      }
      ra[i] = ra[i] / da;
      rb[i] = rb[i] / db;
    }
    __syncwarp();
  }

  if constexpr (MODE == PM_BWD || MODE == PM_FUSED) {
    for (int k = ls; k < nw; k += LS) {
      ova[k] = ra[NR + k];
      ovb[k] = rb[NR + k];
    }
    if constexpr (KIND == 1) {
      // inverse of the separation: G[k], G[N-k] from rows N-1-k and k-1
      if constexpr (ALIAS) {
        constexpr int US = (N / 2 + LS) / LS;
        vec2_t<T> g1[US], g2[US];
        auto put = [&](int u) {
          const int k = ls + LS * u;
          buf[wpad(k)] = g1[u];
          if (k != 0 && 2 * k != N) buf[wpad(N - k)] = g2[u];
        };
#pragma unroll
        for (int u = 0; u < US; ++u) {
          const int k = ls + LS * u;
          if (k <= N / 2) {
            const Post4<TT> t = ldpost(ax.post, k);
            if (k == 0 || 2 * k == N) {
              const TT s = t.x + t.x;
              g1[u] = vec2_t<T>{s * ra[N - 1 - k], s * rb[N - 1 - k]};
            } else {
              const T ar = dot2(t.x, ra[N - 1 - k], t.z, ra[k - 1]);
              const T ai = dot2(-t.y, ra[N - 1 - k], t.w, ra[k - 1]);
              const T br = dot2(t.x, rb[N - 1 - k], t.z, rb[k - 1]);
              const T bi = dot2(-t.y, rb[N - 1 - k], t.w, rb[k - 1]);
              g1[u] = vec2_t<T>{ar - bi, ai + br};
              g2[u] = vec2_t<T>{ar + bi, br - ai};
            }
          }
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < US; ++u)
          if (ls + LS * u <= N / 2) put(u);
      } else {
        for (int k = ls; k <= N / 2; k += LS) {
          const Post4<TT> t = ldpost(ax.post, k);
          if (k == 0 || 2 * k == N) {
            const TT s = t.x + t.x;
            buf[wpad(k)] = vec2_t<T>{s * ra[N - 1 - k], s * rb[N - 1 - k]};
          } else {
            const T ar = dot2(t.x, ra[N - 1 - k], t.z, ra[k - 1]);
            const T ai = dot2(-t.y, ra[N - 1 - k], t.w, ra[k - 1]);
            const T br = dot2(t.x, rb[N - 1 - k], t.z, rb[k - 1]);
            const T bi = dot2(-t.y, rb[N - 1 - k], t.w, rb[k - 1]);
            buf[wpad(k)] = vec2_t<T>{ar - bi, ai + br};
            buf[wpad(N - k)] = vec2_t<T>{ar + bi, br - ai};
          }
        }
      }
    } else {
      // odd extension of the scaled input w_j / (2 D~_j)
      if constexpr (ALIAS) {
        constexpr int UL = N / LS;
        vec2_t<T> gv[UL];
#pragma unroll
        for (int u = 0; u < UL; ++u) {
          const int l = ls + LS * u;
          T va = T(0), vb = T(0);
          if (l != 0 && l != N / 2) {
            const int jj = (l < N / 2) ? l - 1 : N - 1 - l;
            const TT sc = (l < N / 2) ? ldg(ax.post + jj) : -ldg(ax.post + jj);
            va = sc * ra[jj];
            vb = sc * rb[jj];
          }
          gv[u] = vec2_t<T>{va, vb};
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < UL; ++u) buf[wpad(ls + LS * u)] = gv[u];
      } else {
        for (int l = ls; l < N; l += LS) {
          T va = T(0), vb = T(0);
          if (l != 0 && l != N / 2) {
            const int jj = (l < N / 2) ? l - 1 : N - 1 - l;
            const TT sc = (l < N / 2) ? ldg(ax.post + jj) : -ldg(ax.post + jj);
            va = sc * ra[jj];
            vb = sc * rb[jj];
          }
          buf[wpad(l)] = vec2_t<T>{va, vb};
        }
      }
    }
    __syncwarp();
    wstage<T, N, 8, 1>(buf, ls, wt);
    wfft_rest<T, N>(buf, ls, wt);
    // x = V_reg w + W z_out, row by row (DST-III output j is +-Re/Im Z[l(j)];
    // DST-I output j is -Im Z[j+1] / Re Z[j+1]); with ALIAS all rows of the
    // lane are formed from the buffer before any is written (m <= N + kMaxNout)
    auto wa = [&](int j) {
      if constexpr (KIND == 1) {
        const int l = (j & 1) ? N - 1 - (j >> 1) : (j >> 1);
        return neg_if(buf[wpad(l)].x, j & 1);
      } else {
        return -buf[wpad(j + 1)].y;
      }
    };
    auto wb = [&](int j) {
      if constexpr (KIND == 1) {
        const int l = (j & 1) ? N - 1 - (j >> 1) : (j >> 1);
        return neg_if(buf[wpad(l)].y, j & 1);
      } else {
        return buf[wpad(j + 1)].x;
      }
    };
    if constexpr (ALIAS) {
      constexpr int UO = (N + kMaxNout + LS - 1) / LS;
      T xs[UO][2];
#pragma unroll
      for (int u = 0; u < UO; ++u) {
        const int i = ls + LS * u;
        if (i >= m) break;
        T xa, xb;
        if (ax.nblk == 0 && i >= ax.rowsL && i < m - ax.rowsR) {  // identity rows
          xa = wa(i - ax.o);
          xb = wb(i - ax.o);
        } else {
          xa = wscatter_row<T>(i, ax, wa);
          xb = wscatter_row<T>(i, ax, wb);
        }
        if (i < ax.wlo || i >= ax.whi) {
          for (int k = 0; k < nw; ++k) {
            const TT w = ldg(ax.W + i * nw + k);
            xa = fma(w, ova[k], xa);
            xb = fma(w, ovb[k], xb);
          }
        }
        xs[u][0] = xa;
        xs[u][1] = xb;
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < UO; ++u) {
        const int i = ls + LS * u;
        if (i >= m) break;
        ra[i] = xs[u][0];
        rb[i] = xs[u][1];
      }
    } else {
      for (int i = ls; i < m; i += LS) {
        T xa, xb;
        if (ax.nblk == 0 && i >= ax.rowsL && i < m - ax.rowsR) {  // identity rows
          xa = wa(i - ax.o);
          xb = wb(i - ax.o);
        } else {
          xa = wscatter_row<T>(i, ax, wa);
          xb = wscatter_row<T>(i, ax, wb);
        }
        if (i < ax.wlo || i >= ax.whi) {
          for (int k = 0; k < nw; ++k) {
            const TT w = ldg(ax.W + i * nw + k);
            xa = fma(w, ova[k], xa);
            xb = fma(w, ovb[k], xb);
          }
        }
        ra[i] = xa;
        rb[i] = xb;
      }
    }
  }
}

template <int N, typename T, typename Tout, int NDOT>
__device__ __forceinline__ void wstore_tile(const T* tile, Tout* __restrict__ out, int axis, int ldt,
                                            const AxisTab<T>& ax, const long long* pbase, const TileInfo& g,
                                            const double* __restrict__ dotv0, const double* __restrict__ dotv1,
                                            double* __restrict__ partial, int ptile, int pstride) {
  constexpr int PP = warp_pencils<N>();
  const int m = ax.m;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // ---- coalesced store (and the partial dot products of a PCG step)
  double d0 = 0.0, d1 = 0.0;
  constexpr int kW = kThreads / 32, kIPR = (N + kMaxNout + 31) / 32;  // rows of a warp: PP / kW
  constexpr bool kPrefetch = NDOT == 1 && !std::is_same<tab_t<T>, float>::value && (PP / kW) * kIPR <= 20;
  if constexpr (kPrefetch) {
    if (axis == 0) {
      // double-float and FP64 (lengths 128, 256): every value of the dot
      // vector this thread needs is loaded first (all in flight at once),
      // then the store and the dot product run in the same order as below
      constexpr int W = kW, RPW = PP / W, IPR = kIPR;
      double rv[RPW][IPR];
#pragma unroll
      for (int r = 0; r < RPW; ++r) {
        const int pc = warp + r * W;
        const long long off = pbase[pc];
#pragma unroll
        for (int u = 0; u < IPR; ++u) {
          const int i = lane + 32 * u;
          rv[r][u] = (pc < g.nvalid && i < m) ? ldg(dotv0 + off + i) : 0.0;
        }
      }
#pragma unroll
      for (int r = 0; r < RPW; ++r) {
        const int pc = warp + r * W;
        if (pc < g.nvalid) {
          const T* row = tile + pc * ldt;
          Tout* dst = out + pbase[pc];
#pragma unroll
          for (int u = 0; u < IPR; ++u) {
            const int i = lane + 32 * u;
            if (i < m) {
              const Tout v = cvt<Tout>(row[i]);
              dst[i] = v;
              d0 = fma(rv[r][u], cvt<double>(v), d0);
            }
          }
        }
      }
    }
  }
  if (kPrefetch && axis == 0) {
    // stored above
  } else if (axis == 0) {
    for (int pc = warp; pc < g.nvalid; pc += kThreads / 32) {
      const T* row = tile + pc * ldt;
      Tout* dst = out + pbase[pc];
      const long long off0 = pbase[pc];
      for (int i = lane; i < m; i += 32) {
        const Tout v = cvt<Tout>(row[i]);
        dst[i] = v;
        if (NDOT >= 1) d0 = fma(ldg(dotv0 + off0 + i), cvt<double>(v), d0);
        if (NDOT >= 2) d1 = fma(ldg(dotv1 + off0 + i), cvt<double>(v), d1);
      }
    }
  } else {
    constexpr int RS = kThreads / PP;
    const int pc = tid & (PP - 1);
    if (pc < g.nvalid) {
      const long long step = g.S * RS;
      int i = tid / PP;
      long long off = pbase[pc] + i * g.S;
      for (; i < m; i += RS, off += step) {
        const Tout v = cvt<Tout>(tile[pc * ldt + i]);
        out[off] = v;
        if (NDOT >= 1) d0 = fma(ldg(dotv0 + off), cvt<double>(v), d0);
        if (NDOT >= 2) d1 = fma(ldg(dotv1 + off), cvt<double>(v), d1);
      }
    }
  }
  if (NDOT >= 1) {
    __shared__ double red[2][kThreads / 32];
    d0 = warp_sum(d0);
    d1 = warp_sum(d1);
    if (lane == 0) {
      red[0][warp] = d0;
      red[1][warp] = d1;
    }
    __syncthreads();
    if (tid == 0) {
      double s0 = 0.0, s1 = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) {
        s0 += red[0][w];
        s1 += red[1][w];
      }
      partial[ptile] = s0;
      if (NDOT >= 2) partial[pstride + ptile] = s1;
    }
  }
}

// Tile load and store of the paired pass: tile row r (f2) holds pencils
// row_pencil(r) and row_pencil(r) + 2. Along direction 0 a warp reads the two
// pencil rows of a tile row; along the others a thread moves four adjacent
// pencils of one grid line (one 16- or two 8-byte accesses where they are
// contiguous and aligned in memory), the CTA covering 256 / (PP / 4) lines
// per sweep.
template <int N, typename Tin>
__device__ __forceinline__ void wload_tile_pair(const Tin* __restrict__ in, f2* tile, int axis, int ldt, int m,
                                                const long long* pbase, const TileInfo& g) {
  constexpr int PP = warp_pencils<N, true>(), PR = PP / 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (axis == 0) {
    for (int r = warp; r < PR; r += kThreads / 32) {
      const int pa = row_pencil<f2>(r), pb = pa + 2;
      const bool va = pa < g.nvalid, vb = pb < g.nvalid;
      const Tin* sa = in + pbase[pa];
      const Tin* sb = in + pbase[pb];
      f2* row = tile + r * ldt;
#pragma unroll 4
      for (int i = lane; i < m; i += 32)
        row[i] = f2{va ? cvt<float>(sa[i]) : 0.f, vb ? cvt<float>(sb[i]) : 0.f};
    }
  } else {
    constexpr int QU = PP / 4, RS = kThreads / QU;  // pencil quads, lines per sweep
    const int qu = tid % QU;
    const int p0 = 4 * qu;
    const long long b0 = pbase[p0];
    const bool full = p0 + 3 < g.nvalid && pbase[p0 + 3] == b0 + 3;  // four contiguous pencils
    int mode = 0;  // 0: element loads, 1: two 8-byte loads, 2: one 16-byte load
    if constexpr (std::is_same<Tin, float>::value) {
      const uintptr_t a0 = reinterpret_cast<uintptr_t>(in + b0), sb = (uintptr_t)g.S * sizeof(float);
      if (full && (a0 % 16) == 0 && (sb % 16) == 0) mode = 2;
      else if (full && (a0 % 8) == 0 && (sb % 8) == 0) mode = 1;
    }
    bool v[4];
    const Tin* src[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = p0 + k < g.nvalid;
      src[k] = in + pbase[p0 + k];
    }
    f2* ra = tile + (2 * qu) * ldt;  // pencils p0, p0 + 2
    f2* rb = ra + ldt;               // pencils p0 + 1, p0 + 3
    for (int i = tid / QU; i < m; i += RS) {
      const long long o = (long long)i * g.S;
      float x0, x1, x2, x3;
      if constexpr (std::is_same<Tin, float>::value) {
        if (mode == 2) {
          const float4 t = *reinterpret_cast<const float4*>(src[0] + o);
          x0 = t.x; x1 = t.y; x2 = t.z; x3 = t.w;
        } else if (mode == 1) {
          const float2 t0 = *reinterpret_cast<const float2*>(src[0] + o);
          const float2 t1 = *reinterpret_cast<const float2*>(src[0] + o + 2);
          x0 = t0.x; x1 = t0.y; x2 = t1.x; x3 = t1.y;
        } else {
          x0 = v[0] ? src[0][o] : 0.f;
          x1 = v[1] ? src[1][o] : 0.f;
          x2 = v[2] ? src[2][o] : 0.f;
          x3 = v[3] ? src[3][o] : 0.f;
        }
      } else {
        x0 = v[0] ? cvt<float>(src[0][o]) : 0.f;
        x1 = v[1] ? cvt<float>(src[1][o]) : 0.f;
        x2 = v[2] ? cvt<float>(src[2][o]) : 0.f;
        x3 = v[3] ? cvt<float>(src[3][o]) : 0.f;
      }
      ra[i] = f2{x0, x2};
      rb[i] = f2{x1, x3};
    }
  }
}

// Paired store. The partial dot products of a PCG step are formed per half
// tile (pencils 0..PP/2-1 and PP/2..PP-1) with the thread-to-element map and
// summation order of the unpaired pass on its tile of PP/2 pencils, and stored
// as partials 2 ptile and 2 ptile + 1: the same partials as the unpaired pass.
template <int N, typename Tout, int NDOT>
__device__ __forceinline__ void wstore_tile_pair(const f2* tile, Tout* __restrict__ out, int axis, int ldt, int m,
                                                 const long long* pbase, const TileInfo& g,
                                                 const double* __restrict__ dotv0, const double* __restrict__ dotv1,
                                                 double* __restrict__ partial, int ptile, int pstride) {
  constexpr int PP = warp_pencils<N, true>(), HP = PP / 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float* tf = reinterpret_cast<const float*>(tile);
  double d0[2] = {0.0, 0.0}, d1[2] = {0.0, 0.0};  // per half tile (indexed by constants only)
  if (axis == 0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int nv = min(max(g.nvalid - h * HP, 0), HP);
      for (int pc = warp; pc < nv; pc += kThreads / 32) {
        const int P = h * HP + pc;                           // pencil 4 s + k
        const int row = 2 * (P >> 2) + (P & 1), comp = (P >> 1) & 1;  // tile row, f2 component
        const float* src = tf + 2 * (long long)row * ldt + comp;
        Tout* dst = out + pbase[P];
        const long long off0 = pbase[P];
        for (int i = lane; i < m; i += 32) {
          const Tout v = cvt<Tout>(src[2 * i]);
          dst[i] = v;
          if (NDOT >= 1) d0[h] = fma(ldg(dotv0 + off0 + i), cvt<double>(v), d0[h]);
          if (NDOT >= 2) d1[h] = fma(ldg(dotv1 + off0 + i), cvt<double>(v), d1[h]);
        }
      }
    }
  } else {
    constexpr int QU = PP / 4, RS = kThreads / QU;
    const int qu = tid % QU;
    const int p0 = 4 * qu;
    const long long b0 = pbase[p0];
    const bool full = p0 + 3 < g.nvalid && pbase[p0 + 3] == b0 + 3;
    int mode = 0;
    if constexpr (std::is_same<Tout, float>::value) {
      const uintptr_t a0 = reinterpret_cast<uintptr_t>(out + b0), sb = (uintptr_t)g.S * sizeof(float);
      if (full && (a0 % 16) == 0 && (sb % 16) == 0) mode = 2;
      else if (full && (a0 % 8) == 0 && (sb % 8) == 0) mode = 1;
    }
    const f2* ra = tile + (2 * qu) * ldt;
    const f2* rb = ra + ldt;
    for (int i = tid / QU; i < m; i += RS) {
      const long long o = (long long)i * g.S;
      const f2 ya = ra[i], yb = rb[i];
      const float x[4] = {ya.a, yb.a, ya.b, yb.b};
      if constexpr (std::is_same<Tout, float>::value) {
        if (mode == 2) {
          *reinterpret_cast<float4*>(out + b0 + o) = float4{x[0], x[1], x[2], x[3]};
          continue;
        }
        if (mode == 1) {
          *reinterpret_cast<float2*>(out + b0 + o) = float2{x[0], x[1]};
          *reinterpret_cast<float2*>(out + b0 + o + 2) = float2{x[2], x[3]};
          continue;
        }
      }
      const bool hi = p0 >= HP;  // the four pencils lie in one half (HP is a multiple of 4)
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (p0 + k < g.nvalid) {
          const long long off = pbase[p0 + k] + o;
          const Tout v = cvt<Tout>(x[k]);
          out[off] = v;
          if (NDOT >= 1) {
            const double t = ldg(dotv0 + off);
            if (hi) d0[1] = fma(t, cvt<double>(v), d0[1]);
            else d0[0] = fma(t, cvt<double>(v), d0[0]);
          }
          if (NDOT >= 2) {
            const double t = ldg(dotv1 + off);
            if (hi) d1[1] = fma(t, cvt<double>(v), d1[1]);
            else d1[0] = fma(t, cvt<double>(v), d1[0]);
          }
        }
    }
  }
  if (NDOT >= 1) {
    __shared__ double red[2][2][kThreads / 32];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const double s0 = warp_sum(d0[h]), s1 = warp_sum(d1[h]);
      if (lane == 0) {
        red[h][0][warp] = s0;
        red[h][1][warp] = s1;
      }
    }
    __syncthreads();
    if (tid < 2) {
      double s0 = 0.0, s1 = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) {
        s0 += red[tid][0][w];
        s1 += red[tid][1][w];
      }
      partial[2 * ptile + tid] = s0;
      if (NDOT >= 2) partial[pstride + 2 * ptile + tid] = s1;
    }
  }
}

// FP64 FUSED passes divide by the summed eigenvalues between the forward and
// the backward transform as one block-wide step: a multiply with the
// precomputed reciprocal, read in the coalesced order of the tile load (the
// same product as the block kernel's), else a division.
template <int N>
__device__ __forceinline__ void wscale_tile(double* tile, int axis, int ldt, const AxisTab<double>& ax,
                                            const Dims& dims, const double* __restrict__ lamA,
                                            const double* __restrict__ lamB, const long long* pbase, const int* pia,
                                            const int* pib, const TileInfo& g) {
  constexpr int PP = warp_pencils<N>();
  const int m = ax.m;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (ax.rden == nullptr) {
    for (int e = tid; e < PP * m; e += kThreads) {
      const int pc = e / m, i = e - pc * m;
      if (pc >= g.nvalid) continue;
      double den = ldg(ax.lam + i) + ldg(lamA + pia[pc]);
      if (dims.d == 3) den += ldg(lamB + pib[pc]);
      tile[pc * ldt + i] = tile[pc * ldt + i] / den;
    }
  } else if (axis == 0) {
    for (int pc = warp; pc < g.nvalid; pc += kThreads / 32)
      for (int i = lane; i < m; i += 32) tile[pc * ldt + i] = tile[pc * ldt + i] * ldg(ax.rden + pbase[pc] + i);
  } else {
    constexpr int RS = kThreads / PP;
    const int pc = tid & (PP - 1);
    if (pc < g.nvalid)
      for (int i = tid / PP; i < m; i += RS)
        tile[pc * ldt + i] = tile[pc * ldt + i] * ldg(ax.rden + pbase[pc] + i * g.S);
  }
}

// Double-float FUSED passes: the same block-wide step, dividing by the summed
// eigenvalues through a double-float reciprocal formed on the fly (no
// per-DoF table is read): the eigenvalues of the other directions are summed
// once per pencil, then lam_i is added and the reciprocal refined by Newton.
template <int N>
__device__ __forceinline__ void wscale_tile_df(df* tile, int ldt, const AxisTab<df>& ax, const Dims& dims,
                                               const df* __restrict__ lamA, const df* __restrict__ lamB,
                                               const int* pia, const int* pib, const TileInfo& g) {
  const int m = ax.m;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int pc = warp; pc < g.nvalid; pc += kThreads / 32) {
    df lp = ldg(lamA + pia[pc]);
    if (dims.d == 3) lp = lp + ldg(lamB + pib[pc]);
    df* row = tile + pc * ldt;
    for (int i = lane; i < m; i += 32) row[i] = row[i] * recip(ldg(ax.lam + i) + lp);
  }
}

// The transform of one loaded tile, in place (FWD, BWD, or both with the
// eigenvalue scaling between them), by the whole CTA.
template <typename T, int N, int KIND, int MODE>
__device__ __forceinline__ void wcompute(T* tile, vec2_t<T>* wbuf, T* outv, const Dims& dims, int axis, int ldt,
                                         const AxisTab<tab_t<T>>& ax, const vec2_t<tab_t<T>>* __restrict__ wt,
                                         const tab_t<T>* __restrict__ lamA, const tab_t<T>* __restrict__ lamB,
                                         const long long* pbase, const int* pia, const int* pib, const TileInfo& g) {
  if constexpr (std::is_same<T, double>::value && MODE == PM_FUSED) {
    wtransform<T, N, KIND, PM_FWD, walias<T>()>(tile, wbuf, outv, dims, ldt, ax, wt, lamA, lamB, pia, pib);
    __syncthreads();
    wscale_tile<N>(tile, axis, ldt, ax, dims, lamA, lamB, pbase, pia, pib, g);
    __syncthreads();
    wtransform<T, N, KIND, PM_BWD, walias<T>()>(tile, wbuf, outv, dims, ldt, ax, wt, lamA, lamB, pia, pib);
  } else if constexpr (std::is_same<T, df>::value && MODE == PM_FUSED) {
    wtransform<T, N, KIND, PM_FWD, walias<T>()>(tile, wbuf, outv, dims, ldt, ax, wt, lamA, lamB, pia, pib);
    __syncthreads();
    wscale_tile_df<N>(tile, ldt, ax, dims, lamA, lamB, pia, pib, g);
    __syncthreads();
    wtransform<T, N, KIND, PM_BWD, walias<T>()>(tile, wbuf, outv, dims, ldt, ax, wt, lamA, lamB, pia, pib);
  } else {
    wtransform<T, N, KIND, MODE, walias<T>()>(tile, wbuf, outv, dims, ldt, ax, wt, lamA, lamB, pia, pib);
  }
}

template <int N, typename T, typename Tout, int NDOT>
__device__ __forceinline__ void wstore_any(const T* tile, Tout* __restrict__ out, int axis, int ldt,
                                           const AxisTab<tab_t<T>>& ax, const long long* pbase, const TileInfo& g,
                                           const double* __restrict__ dotv0, const double* __restrict__ dotv1,
                                           double* __restrict__ partial, int ptile, int pstride) {
  if constexpr (IsPair<T>::value)
    wstore_tile_pair<N, Tout, NDOT>(tile, out, axis, ldt, ax.m, pbase, g, dotv0, dotv1, partial, ptile, pstride);
  else
    wstore_tile<N, T, Tout, NDOT>(tile, out, axis, ldt, ax, pbase, g, dotv0, dotv1, partial, ptile, pstride);
}

// One CTA: tile `tile_id` of PP = warp_pencils<N, pair>() pencils (T = f2:
// the paired pass, PP / 2 tile rows of two pencils each).
template <typename T, int N, int KIND, typename Tin, typename Tout, int MODE, int NDOT>
__device__ __forceinline__ void wpass_body(const Tin* __restrict__ in, Tout* __restrict__ out, const Dims& dims,
                                           int axis, int ldt, const AxisTab<tab_t<T>>& ax,
                                           const vec2_t<tab_t<T>>* __restrict__ wt,
                                           const tab_t<T>* __restrict__ lamA, const tab_t<T>* __restrict__ lamB,
                                           const double* __restrict__ dotv0, const double* __restrict__ dotv1,
                                           double* __restrict__ partial, long long tile_id, int ptile, int pstride,
                                           unsigned char* smem) {
  constexpr bool PAIR = IsPair<T>::value;
  constexpr int PP = warp_pencils<N, PAIR>(), PR = PAIR ? PP / 2 : PP;  // pencils, tile rows
  T* tile = reinterpret_cast<T*>(smem);  // PR rows of ldt values
  // sequence buffers inside the rows (walias) or after them
  vec2_t<T>* wbuf = walias<T>() ? nullptr : reinterpret_cast<vec2_t<T>*>(tile + (size_t)PR * ldt);
  T* outv = walias<T>() ? tile + (size_t)PR * ldt
                        : reinterpret_cast<T*>(wbuf + (size_t)(PR / 2) * wbuf_len<N>());  // PR * kMaxNout
  __shared__ long long pbase[PP];
  __shared__ int pia[PP], pib[PP];
  const TileInfo g = wtile_setup(dims, axis, PP, tile_id, pbase, pia, pib);
  __syncthreads();
  if constexpr (PAIR) wload_tile_pair<N, Tin>(in, tile, axis, ldt, ax.m, pbase, g);
  else wload_tile<N, T, Tin>(in, tile, axis, ldt, ax, pbase, g);
  __syncthreads();
  wcompute<T, N, KIND, MODE>(tile, wbuf, outv, dims, axis, ldt, ax, wt, lamA, lamB, pbase, pia, pib, g);
  __syncthreads();
  wstore_any<N, T, Tout, NDOT>(tile, out, axis, ldt, ax, pbase, g, dotv0, dotv1, partial, ptile, pstride);
}

template <typename T, int N, int KIND, typename Tin, typename Tout, int MODE, int NDOT>
__global__ void __launch_bounds__(kThreads)
precond_wpass(const Tin* in, Tout* out, Dims dims, int axis, int ldt, AxisTab<tab_t<T>> ax,
              const vec2_t<tab_t<T>>* wt, const tab_t<T>* __restrict__ lamA, const tab_t<T>* __restrict__ lamB,
              const double* __restrict__ dotv0, const double* __restrict__ dotv1, double* __restrict__ partial,
              const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  // the paired pass stores two partial sums per tile
  const int np = IsPair<T>::value ? 2 * gridDim.x : gridDim.x;
  wpass_body<T, N, KIND, Tin, Tout, MODE, NDOT>(in, out, dims, axis, ldt, ax, wt, lamA, lamB, dotv0, dotv1, partial,
                                                blockIdx.x, blockIdx.x, np, smem);
}

// Batched warp-FFT pass (FP32, T = float or the pair f2): every system of the
// launch runs the warp-FFT pass of length N (a separate kernel from the block
// one, so that neither carries the other's register allocation).
template <typename T, int N, int KIND, typename Tin, typename Tout, int MODE, int NDOT>
__global__ void __launch_bounds__(kThreads)
precond_wpass_batched(const PassDesc<float, Tin, Tout>* __restrict__ sys, const long long* __restrict__ tile_prefix,
                      int nsys) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ PassDesc<float, Tin, Tout> sd;
  __shared__ int s_sys;
  if (threadIdx.x == 0) {
    const long long b = blockIdx.x;
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {  // last s with tile_prefix[s] <= b
      const int mid = (lo + hi + 1) >> 1;
      if (tile_prefix[mid] <= b) lo = mid;
      else hi = mid - 1;
    }
    s_sys = lo;
    sd = sys[lo];
  }
  __syncthreads();
  if (sd.done != nullptr && *((volatile const int*)sd.done)) return;
  const long long tile = (long long)blockIdx.x - tile_prefix[s_sys];
  const int ntiles = (int)(tile_prefix[s_sys + 1] - tile_prefix[s_sys]);
  // the paired pass stores two partial sums per tile
  const int np = IsPair<T>::value ? 2 * ntiles : ntiles;
  wpass_body<T, N, KIND, Tin, Tout, MODE, NDOT>(sd.in, sd.out, sd.dims, sd.axis, sd.ldt, sd.ax, sd.wt, sd.lamA,
                                                sd.lamB, sd.dot0, sd.dot1, sd.partial, tile, (int)tile, np, smem);
}

// ---------------------------------------------------------------- launchers
template <typename T, int N, int KIND, typename Tin, typename Tout, int MODE, int NDOT>
cudaError_t launch_wpass_n(const PassLaunch<tab_t<T>>& P, const Tin* in, Tout* out, cudaStream_t st) {
  constexpr bool PAIR = IsPair<T>::value;
  const size_t sm = wpass_smem_bytes(N, P.ldt, sizeof(tab_t<T>), PAIR, walias<T>());
  const int tiles = precond_tiles(P.dims, P.axis, warp_pencils<N, PAIR>());
  auto kern = precond_wpass<T, N, KIND, Tin, Tout, MODE, NDOT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  kern<<<tiles, kThreads, sm, st>>>(in, out, P.dims, P.axis, P.ldt, P.ax, P.wt, P.lamA, P.lamB, P.dot0, P.dot1,
                                    P.partial, P.done);
  return cudaGetLastError();
}

template <typename T, int N, int KIND, typename Tin, typename Tout, int MODE, int NDOT>
cudaError_t launch_wbatched_t(const PassDesc<float, Tin, Tout>* sys, const long long* tile_prefix, int nsys,
                              long long total_tiles, size_t smem, cudaStream_t st) {
  auto kern = precond_wpass_batched<T, N, KIND, Tin, Tout, MODE, NDOT>;
  static size_t smem_set = 0;  // attribute is raised only when needed (not inside a graph capture)
  if (smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    smem_set = smem;
  }
  if (total_tiles <= 0) return cudaSuccess;
  kern<<<(unsigned)total_tiles, kThreads, smem, st>>>(sys, tile_prefix, nsys);
  return cudaGetLastError();
}

// Only the (arithmetic, input, output) type and mode combinations the
// preconditioners use exist: FP64 throughout (every mode, 0..2 dot products
// in backward passes); FP32 transforms with FP64 input (forward passes of the
// first direction), FP32 in and out (forward, fused and backward passes
// without dot products), FP64 output (backward passes of the first direction,
// 0..2 dot products).
template <typename Tc, typename Tin, typename Tout>
constexpr bool wpass_combo_ok(int mode, int ndot) {
  if (std::is_same<Tc, double>::value) return std::is_same<Tin, double>::value && std::is_same<Tout, double>::value;
  if (std::is_same<Tc, df>::value) {
    // double-float: FP64 in (forward passes of the first direction), FP64 out
    // (backward passes of the first direction, 0..2 dot products), df between
    if (std::is_same<Tin, double>::value) return mode == PM_FWD && std::is_same<Tout, df>::value;
    if (std::is_same<Tout, double>::value) return mode == PM_BWD;
    return ndot == 0;
  }
  if (std::is_same<Tin, double>::value) return mode == PM_FWD;
  if (std::is_same<Tout, double>::value) return mode == PM_BWD;
  return ndot == 0;
}

// The kernel of one (mode, dot count): transform kind 1 or 0, paired (FP32,
// N <= 256, P.pair set) or not.
template <typename Tc, int N, typename Tin, typename Tout, int MODE, int NDOT>
cudaError_t launch_wk(const PassLaunch<Tc>& P, const Tin* in, Tout* out, cudaStream_t st) {
  const bool k1 = P.ax.kind == 1;
  if constexpr (std::is_same<Tc, float>::value && N <= 256) {
    if (P.pair)
      return k1 ? launch_wpass_n<f2, N, 1, Tin, Tout, MODE, NDOT>(P, in, out, st)
                : launch_wpass_n<f2, N, 0, Tin, Tout, MODE, NDOT>(P, in, out, st);
  }
  if (P.pair) return cudaErrorInvalidValue;
  return k1 ? launch_wpass_n<Tc, N, 1, Tin, Tout, MODE, NDOT>(P, in, out, st)
            : launch_wpass_n<Tc, N, 0, Tin, Tout, MODE, NDOT>(P, in, out, st);
}

template <int N, typename Tc, typename Tin, typename Tout>
cudaError_t launch_wpass(const PassLaunch<Tc>& P, int mode, int ndot, const Tin* in, Tout* out, cudaStream_t st) {
  if (!wpass_combo_ok<Tc, Tin, Tout>(mode, ndot)) return cudaErrorInvalidValue;
#define IFFD_WL(MODE, NDOT) return launch_wk<Tc, N, Tin, Tout, MODE, NDOT>(P, in, out, st);
  if constexpr (std::is_same<Tc, double>::value) {
    if (mode == PM_FWD) { IFFD_WL(PM_FWD, 0) }
    if (mode == PM_FUSED) { IFFD_WL(PM_FUSED, 0) }
    if (ndot == 0) { IFFD_WL(PM_BWD, 0) }
    if (ndot == 1) { IFFD_WL(PM_BWD, 1) }
    IFFD_WL(PM_BWD, 2)
  } else if constexpr (std::is_same<Tin, double>::value) {
    IFFD_WL(PM_FWD, 0)
  } else if constexpr (std::is_same<Tout, double>::value) {
    if (ndot == 0) { IFFD_WL(PM_BWD, 0) }
    if (ndot == 1) { IFFD_WL(PM_BWD, 1) }
    IFFD_WL(PM_BWD, 2)
  } else {
    if (mode == PM_FWD) { IFFD_WL(PM_FWD, 0) }
    if (mode == PM_FUSED) { IFFD_WL(PM_FUSED, 0) }
    IFFD_WL(PM_BWD, 0)
  }
#undef IFFD_WL
}

template <int N, typename Tin, typename Tout, int MODE, int NDOT>
cudaError_t launch_wbk(const PassDesc<float, Tin, Tout>* sys, const long long* tile_prefix, int nsys,
                       long long total_tiles, size_t smem, int kind, int pair, cudaStream_t st) {
  const bool k1 = kind == 1;
  if constexpr (N <= 256) {
    if (pair)
      return k1 ? launch_wbatched_t<f2, N, 1, Tin, Tout, MODE, NDOT>(sys, tile_prefix, nsys, total_tiles, smem, st)
                : launch_wbatched_t<f2, N, 0, Tin, Tout, MODE, NDOT>(sys, tile_prefix, nsys, total_tiles, smem, st);
  }
  if (pair) return cudaErrorInvalidValue;
  return k1 ? launch_wbatched_t<float, N, 1, Tin, Tout, MODE, NDOT>(sys, tile_prefix, nsys, total_tiles, smem, st)
            : launch_wbatched_t<float, N, 0, Tin, Tout, MODE, NDOT>(sys, tile_prefix, nsys, total_tiles, smem, st);
}

template <int N, typename Tin, typename Tout>
cudaError_t launch_wpass_batched_n(const PassDesc<float, Tin, Tout>* sys, const long long* tile_prefix, int nsys,
                                   long long total_tiles, size_t smem, int kind, int pair, int mode, int ndot,
                                   cudaStream_t st) {
  if (!wpass_combo_ok<float, Tin, Tout>(mode, ndot)) return cudaErrorInvalidValue;
#define IFFD_WB(MODE, NDOT) \
  return launch_wbk<N, Tin, Tout, MODE, NDOT>(sys, tile_prefix, nsys, total_tiles, smem, kind, pair, st);
  if constexpr (std::is_same<Tin, double>::value) {
    IFFD_WB(PM_FWD, 0)
  } else if constexpr (std::is_same<Tout, double>::value) {
    if (ndot == 0) { IFFD_WB(PM_BWD, 0) }
    if (ndot == 1) { IFFD_WB(PM_BWD, 1) }
    IFFD_WB(PM_BWD, 2)
  } else {
    if (mode == PM_FWD) { IFFD_WB(PM_FWD, 0) }
    if (mode == PM_FUSED) { IFFD_WB(PM_FUSED, 0) }
    IFFD_WB(PM_BWD, 0)
  }
#undef IFFD_WB
}

// Explicit instantiation of one FFT length (one translation unit each, so
// that they compile in parallel): the FP32 passes and their batched forms,
// and (IFFD_WARP_INSTANTIATE_F64, lengths up to 256) the FP64 passes.
#define IFFD_WARP_INSTANTIATE(NN)                                                                              \
  template cudaError_t launch_wpass<NN, float, double, float>(const PassLaunch<float>&, int, int, const double*,  \
                                                              float*, cudaStream_t);                             \
  template cudaError_t launch_wpass<NN, float, float, float>(const PassLaunch<float>&, int, int, const float*,    \
                                                             float*, cudaStream_t);                              \
  template cudaError_t launch_wpass<NN, float, float, double>(const PassLaunch<float>&, int, int, const float*,   \
                                                              double*, cudaStream_t);                            \
  template cudaError_t launch_wpass_batched_n<NN, double, float>(const PassDesc<float, double, float>*,            \
                                                                 const long long*, int, long long, size_t, int,   \
                                                                 int, int, int, cudaStream_t);                         \
  template cudaError_t launch_wpass_batched_n<NN, float, float>(const PassDesc<float, float, float>*,              \
                                                                const long long*, int, long long, size_t, int,    \
                                                                int, int, int, cudaStream_t);                          \
  template cudaError_t launch_wpass_batched_n<NN, float, double>(const PassDesc<float, float, double>*,            \
                                                                 const long long*, int, long long, size_t, int,   \
                                                                 int, int, int, cudaStream_t);
#define IFFD_WARP_INSTANTIATE_F64(NN)                                                                             \
  template cudaError_t launch_wpass<NN, double, double, double>(const PassLaunch<double>&, int, int,               \
                                                                const double*, double*, cudaStream_t);
// Double-float passes (FP64-accurate transforms on the FP32 pipe), lengths up to 256.
#define IFFD_WARP_INSTANTIATE_DF(NN)                                                                                 \
  template cudaError_t launch_wpass<NN, df, double, df>(const PassLaunch<df>&, int, int, const double*, df*,          \
                                                        cudaStream_t);                                              \
  template cudaError_t launch_wpass<NN, df, df, df>(const PassLaunch<df>&, int, int, const df*, df*, cudaStream_t); \
  template cudaError_t launch_wpass<NN, df, df, double>(const PassLaunch<df>&, int, int, const df*, double*,         \
                                                        cudaStream_t);

}  // namespace iffd
