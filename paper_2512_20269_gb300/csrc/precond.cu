// IFFD preconditioner passes (eq. "preconditioner" of the paper):
//   P^{-1} r = (Q~_d x .. x Q~_1) (sum_k Lambda~_k)^{-1} (Q~_d^T x .. x Q~_1^T) r,
//   Q~ = [V_reg U_reg D~^{-1}, V_out Q_out]   (Sections 4 and 6).
//
// One kernel launch applies Q~^T (FWD), Q~ (BWD), or Q~^T, the eigenvalue
// scaling and Q~ (FUSED, used on the last direction) to every pencil along one
// direction. A CTA owns a tile of PP pencils: it loads them (coalesced along x)
// into shared memory and, per pencil pair, runs
//   FWD: remainder projections y_out = W^T r (W = V_out Q_out), the V_reg^T edge
//        gather, Makhoul's reordering, a two-for-one complex Stockham FFT of
//        length L and the separation / twiddle / D~^{-1} step, giving
//        [D~^{-1} U^T V_reg^T r | Q_out^T V_out^T r];
//   BWD: the transpose of the same steps (DST-III for even p, DST-I for odd p,
//        Table 1) followed by the V_reg edge scatter and the rank-n_out update
//        V_out Q_out z_out.
// All arithmetic is in Tc (double, or float for the reduced-precision
// transform variant); Tin/Tout are the global storage types.
#include <cuda_pipeline.h>

#include <algorithm>

#include <type_traits>

#include "device_common.cuh"
#include "kernels.h"
#include "precond_dev.cuh"
#include "precond_warp_geom.h"

namespace iffd {

template <typename T>
__device__ __forceinline__ void dft3(Cplx<T>* v) {
  const T c = T(-0.5);
  const T s = T(-0.86602540378443864676372317075293618347);  // -sin(2 pi / 3)
  const Cplx<T> t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
  const Cplx<T> y0 = cadd(v[0], t1);
  const Cplx<T> m1 = {fma(c, t1.x, v[0].x), fma(c, t1.y, v[0].y)};
  const Cplx<T> is = {-s * t2.y, s * t2.x};  // i * s * t2
  v[0] = y0;
  v[1] = cadd(m1, is);
  v[2] = csub(m1, is);
}

template <typename T>
__device__ __forceinline__ void dft5(Cplx<T>* v) {
  const T c1 = T(0.30901699437494742410229341718281905886);   // cos(2pi/5)
  const T c2 = T(-0.80901699437494742410229341718281905886);  // cos(4pi/5)
  const T s1 = T(0.95105651629515357211643933337938214340);   // sin(2pi/5)
  const T s2 = T(0.58778525229247312916870595463907276860);   // sin(4pi/5)
  const Cplx<T> t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  const Cplx<T> t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
  const Cplx<T> y0 = cadd(v[0], cadd(t1, t2));
  const Cplx<T> m1 = {fma(c2, t2.x, fma(c1, t1.x, v[0].x)), fma(c2, t2.y, fma(c1, t1.y, v[0].y))};
  const Cplx<T> m2 = {fma(c1, t2.x, fma(c2, t1.x, v[0].x)), fma(c1, t2.y, fma(c2, t1.y, v[0].y))};
  const Cplx<T> n1 = {fma(s2, t4.x, s1 * t3.x), fma(s2, t4.y, s1 * t3.y)};
  const Cplx<T> n2 = {fma(-s1, t4.x, s2 * t3.x), fma(-s1, t4.y, s2 * t3.y)};
  v[0] = y0;
  v[1] = cadd(m1, mul_mi(n1));
  v[4] = csub(m1, mul_mi(n1));
  v[2] = cadd(m2, mul_mi(n2));
  v[3] = csub(m2, mul_mi(n2));
}

template <typename T, int R>
__device__ __forceinline__ void butterfly(const Cplx<T>* in, Cplx<T>* out, int j, int k, int nb, int Ns,
                                          const T* tw) {
  Cplx<T> v[R];
#pragma unroll
  for (int q = 0; q < R; ++q) v[q] = in[j + q * nb];
  if (Ns > 1) {
#pragma unroll
    for (int q = 1; q < R; ++q) v[q] = cmul(v[q], ldc(tw + 2 * ((q - 1) * Ns + k)));
  }
  if constexpr (R == 2) dft2(v);
  else if constexpr (R == 3) dft3(v);
  else if constexpr (R == 4) dft4(v);
  else if constexpr (R == 5) dft5(v);
  else dft8(v);
  const int base = (j - k) * R + k;
#pragma unroll
  for (int t = 0; t < R; ++t) out[base + t * Ns] = v[t];
}

// Stockham autosort FFT of npairs independent length-F sequences stored
// contiguously in bufA; ping-pongs with bufB. Returns the buffer holding the
// natural-order result. Must be called by the whole CTA.
// Radices 8, 4, 2, 3, 5 run as register butterflies; any other factor r runs as
// a direct DFT stage in which each thread forms one output
//   y_t(j) = sum_q in[j + q nb] exp(-2 pi i q (k + t Ns) / (Ns r)),  k = j mod Ns,
// from a table of exp(-2 pi i s / (Ns r)), s < Ns r.
template <typename T>
__device__ Cplx<T>* fft_block(Cplx<T>* bufA, Cplx<T>* bufB, int npairs, const AxisTab<T>& ax) {
  const int L = ax.F;
  Cplx<T>* src = bufA;
  Cplx<T>* dst = bufB;
  int Ns = 1;
  for (int s = 0; s < ax.nst; ++s) {
    const int r = ax.radix[s];
    const int nb = L / r;
    const FastDiv fnb = ax.fnb[s], fNs = ax.fNs[s];
    const T* tw = ax.tw + 2 * ax.twoff[s];
    if (r == 8 || r == 4 || r == 2 || r == 3 || r == 5) {
      const int total = npairs * nb;
      for (int w = threadIdx.x; w < total; w += blockDim.x) {
        const int pr = fnb.div(w);
        const int j = w - pr * nb;
        const int k = fNs.mod(j);
        const Cplx<T>* in = src + (size_t)pr * L;
        Cplx<T>* out = dst + (size_t)pr * L;
        switch (r) {
          case 8: butterfly<T, 8>(in, out, j, k, nb, Ns, tw); break;
          case 4: butterfly<T, 4>(in, out, j, k, nb, Ns, tw); break;
          case 2: butterfly<T, 2>(in, out, j, k, nb, Ns, tw); break;
          case 3: butterfly<T, 3>(in, out, j, k, nb, Ns, tw); break;
          default: butterfly<T, 5>(in, out, j, k, nb, Ns, tw); break;
        }
      }
    } else {
      const int NsR = Ns * r;
      const int total = npairs * L;
      for (int w = threadIdx.x; w < total; w += blockDim.x) {
        const int pr = ax.fF.div(w);
        const int o = w - pr * L;
        const int t = fnb.div(o);
        const int j = o - t * nb;
        const int k = fNs.mod(j);
        const int step = k + t * Ns;
        const Cplx<T>* in = src + (size_t)pr * L;
        Cplx<T> acc = in[j];
        int e = 0;
        for (int q = 1; q < r; ++q) {
          e += step;
          if (e >= NsR) e -= NsR;
          const Cplx<T> a = in[j + q * nb];
          const Cplx<T> wv = ldc(tw + 2 * e);
          acc.x = fma(a.x, wv.x, fma(-a.y, wv.y, acc.x));
          acc.y = fma(a.x, wv.y, fma(a.y, wv.x, acc.y));
        }
        dst[(size_t)pr * L + (j - k) * r + k + t * Ns] = acc;
      }
    }
    __syncthreads();
    Cplx<T>* tmp = src;
    src = dst;
    dst = tmp;
    Ns *= r;
  }
  return src;
}

// Length-L forward DFT of npairs sequences (stride F in shared memory; entries
// j < L hold the data). Without Bluestein this is fft_block. With it (L has a
// large prime factor), jk = (j^2 + k^2 - (k-j)^2)/2 turns the DFT into the
// cyclic convolution of length F >= 2L-1
//   X_k = conj(c_k) sum_j (x_j conj(c_j)) c_{k-j},   c_j = exp(i pi j^2 / L),
// evaluated as two length-F FFTs: the inverse one through conjugation,
// IDFT(y) = conj(DFT(conj y)) / F, with 1/F folded into bhat = DFT_F(b) / F.
template <typename T>
__device__ Cplx<T>* dft_block(Cplx<T>* bufA, Cplx<T>* bufB, int npairs, const AxisTab<T>& ax) {
  if (!ax.blu) return fft_block(bufA, bufB, npairs, ax);
  const int L = ax.L, F = ax.F;
  for (int w = threadIdx.x; w < npairs * F; w += blockDim.x) {
    const int j = ax.fF.mod(w);
    Cplx<T> v = {T(0), T(0)};
    if (j < L) {  // a_j = x_j conj(c_j); zero padding beyond L
      const Cplx<T> x = bufA[w], c = ldc(ax.chirp + 2 * j);
      v = {fma(x.x, c.x, x.y * c.y), fma(x.y, c.x, -x.x * c.y)};
    }
    bufA[w] = v;
  }
  __syncthreads();
  Cplx<T>* R = fft_block(bufA, bufB, npairs, ax);
  for (int w = threadIdx.x; w < npairs * F; w += blockDim.x) {
    const Cplx<T> v = cmul(R[w], ldc(ax.bhat + 2 * ax.fF.mod(w)));
    R[w] = {v.x, -v.y};
  }
  __syncthreads();
  Cplx<T>* S = fft_block(R, R == bufA ? bufB : bufA, npairs, ax);
  for (int w = threadIdx.x; w < npairs * L; w += blockDim.x) {
    const int pr = ax.fL.div(w), k = w - pr * L;
    const Cplx<T> v = cmul(S[(size_t)pr * F + k], ldc(ax.chirp + 2 * k));
    S[(size_t)pr * F + k] = {v.x, -v.y};  // X_k = conj(c_k S_k)
  }
  __syncthreads();
  return S;
}

// Generic Table 1 transform (kind 2): output of frequency k of the two real
// pencils a (x) and b (y) packed in the length-L sequence Zp,
// T(k) = sum_l s_l exp(+2 pi i l k / L), times 2; Im(f T(k)) for the complex
// post factor f (which carries the 1/2 of the separation).
template <typename T>
__device__ __forceinline__ void gen_im(const Cplx<T>* Zp, int k, int L, T fx, T fy, T& ya, T& yb) {
  const Cplx<T> z1 = Zp[k == 0 ? 0 : L - k], z2 = Zp[k];
  const T tax = z1.x + z2.x, tay = z1.y - z2.y;  // 2 T_a(k)
  const T tbx = z1.y + z2.y, tby = z2.x - z1.x;  // 2 T_b(k)
  ya = fma(fx, tay, fy * tax);
  yb = fma(fx, tby, fy * tbx);
}


// A transform pass processes tiles of PP pencils along `axis` (tile_setup):
// load the tile into shared memory, transform it (compute_tile), store it.
// Partial dot products go to partial[ptile] (and partial[pstride + ptile]).

// Synchronous tile load (the caller synchronises afterwards).
template <typename Tc, typename Tin>
__device__ __forceinline__ void load_tile(const Tin* __restrict__ in, Tc* tile, int axis, int PP, int ldt,
                                          const AxisTab<Tc>& ax, const long long* pbase, const TileInfo& g) {
  const int lpp = 31 - __clz(PP);
  const int m = ax.m;
  const int tid = threadIdx.x;
  // ---- load the tile. Padding pencils are zero: two pencils share one complex
  // FFT, so a padding partner must not carry data (its rounding would leak into
  // the valid pencil, e.g. undivided values in the fused pass). Each thread
  // issues four independent global loads before its shared-memory stores, so
  // that enough loads are in flight to cover the DRAM latency.
  {
    constexpr int U = 4;
    const int total = PP * m;
    for (int e0 = tid; e0 < total; e0 += U * blockDim.x) {
      Tin v[U];
      int slot[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * blockDim.x;
        v[u] = Tin(0);
        slot[u] = -1;
        if (e < total) {
          int pc, i;
          if (axis == 0) { pc = ax.fm.div(e); i = e - pc * m; }
          else { i = e >> lpp; pc = e & (PP - 1); }
          slot[u] = pc * ldt + i;
          if (pc < g.nvalid) v[u] = in[pbase[pc] + i * g.S];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (slot[u] >= 0) tile[slot[u]] = (Tc)v[u];
    }
  }
}

// The transform of one loaded tile, in place in `tile` (bufA, bufB: FFT
// sequences; outv: remainder coefficients). Starts after and ends with a
// block-wide synchronisation.
template <typename Tc, int MODE>
__device__ __forceinline__ void compute_tile(Tc* tile, Cplx<Tc>* bufA, Cplx<Tc>* bufB, Tc* outv, const Dims& dims,
                                             int axis, int PP, int ldt, const AxisTab<Tc>& ax,
                                             const Tc* __restrict__ lamA, const Tc* __restrict__ lamB,
                                             const long long* pbase, const int* pia, const int* pib,
                                             const TileInfo& g) {
  const int npairs = PP / 2;
  const int lpp = 31 - __clz(PP);  // PP is a power of two
  const int L = ax.L;  // DFT length
  const int F = ax.F;  // stride of a sequence in shared memory
  const int m = ax.m;
  const int tid = threadIdx.x;
  const int N = ax.n_reg;
  if (MODE == PM_FWD || MODE == PM_FUSED) {
    // remainder projections y_out = W^T r over the two support ranges of W:
    // one group of 8 consecutive lanes per (pencil, column), reduced with three
    // shuffles. Every lane runs the same number of rounds (inactive groups add
    // zeros), so the full-warp shuffles never diverge.
    const int nw = ax.n_out;
    const int grp = tid >> 3, sub = tid & 7, ngrp = blockDim.x >> 3;
    for (int base = 0; base < PP * nw; base += ngrp) {
      const int job = base + grp;
      Tc acc = Tc(0);
      int pc = 0, k = 0;
      if (job < PP * nw) {
        pc = ax.fnout.div(job);
        k = job - pc * nw;
        const Tc* row = tile + pc * ldt;
        for (int i = sub; i < ax.wlo; i += 8) acc = fma(__ldg(ax.W + i * nw + k), row[i], acc);
        for (int i = ax.whi + sub; i < m; i += 8) acc = fma(__ldg(ax.W + i * nw + k), row[i], acc);
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 4);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      if (sub == 0 && job < PP * nw) outv[pc * kMaxNout + k] = acc;
    }
    // pack the regular part of two pencils into one complex sequence
    for (int w = tid; w < npairs * L; w += blockDim.x) {
      const int pr = ax.fL.div(w), l = w - pr * L;
      const Tc* ra = tile + (2 * pr) * ldt;
      const Tc* rb = ra + ldt;
      Tc va, vb;
      if (ax.kind == 1) {  // DST-II: Makhoul order of u_i = (-1)^i y_i
        const int i = (l < (N + 1) / 2) ? 2 * l : 2 * (N - 1 - l) + 1;
        va = neg_if(reg_gather(ra, i, ax), i & 1);
        vb = neg_if(reg_gather(rb, i, ax), i & 1);
      } else if (ax.kind == 2) {  // generic: y_reg at positions 1..N, zero padding
        if (l >= 1 && l <= N) { va = reg_gather(ra, l - 1, ax); vb = reg_gather(rb, l - 1, ax); }
        else { va = Tc(0); vb = Tc(0); }
      } else {  // DST-I: odd extension of length L = 2n
        const int n = N + 1;
        if (l == 0 || l == n) { va = Tc(0); vb = Tc(0); }
        else if (l < n) { va = reg_gather(ra, l - 1, ax); vb = reg_gather(rb, l - 1, ax); }
        else { va = neg_if(reg_gather(ra, 2 * n - 1 - l, ax), true); vb = neg_if(reg_gather(rb, 2 * n - 1 - l, ax), true); }
      }
      bufA[(size_t)pr * F + l] = {va, vb};
    }
    __syncthreads();
    const Cplx<Tc>* Z = dft_block(bufA, bufB, npairs, ax);
    if (ax.kind == 1) {
      const int K = N / 2 + 1;
      for (int w = tid; w < npairs * K; w += blockDim.x) {
        const int pr = ax.fK.div(w), k = w - pr * K;
        Tc* ra = tile + (2 * pr) * ldt;
        Tc* rb = ra + ldt;
        const Cplx<Tc> zk = Z[(size_t)pr * F + k];
        const Cplx<Tc> zm = Z[(size_t)pr * F + (k == 0 ? 0 : N - k)];
        const Tc Ar = zk.x + zm.x, Ai = zk.y - zm.y;
        const Tc Br = zk.y + zm.y, Bi = zm.x - zk.x;
        const Tc* t4 = ax.post + 4 * k;
        const Tc A = __ldg(t4), B = __ldg(t4 + 1), C = __ldg(t4 + 2), E = __ldg(t4 + 3);
        ra[N - 1 - k] = fma(A, Ar, B * Ai);
        rb[N - 1 - k] = fma(A, Br, B * Bi);
        if (k > 0 && 2 * k != N) {
          ra[k - 1] = fma(C, Ar, -E * Ai);
          rb[k - 1] = fma(C, Br, -E * Bi);
        }
      }
    } else if (ax.kind == 2) {
      for (int w = tid; w < npairs * N; w += blockDim.x) {
        const int pr = ax.fN.div(w), j = w - pr * N;
        Tc ya, yb;
        gen_im(Z + (size_t)pr * F, ax.gq * (j + 1) - ax.gqe, L, __ldg(ax.post + 2 * j), __ldg(ax.post + 2 * j + 1),
               ya, yb);
        tile[(2 * pr) * ldt + j] = ya;
        tile[(2 * pr + 1) * ldt + j] = yb;
      }
    } else {
      for (int w = tid; w < npairs * N; w += blockDim.x) {
        const int pr = ax.fN.div(w), j = w - pr * N;
        const Cplx<Tc> z = Z[(size_t)pr * F + j + 1];
        const Tc sc = __ldg(ax.post + j);
        tile[(2 * pr) * ldt + j] = -sc * z.y;
        tile[(2 * pr + 1) * ldt + j] = sc * z.x;
      }
    }
    for (int w = tid; w < PP * ax.n_out; w += blockDim.x) {
      const int pc = ax.fnout.div(w), k = w - pc * ax.n_out;
      tile[pc * ldt + N + k] = outv[pc * kMaxNout + k];
    }
    __syncthreads();
  }

  if (MODE == PM_FUSED) {
    // divide by the summed eigenvalues of all directions: by a multiply with
    // the precomputed reciprocal (FP64 plans; read in the coalesced order of
    // the tile load), else by a division
    if (ax.rden != nullptr) {
      for (int e = tid; e < PP * m; e += blockDim.x) {
        int pc, i;
        if (axis == 0) { pc = ax.fm.div(e); i = e - pc * m; }
        else { i = e >> lpp; pc = e & (PP - 1); }
        if (pc >= g.nvalid) continue;  // padding pencils
        tile[pc * ldt + i] = tile[pc * ldt + i] * (Tc)__ldg(ax.rden + pbase[pc] + i * g.S);
      }
    } else {
      for (int e = tid; e < PP * m; e += blockDim.x) {
        const int pc = ax.fm.div(e), i = e - pc * m;
        if (pc >= g.nvalid) continue;  // padding pencils
        Tc den = __ldg(ax.lam + i) + __ldg(lamA + pia[pc]);
        if (dims.d == 3) den += __ldg(lamB + pib[pc]);
        tile[pc * ldt + i] = tile[pc * ldt + i] / den;
      }
    }
    __syncthreads();
  }

  if (MODE == PM_BWD || MODE == PM_FUSED) {
    for (int w = tid; w < PP * ax.n_out; w += blockDim.x) {
      const int pc = ax.fnout.div(w), k = w - pc * ax.n_out;
      outv[pc * kMaxNout + k] = tile[pc * ldt + N + k];
    }
    if (ax.kind == 1) {
      const int K = N / 2 + 1;
      for (int w = tid; w < npairs * K; w += blockDim.x) {
        const int pr = ax.fK.div(w), k = w - pr * K;
        const Tc* za = tile + (2 * pr) * ldt;
        const Tc* zb = za + ldt;
        const Tc* t4 = ax.post + 4 * k;
        const Tc A = __ldg(t4), B = __ldg(t4 + 1), C = __ldg(t4 + 2), E = __ldg(t4 + 3);
        Cplx<Tc>* G = bufA + (size_t)pr * F;
        if (k == 0 || 2 * k == N) {
          const Tc s = A + A;
          G[k] = {s * za[N - 1 - k], s * zb[N - 1 - k]};
        } else {
          const Tc ar = fma(A, za[N - 1 - k], C * za[k - 1]);
          const Tc ai = fma(-B, za[N - 1 - k], E * za[k - 1]);
          const Tc br = fma(A, zb[N - 1 - k], C * zb[k - 1]);
          const Tc bi = fma(-B, zb[N - 1 - k], E * zb[k - 1]);
          G[k] = {ar - bi, ai + br};
          G[N - k] = {ar + bi, br - ai};
        }
      }
    } else if (ax.kind == 2) {
      for (int w = tid; w < npairs * L; w += blockDim.x) {
        const int pr = ax.fL.div(w), l = w - pr * L;
        const Tc* za = tile + (2 * pr) * ldt;
        const Tc* zb = za + ldt;
        Tc va = Tc(0), vb = Tc(0);
        if (l >= 1 && l <= N) {
          const Tc sc = __ldg(ax.post + 4 * N + l - 1);  // 1 / D~
          va = sc * za[l - 1];
          vb = sc * zb[l - 1];
        }
        bufA[(size_t)pr * F + l] = {va, vb};
      }
    } else {
      const int n = N + 1;
      for (int w = tid; w < npairs * L; w += blockDim.x) {
        const int pr = ax.fL.div(w), l = w - pr * L;
        const Tc* za = tile + (2 * pr) * ldt;
        const Tc* zb = za + ldt;
        Tc va, vb;
        if (l == 0 || l == n) { va = Tc(0); vb = Tc(0); }
        else if (l < n) {
          const Tc sc = __ldg(ax.post + l - 1);
          va = sc * za[l - 1];
          vb = sc * zb[l - 1];
        } else {
          const Tc sc = __ldg(ax.post + 2 * n - 1 - l);
          va = -sc * za[2 * n - 1 - l];
          vb = -sc * zb[2 * n - 1 - l];
        }
        bufA[(size_t)pr * F + l] = {va, vb};
      }
    }
    __syncthreads();
    const Cplx<Tc>* Z = dft_block(bufA, bufB, npairs, ax);
    // scatter: x = V_reg w + W z_out
    for (int e = tid; e < PP * m; e += blockDim.x) {
      const int pc = ax.fm.div(e), i = e - pc * m;
      const int pr = pc >> 1;
      const bool isb = pc & 1;
      const Cplx<Tc>* Zp = Z + (size_t)pr * F;
      auto wreg = [&](int j) -> Tc {
        if (ax.kind == 1) {
          const int l = (j & 1) ? N - 1 - (j >> 1) : (j >> 1);
          const Cplx<Tc> z = Zp[l];
          return neg_if(isb ? z.y : z.x, j & 1);
        } else if (ax.kind == 2) {
          Tc xa, xb;
          gen_im(Zp, ax.gq * (j + 1) - ax.gqc, L, __ldg(ax.post + 2 * N + 2 * j), __ldg(ax.post + 2 * N + 2 * j + 1),
                 xa, xb);
          return isb ? xb : xa;
        } else {
          const Cplx<Tc> z = Zp[j + 1];
          return isb ? z.x : -z.y;
        }
      };
      Tc x;
      if (i < ax.rowsL) {
        x = Tc(0);
        for (int c = 0; c < ax.nL; ++c) x = fma(__ldg(ax.VL + i * ax.nL + c), wreg(c), x);
      } else if (i >= m - ax.rowsR) {
        const int r = m - 1 - i;
        x = Tc(0);
        for (int c = 0; c < ax.nR; ++c) x = fma(__ldg(ax.VR + r * ax.nR + c), wreg(N - 1 - c), x);
      } else {
        int o = ax.o;
        bool inblk = false;
        for (int b = 0; b < ax.nblk; ++b) {  // interior blocks (repeated knots only)
          const int* B = ax.blk + 6 * b;
          const int r0 = __ldg(B + 2), r1 = __ldg(B + 3);
          if (i < r0) break;
          if (i < r1) {
            const int c0 = __ldg(B), c1 = __ldg(B + 1);
            const Tc* V = ax.VB + __ldg(B + 5) + (i - r0) * (c1 - c0);
            x = Tc(0);
            for (int c = c0; c < c1; ++c) x = fma(__ldg(V + (c - c0)), wreg(c), x);
            inblk = true;
            break;
          }
          o = __ldg(B + 4);
        }
        if (!inblk) x = wreg(i - o);
      }
      if (i < ax.wlo || i >= ax.whi) {
        for (int k = 0; k < ax.n_out; ++k) x = fma(__ldg(ax.W + i * ax.n_out + k), outv[pc * kMaxNout + k], x);
      }
      tile[pc * ldt + i] = x;
    }
    __syncthreads();
  }

}

// Store the tile (and the partial dot products of the last pass of a PCG step).
template <typename Tc, typename Tout, int NDOT>
__device__ __forceinline__ void store_tile(const Tc* tile, Tout* __restrict__ out, int axis, int PP, int ldt,
                                           const AxisTab<Tc>& ax, const long long* pbase, const TileInfo& g,
                                           const double* __restrict__ dotv0, const double* __restrict__ dotv1,
                                           double* __restrict__ partial, int ptile, int pstride) {
  const int lpp = 31 - __clz(PP);
  const int m = ax.m;
  const int tid = threadIdx.x;
  // ---- store (and, on the last pass of a PCG step, partial dot products)
  double d0 = 0.0, d1 = 0.0;
  for (int e = tid; e < PP * m; e += blockDim.x) {
    int pc, i;
    if (axis == 0) { pc = ax.fm.div(e); i = e - pc * m; }
    else { i = e >> lpp; pc = e & (PP - 1); }
    if (pc < g.nvalid) {
      const long long off = pbase[pc] + i * g.S;
      const Tc v = tile[pc * ldt + i];
      out[off] = (Tout)v;
      if (NDOT >= 1) d0 = fma(__ldg(dotv0 + off), (double)(Tout)v, d0);
      if (NDOT >= 2) d1 = fma(__ldg(dotv1 + off), (double)(Tout)v, d1);
    }
  }
  if (NDOT >= 1) {
    __shared__ double red[2][kThreads / 32];
    d0 = warp_sum(d0);
    d1 = warp_sum(d1);
    if ((tid & 31) == 0) { red[0][tid >> 5] = d0; red[1][tid >> 5] = d1; }
    __syncthreads();
    if (tid == 0) {
      double s0 = 0.0, s1 = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { s0 += red[0][w]; s1 += red[1][w]; }
      partial[ptile] = s0;
      if (NDOT >= 2) partial[pstride + ptile] = s1;
    }
  }
}

// Body of one CTA of a (non-persistent) transform pass: tile `tile_id`.
template <typename Tc, typename Tin, typename Tout, int MODE, int NDOT>
__device__ __forceinline__ void precond_body(const Tin* in, Tout* out, const Dims& dims, int axis, int PP, int ldt,
                                             const AxisTab<Tc>& ax, const Tc* __restrict__ lamA,
                                             const Tc* __restrict__ lamB, const double* __restrict__ dotv0,
                                             const double* __restrict__ dotv1, double* __restrict__ partial,
                                             long long tile_id, int ptile, int pstride, unsigned char* smem) {
  const int npairs = PP / 2;
  const int F = ax.F;
  Cplx<Tc>* bufA = reinterpret_cast<Cplx<Tc>*>(smem);
  Cplx<Tc>* bufB = bufA + (size_t)npairs * F;
  Tc* tile = reinterpret_cast<Tc*>(bufB + (size_t)npairs * F);
  Tc* outv = tile + (size_t)PP * ldt;  // PP * kMaxNout
  __shared__ long long pbase[64];
  __shared__ int pia[64], pib[64];
  const TileInfo g = tile_setup(dims, axis, PP, tile_id, pbase, pia, pib);
  __syncthreads();
  load_tile<Tc, Tin>(in, tile, axis, PP, ldt, ax, pbase, g);
  __syncthreads();
  compute_tile<Tc, MODE>(tile, bufA, bufB, outv, dims, axis, PP, ldt, ax, lamA, lamB, pbase, pia, pib, g);
  store_tile<Tc, Tout, NDOT>(tile, out, axis, PP, ldt, ax, pbase, g, dotv0, dotv1, partial, ptile, pstride);
}

template <typename Tc, typename Tin, typename Tout, int MODE, int NDOT>
__global__ void __launch_bounds__(kThreads)
precond_pass(const Tin* in, Tout* out, Dims dims, int axis, int PP, int ldt, AxisTab<Tc> ax,
             const Tc* __restrict__ lamA, const Tc* __restrict__ lamB,
             const double* __restrict__ dotv0, const double* __restrict__ dotv1,
             double* __restrict__ partial, const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  precond_body<Tc, Tin, Tout, MODE, NDOT>(in, out, dims, axis, PP, ldt, ax, lamA, lamB, dotv0, dotv1, partial,
                                          blockIdx.x, blockIdx.x, gridDim.x, smem);
}

// Asynchronous tile load: one cp.async element copy per DoF (padding pencils
// are written as zeros); the caller commits the copy group.
template <typename Tc>
__device__ __forceinline__ void load_tile_async(const Tc* __restrict__ in, Tc* tile, int axis, int PP, int ldt,
                                                const AxisTab<Tc>& ax, const long long* pbase, const TileInfo& g) {
  const int lpp = 31 - __clz(PP);
  const int m = ax.m;
  for (int e = threadIdx.x; e < PP * m; e += blockDim.x) {
    int pc, i;
    if (axis == 0) { pc = ax.fm.div(e); i = e - pc * m; }
    else { i = e >> lpp; pc = e & (PP - 1); }
    Tc* dst = tile + pc * ldt + i;
    if (pc < g.nvalid) __pipeline_memcpy_async(dst, in + pbase[pc] + i * g.S, sizeof(Tc));
    else *dst = Tc(0);
  }
}

// Persistent transform pass with a two-stage pipeline: each CTA walks the
// tiles t = blockIdx.x, + gridDim.x, ...; while it transforms tile t the
// copies of its next tile are already in flight into the second tile buffer.
// Same arithmetic and partial sums as precond_pass (only the loading differs).
template <typename Tc, int MODE, int NDOT>
__global__ void __launch_bounds__(kThreads)
precond_pass_pipe(const Tc* in, Tc* out, Dims dims, int axis, int PP, int ldt, AxisTab<Tc> ax,
                  const Tc* __restrict__ lamA, const Tc* __restrict__ lamB, const double* __restrict__ dotv0,
                  const double* __restrict__ dotv1, double* __restrict__ partial, int ntiles,
                  const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int npairs = PP / 2, F = ax.F;
  Cplx<Tc>* bufA = reinterpret_cast<Cplx<Tc>*>(smem);
  Cplx<Tc>* bufB = bufA + (size_t)npairs * F;
  Tc* tiles = reinterpret_cast<Tc*>(bufB + (size_t)npairs * F);  // two tile buffers
  Tc* outv = tiles + (size_t)2 * PP * ldt;                          // PP * kMaxNout
  __shared__ long long pbase[2][64];
  __shared__ int pia[2][64], pib[2][64];
  int t = blockIdx.x;
  if (t >= ntiles) return;  // the same for every thread of the CTA
  TileInfo g = tile_setup(dims, axis, PP, t, pbase[0], pia[0], pib[0]);
  __syncthreads();
  load_tile_async<Tc>(in, tiles, axis, PP, ldt, ax, pbase[0], g);
  __pipeline_commit();
  int cur = 0;
  for (; t < ntiles; t += gridDim.x) {
    const int tn = t + gridDim.x;
    const int nx = cur ^ 1;
    TileInfo gn = g;
    if (tn < ntiles) gn = tile_setup(dims, axis, PP, tn, pbase[nx], pia[nx], pib[nx]);
    __syncthreads();  // pbase[nx] written
    if (tn < ntiles) load_tile_async<Tc>(in, tiles + (size_t)nx * PP * ldt, axis, PP, ldt, ax, pbase[nx], gn);
    __pipeline_commit();
    __pipeline_wait_prior(1);  // this thread's copies of tile t have landed
    __syncthreads();           // and every thread's
    Tc* tile = tiles + (size_t)cur * PP * ldt;
    compute_tile<Tc, MODE>(tile, bufA, bufB, outv, dims, axis, PP, ldt, ax, lamA, lamB, pbase[cur], pia[cur],
                           pib[cur], g);
    store_tile<Tc, Tc, NDOT>(tile, out, axis, PP, ldt, ax, pbase[cur], g, dotv0, dotv1, partial, t, ntiles);
    __syncthreads();  // tile buffer and pbase of `cur` are free for tile t + 2 gridDim.x
    g = gn;
    cur = nx;
  }
  __pipeline_wait_prior(0);
}

// Batched pass: the grid covers the tiles of many independent systems; CTA b
// serves tile b - tile_prefix[s] of system s with tile_prefix[s] <= b <
// tile_prefix[s+1]. Each system's work and reductions are exactly those of the
// single-system kernel, so a result does not depend on the rest of the batch.
template <typename Tc, typename Tin, typename Tout, int MODE, int NDOT>
__global__ void __launch_bounds__(kThreads)
precond_pass_batched(const PassDesc<Tc, Tin, Tout>* __restrict__ sys, const long long* __restrict__ tile_prefix,
                     int nsys) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ PassDesc<Tc, Tin, Tout> sd;
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
  precond_body<Tc, Tin, Tout, MODE, NDOT>(sd.in, sd.out, sd.dims, sd.axis, sd.PP, sd.ldt, sd.ax, sd.lamA, sd.lamB,
                                          sd.dot0, sd.dot1, sd.partial, tile, (int)tile, ntiles, smem);
}

// rden[x + m0 (y + m1 z)] = 1 / (lam_F[i_F] + lam_0[x] (+ lam_1[y])): the
// reciprocal of the summed eigenvalues, added in the order of the FUSED pass
// (last direction F = d-1 first, then direction 0, then direction 1).
__global__ void rden_fill(double* __restrict__ rden, Dims dims, const double* __restrict__ lamF,
                          const double* __restrict__ lam0, const double* __restrict__ lam1) {
  const long long m0 = dims.m[0], m1 = dims.m[1];
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < dims.N;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long x = idx % m0, rest = idx / m0;
    double den;
    if (dims.d == 3) den = (__ldg(lamF + rest / m1) + __ldg(lam0 + x)) + __ldg(lam1 + rest % m1);
    else den = __ldg(lamF + rest) + __ldg(lam0 + x);
    rden[idx] = 1.0 / den;
  }
}

cudaError_t launch_rden_fill(double* rden, const Dims& dims, const double* lamF, const double* lam0,
                             const double* lam1, cudaStream_t st) {
  long long g = (dims.N + kThreads - 1) / kThreads;
  if (g > 8 * 152) g = 8 * 152;
  rden_fill<<<(unsigned)g, kThreads, 0, st>>>(rden, dims, lamF, lam0, lam1);
  return cudaGetLastError();
}

// ------------------------------------------------------------ host launchers
// F: FFT length (stride of a sequence); two ping-pong buffers of PP/2 complex
// sequences, the tile and the remainder coefficients.
size_t precond_smem_bytes(int PP, int ldt, int F, size_t elt) {
  return (size_t)2 * (PP / 2) * F * 2 * elt + (size_t)PP * ldt * elt + (size_t)PP * kMaxNout * elt;
}

int precond_tiles(const Dims& dims, int axis, int PP) { return (int)host_num_tiles(dims, axis, PP); }

static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 152;
  }
  return n;
}

size_t precond_smem_bytes_pipe(int PP, int ldt, int F, size_t elt) {
  return precond_smem_bytes(PP, ldt, F, elt) + (size_t)PP * ldt * elt;
}

template <typename Tc, int MODE, int NDOT>
static cudaError_t launch_pipe_t(const PassLaunch<Tc>& P, const Tc* in, Tc* out, cudaStream_t st) {
  auto kern = precond_pass_pipe<Tc, MODE, NDOT>;
  const size_t sm = precond_smem_bytes_pipe(P.PP, P.ldt, P.ax.F, sizeof(Tc));
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int tiles = precond_tiles(P.dims, P.axis, P.PP);
  const int grid = std::min(tiles, per_sm * sm_count());
  kern<<<grid, kThreads, sm, st>>>(in, out, P.dims, P.axis, P.PP, P.ldt, P.ax, P.lamA, P.lamB, P.dot0, P.dot1,
                                   P.partial, tiles, P.done);
  return cudaGetLastError();
}

template <typename T>
static int wpass_len_t(const AxisTab<T>& ax, int nmax) {
  int N = 0;
  if (ax.kind == 1) N = ax.n_reg;                 // DST-II/III: Makhoul, length n_reg
  else if (ax.kind == 0) N = 2 * (ax.n_reg + 1);  // DST-I: odd extension
  else return 0;
  if (ax.blu || ax.L != N || ax.F != N || N > nmax) return 0;
  return (N == 64 || N == 128 || N == 256 || N == 512) ? N : 0;
}
int wpass_len(const AxisTab<float>& ax) { return wpass_len_t(ax, 512); }
// FP64: a length-512 tile (141 KB of shared memory) would leave one CTA per SM
int wpass_len(const AxisTab<double>& ax) { return wpass_len_t(ax, 256); }
int wpass_len(const AxisTab<df>& ax) { return wpass_len_t(ax, 256); }

template <typename Tin, typename Tout>
cudaError_t launch_pass_df(const PassLaunch<df>& P, int mode, int ndot, const Tin* in, Tout* out, cudaStream_t st) {
  if (P.PP != wpass_pencils(P.wN) || P.ldt < P.ax.m) return cudaErrorInvalidConfiguration;
  switch (P.wN) {
    case 64: return launch_wpass<64, df, Tin, Tout>(P, mode, ndot, in, out, st);
    case 128: return launch_wpass<128, df, Tin, Tout>(P, mode, ndot, in, out, st);
    case 256: return launch_wpass<256, df, Tin, Tout>(P, mode, ndot, in, out, st);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_pass_df<double, df>(const PassLaunch<df>&, int, int, const double*, df*, cudaStream_t);
template cudaError_t launch_pass_df<df, df>(const PassLaunch<df>&, int, int, const df*, df*, cudaStream_t);
template cudaError_t launch_pass_df<df, double>(const PassLaunch<df>&, int, int, const df*, double*, cudaStream_t);

int wpass_pencils(int N) {
  switch (N) {
    case 64: return warp_pencils<64>();
    case 128: return warp_pencils<128>();
    case 256: return warp_pencils<256>();
    default: return warp_pencils<512>();
  }
}

size_t wpass_smem_bytes(int N, int ldt, size_t elt) {
  const int PP = wpass_pencils(N);
  return (size_t)PP * ldt * elt + (size_t)(PP / 2) * wpad(N) * 2 * elt + (size_t)PP * kMaxNout * elt;
}

template <typename Tc, typename Tin, typename Tout, int MODE, int NDOT>
cudaError_t launch_pass_t(const PassLaunch<Tc>& P, const Tin* in, Tout* out, cudaStream_t st) {
  if (P.wN != 0) {
    if (P.PP != wpass_pencils(P.wN) || P.ldt < P.ax.m) return cudaErrorInvalidConfiguration;
    switch (P.wN) {
      case 64: return launch_wpass<64, Tc, Tin, Tout>(P, MODE, NDOT, in, out, st);
      case 128: return launch_wpass<128, Tc, Tin, Tout>(P, MODE, NDOT, in, out, st);
      case 256: return launch_wpass<256, Tc, Tin, Tout>(P, MODE, NDOT, in, out, st);
      case 512:
        if constexpr (std::is_same<Tc, float>::value) return launch_wpass<512, Tc, Tin, Tout>(P, MODE, NDOT, in, out, st);
        else return cudaErrorInvalidValue;
      default: return cudaErrorInvalidValue;
    }
  }
  if constexpr (std::is_same<Tin, Tc>::value && std::is_same<Tout, Tc>::value) {
    if (P.pipe) return launch_pipe_t<Tc, MODE, NDOT>(P, in, out, st);
  }
  auto kern = precond_pass<Tc, Tin, Tout, MODE, NDOT>;
  const size_t sm = precond_smem_bytes(P.PP, P.ldt, P.ax.F, sizeof(Tc));
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int tiles = precond_tiles(P.dims, P.axis, P.PP);
  kern<<<tiles, kThreads, sm, st>>>(in, out, P.dims, P.axis, P.PP, P.ldt, P.ax, P.lamA, P.lamB, P.dot0,
                                     P.dot1, P.partial, P.done);
  return cudaGetLastError();
}

// Only the (arithmetic, input, output) type and mode combinations the
// preconditioners use are instantiated: FP64 throughout (every mode); FP32
// transforms with FP64 input (forward passes of the first direction), FP32
// in and out (forward, fused, backward without dot products), FP64 output
// (backward passes of the first direction, with 0..2 dot products).
template <typename Tc, typename Tin, typename Tout>
cudaError_t launch_pass(const PassLaunch<Tc>& P, int mode, int ndot, const Tin* in, Tout* out, cudaStream_t st) {
  constexpr bool in64 = std::is_same<Tc, float>::value && std::is_same<Tin, double>::value;
  constexpr bool out64 = std::is_same<Tc, float>::value && std::is_same<Tout, double>::value;
  constexpr bool f32 = std::is_same<Tc, float>::value && !in64 && !out64;
  if constexpr (in64) {
    if (mode != PM_FWD) return cudaErrorInvalidValue;
    return launch_pass_t<Tc, Tin, Tout, PM_FWD, 0>(P, in, out, st);
  } else if constexpr (out64) {
    if (mode != PM_BWD) return cudaErrorInvalidValue;
    if (ndot == 0) return launch_pass_t<Tc, Tin, Tout, PM_BWD, 0>(P, in, out, st);
    if (ndot == 1) return launch_pass_t<Tc, Tin, Tout, PM_BWD, 1>(P, in, out, st);
    return launch_pass_t<Tc, Tin, Tout, PM_BWD, 2>(P, in, out, st);
  } else if constexpr (f32) {
    if (ndot != 0) return cudaErrorInvalidValue;
    if (mode == PM_FWD) return launch_pass_t<Tc, Tin, Tout, PM_FWD, 0>(P, in, out, st);
    if (mode == PM_FUSED) return launch_pass_t<Tc, Tin, Tout, PM_FUSED, 0>(P, in, out, st);
    return launch_pass_t<Tc, Tin, Tout, PM_BWD, 0>(P, in, out, st);
  } else {
    if (mode == PM_FWD) return launch_pass_t<Tc, Tin, Tout, PM_FWD, 0>(P, in, out, st);
    if (mode == PM_FUSED) return launch_pass_t<Tc, Tin, Tout, PM_FUSED, 0>(P, in, out, st);
    if (ndot == 0) return launch_pass_t<Tc, Tin, Tout, PM_BWD, 0>(P, in, out, st);
    if (ndot == 1) return launch_pass_t<Tc, Tin, Tout, PM_BWD, 1>(P, in, out, st);
    return launch_pass_t<Tc, Tin, Tout, PM_BWD, 2>(P, in, out, st);
  }
}

template <typename Tc, typename Tin, typename Tout, int MODE, int NDOT>
static cudaError_t launch_batched_t(const PassDesc<Tc, Tin, Tout>* sys, const long long* tile_prefix, int nsys,
                                   long long total_tiles, size_t smem, cudaStream_t st) {
  auto kern = precond_pass_batched<Tc, Tin, Tout, MODE, NDOT>;
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

template <typename Tc, typename Tin, typename Tout>
cudaError_t launch_pass_batched(const PassDesc<Tc, Tin, Tout>* sys, const long long* tile_prefix, int nsys,
                                long long total_tiles, size_t smem, int mode, int ndot, cudaStream_t st) {
  constexpr bool in64 = std::is_same<Tc, float>::value && std::is_same<Tin, double>::value;
  constexpr bool out64 = std::is_same<Tc, float>::value && std::is_same<Tout, double>::value;
  constexpr bool f32 = std::is_same<Tc, float>::value && !in64 && !out64;
  if constexpr (in64) {  // the same combinations as launch_pass
    if (mode != PM_FWD) return cudaErrorInvalidValue;
    return launch_batched_t<Tc, Tin, Tout, PM_FWD, 0>(sys, tile_prefix, nsys, total_tiles, smem, st);
  } else if constexpr (out64) {
    if (mode != PM_BWD) return cudaErrorInvalidValue;
    if (ndot == 0) return launch_batched_t<Tc, Tin, Tout, PM_BWD, 0>(sys, tile_prefix, nsys, total_tiles, smem, st);
    if (ndot == 1) return launch_batched_t<Tc, Tin, Tout, PM_BWD, 1>(sys, tile_prefix, nsys, total_tiles, smem, st);
    return launch_batched_t<Tc, Tin, Tout, PM_BWD, 2>(sys, tile_prefix, nsys, total_tiles, smem, st);
  } else if constexpr (f32) {
    if (ndot != 0) return cudaErrorInvalidValue;
    if (mode == PM_FWD) return launch_batched_t<Tc, Tin, Tout, PM_FWD, 0>(sys, tile_prefix, nsys, total_tiles, smem, st);
    if (mode == PM_FUSED)
      return launch_batched_t<Tc, Tin, Tout, PM_FUSED, 0>(sys, tile_prefix, nsys, total_tiles, smem, st);
    return launch_batched_t<Tc, Tin, Tout, PM_BWD, 0>(sys, tile_prefix, nsys, total_tiles, smem, st);
  } else {
    if (mode == PM_FWD) return launch_batched_t<Tc, Tin, Tout, PM_FWD, 0>(sys, tile_prefix, nsys, total_tiles, smem, st);
    if (mode == PM_FUSED)
      return launch_batched_t<Tc, Tin, Tout, PM_FUSED, 0>(sys, tile_prefix, nsys, total_tiles, smem, st);
    if (ndot == 0) return launch_batched_t<Tc, Tin, Tout, PM_BWD, 0>(sys, tile_prefix, nsys, total_tiles, smem, st);
    if (ndot == 1) return launch_batched_t<Tc, Tin, Tout, PM_BWD, 1>(sys, tile_prefix, nsys, total_tiles, smem, st);
    return launch_batched_t<Tc, Tin, Tout, PM_BWD, 2>(sys, tile_prefix, nsys, total_tiles, smem, st);
  }
}

template <typename Tin, typename Tout>
cudaError_t launch_wpass_batched(const PassDesc<float, Tin, Tout>* sys, const long long* tile_prefix, int nsys,
                                 long long total_tiles, size_t smem, int N, int kind, int mode, int ndot,
                                 cudaStream_t st) {
  switch (N) {
    case 64: return launch_wpass_batched_n<64, Tin, Tout>(sys, tile_prefix, nsys, total_tiles, smem, kind, mode, ndot, st);
    case 128: return launch_wpass_batched_n<128, Tin, Tout>(sys, tile_prefix, nsys, total_tiles, smem, kind, mode, ndot, st);
    case 256: return launch_wpass_batched_n<256, Tin, Tout>(sys, tile_prefix, nsys, total_tiles, smem, kind, mode, ndot, st);
    case 512: return launch_wpass_batched_n<512, Tin, Tout>(sys, tile_prefix, nsys, total_tiles, smem, kind, mode, ndot, st);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_wpass_batched<double, float>(const PassDesc<float, double, float>*, const long long*, int,
                                                         long long, size_t, int, int, int, int, cudaStream_t);
template cudaError_t launch_wpass_batched<float, float>(const PassDesc<float, float, float>*, const long long*, int,
                                                        long long, size_t, int, int, int, int, cudaStream_t);
template cudaError_t launch_wpass_batched<float, double>(const PassDesc<float, float, double>*, const long long*, int,
                                                         long long, size_t, int, int, int, int, cudaStream_t);

#define IFFD_INST_BATCHED(Tc, Tin, Tout)                                                                      \
  template cudaError_t launch_pass_batched<Tc, Tin, Tout>(const PassDesc<Tc, Tin, Tout>*, const long long*, int, \
                                                          long long, size_t, int, int, cudaStream_t);
IFFD_INST_BATCHED(double, double, double)
IFFD_INST_BATCHED(float, double, float)
IFFD_INST_BATCHED(float, float, float)
IFFD_INST_BATCHED(float, float, double)

template cudaError_t launch_pass<double, double, double>(const PassLaunch<double>&, int, int, const double*,
                                                         double*, cudaStream_t);
template cudaError_t launch_pass<float, double, float>(const PassLaunch<float>&, int, int, const double*, float*,
                                                       cudaStream_t);
template cudaError_t launch_pass<float, float, float>(const PassLaunch<float>&, int, int, const float*, float*,
                                                      cudaStream_t);
template cudaError_t launch_pass<float, float, double>(const PassLaunch<float>&, int, int, const float*, double*,
                                                       cudaStream_t);

}  // namespace iffd
