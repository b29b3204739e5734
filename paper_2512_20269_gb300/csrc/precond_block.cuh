// Device code of the block-wide transform passes (eq. "preconditioner"):
// small DFTs, the Stockham and Bluestein FFTs in shared memory, and the load /
// transform / store steps of one tile. Shared by the pass kernels
// (precond.cu) and the persistent engine launch (persist.cu); CG selects
// L2-coherent loads of the solver data.
#pragma once

#include <cuda_pipeline.h>

#include "device_common.cuh"
#include "kernels.h"
#include "precond_dev.cuh"

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
  ya = dot2(fx, tay, fy, tax);
  yb = dot2(fx, tby, fy, tbx);
}


// A transform pass processes tiles of PP pencils along `axis` (tile_setup):
// load the tile into shared memory, transform it (compute_tile), store it.
// Partial dot products go to partial[ptile] (and partial[pstride + ptile]).

// Synchronous tile load (the caller synchronises afterwards).
template <typename Tc, typename Tin, bool CG = false>
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
          if (pc < g.nvalid) v[u] = ldd<CG>(in + pbase[pc] + i * g.S);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (slot[u] >= 0) tile[slot[u]] = cvt<Tc>(v[u]);
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
        for (int i = sub; i < ax.wlo; i += 8) acc = fma(ldg(ax.W + i * nw + k), row[i], acc);
        for (int i = ax.whi + sub; i < m; i += 8) acc = fma(ldg(ax.W + i * nw + k), row[i], acc);
      }
      acc += shfl_xor(acc, 4);
      acc += shfl_xor(acc, 2);
      acc += shfl_xor(acc, 1);
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
        const Tc A = ldg(t4), B = ldg(t4 + 1), C = ldg(t4 + 2), E = ldg(t4 + 3);
        ra[N - 1 - k] = dot2(A, Ar, B, Ai);
        rb[N - 1 - k] = dot2(A, Br, B, Bi);
        if (k > 0 && 2 * k != N) {
          ra[k - 1] = dot2(C, Ar, -E, Ai);
          rb[k - 1] = dot2(C, Br, -E, Bi);
        }
      }
    } else if (ax.kind == 2) {
      for (int w = tid; w < npairs * N; w += blockDim.x) {
        const int pr = ax.fN.div(w), j = w - pr * N;
        Tc ya, yb;
        gen_im(Z + (size_t)pr * F, ax.gq * (j + 1) - ax.gqe, L, ldg(ax.post + 2 * j), ldg(ax.post + 2 * j + 1),
               ya, yb);
        tile[(2 * pr) * ldt + j] = ya;
        tile[(2 * pr + 1) * ldt + j] = yb;
      }
    } else {
      for (int w = tid; w < npairs * N; w += blockDim.x) {
        const int pr = ax.fN.div(w), j = w - pr * N;
        const Cplx<Tc> z = Z[(size_t)pr * F + j + 1];
        const Tc sc = ldg(ax.post + j);
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
    if constexpr (std::is_same<Tc, df>::value) {
      // double-float: the product with a Newton-refined reciprocal of the sum
      for (int e = tid; e < PP * m; e += blockDim.x) {
        const int pc = ax.fm.div(e), i = e - pc * m;
        if (pc >= g.nvalid) continue;  // padding pencils
        df den = ldg(lamA + pia[pc]);
        if (dims.d == 3) den = den + ldg(lamB + pib[pc]);
        tile[pc * ldt + i] = tile[pc * ldt + i] * recip(ldg(ax.lam + i) + den);
      }
    } else if (ax.rden != nullptr) {
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
        Tc den = ldg(ax.lam + i) + ldg(lamA + pia[pc]);
        if (dims.d == 3) den += ldg(lamB + pib[pc]);
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
        const Tc A = ldg(t4), B = ldg(t4 + 1), C = ldg(t4 + 2), E = ldg(t4 + 3);
        Cplx<Tc>* G = bufA + (size_t)pr * F;
        if (k == 0 || 2 * k == N) {
          const Tc s = A + A;
          G[k] = {s * za[N - 1 - k], s * zb[N - 1 - k]};
        } else {
          const Tc ar = dot2(A, za[N - 1 - k], C, za[k - 1]);
          const Tc ai = dot2(-B, za[N - 1 - k], E, za[k - 1]);
          const Tc br = dot2(A, zb[N - 1 - k], C, zb[k - 1]);
          const Tc bi = dot2(-B, zb[N - 1 - k], E, zb[k - 1]);
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
          const Tc sc = ldg(ax.post + 4 * N + l - 1);  // 1 / D~
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
          const Tc sc = ldg(ax.post + l - 1);
          va = sc * za[l - 1];
          vb = sc * zb[l - 1];
        } else {
          const Tc sc = ldg(ax.post + 2 * n - 1 - l);
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
          gen_im(Zp, ax.gq * (j + 1) - ax.gqc, L, ldg(ax.post + 2 * N + 2 * j), ldg(ax.post + 2 * N + 2 * j + 1),
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
        for (int c = 0; c < ax.nL; ++c) x = fma(ldg(ax.VL + i * ax.nL + c), wreg(c), x);
      } else if (i >= m - ax.rowsR) {
        const int r = m - 1 - i;
        x = Tc(0);
        for (int c = 0; c < ax.nR; ++c) x = fma(ldg(ax.VR + r * ax.nR + c), wreg(N - 1 - c), x);
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
            for (int c = c0; c < c1; ++c) x = fma(ldg(V + (c - c0)), wreg(c), x);
            inblk = true;
            break;
          }
          o = __ldg(B + 4);
        }
        if (!inblk) x = wreg(i - o);
      }
      if (i < ax.wlo || i >= ax.whi) {
        for (int k = 0; k < ax.n_out; ++k) x = fma(ldg(ax.W + i * ax.n_out + k), outv[pc * kMaxNout + k], x);
      }
      tile[pc * ldt + i] = x;
    }
    __syncthreads();
  }

}

// Store the tile (and the partial dot products of the last pass of a PCG step).
template <typename Tc, typename Tout, int NDOT, bool CG = false>
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
      const Tout vo = cvt<Tout>(v);
      out[off] = vo;
      if (NDOT >= 1) d0 = fma(ldr<CG>(dotv0 + off), cvt<double>(vo), d0);
      if (NDOT >= 2) d1 = fma(ldr<CG>(dotv1 + off), cvt<double>(vo), d1);
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
template <typename Tc, typename Tin, typename Tout, int MODE, int NDOT, bool CG = false>
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
  load_tile<Tc, Tin, CG>(in, tile, axis, PP, ldt, ax, pbase, g);
  __syncthreads();
  compute_tile<Tc, MODE>(tile, bufA, bufB, outv, dims, axis, PP, ldt, ax, lamA, lamB, pbase, pia, pib, g);
  store_tile<Tc, Tout, NDOT, CG>(tile, out, axis, PP, ldt, ax, pbase, g, dotv0, dotv1, partial, ptile, pstride);
}

}  // namespace iffd
