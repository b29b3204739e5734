// Device bodies of the PCG vector kernels and the fixed-order reductions
// (Section 3), shared by the kernels of pcg.cu and the persistent engine
// launch (persist.cu). CG selects L2-coherent loads of the solver data.
#pragma once

#include "device_common.cuh"
#include "kernels.h"

namespace iffd {

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[kThreads / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// x = 0, r = f, partial ||f||^2 (block `blk` of `nblk`)
__device__ __forceinline__ void init_body(const double* __restrict__ f, double* __restrict__ x, double* __restrict__ r,
                                          long long N, double* __restrict__ partial, int blk, int nblk) {
  double s = 0.0;
  for (long long i = blk * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)nblk * blockDim.x) {
    const double v = f[i];
    x[i] = 0.0;
    r[i] = v;
    s = fma(v, v, s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blk] = s;
}

// x += alpha p, r -= alpha q, partial ||r||^2. Where the four vectors are
// 16-byte aligned a thread moves two values per access (twice the bytes in
// flight for the same number of loads); the same values either way, only the
// grouping of the partial sums differs.
template <bool CG = false>
__device__ __forceinline__ void update_body(double* __restrict__ x, double* __restrict__ r,
                                            const double* __restrict__ p, const double* __restrict__ q,
                                            const SolveState* __restrict__ st, long long N,
                                            double* __restrict__ partial, int blk, int nblk) {
  const double alpha = ldd<CG>(&st->alpha);
  double s = 0.0;
  const long long t0 = blk * (long long)blockDim.x + threadIdx.x, stride = (long long)nblk * blockDim.x;
  const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(r) |
                     reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(q)) & 15) == 0;
  long long i0 = 0;
  if (vec) {
    const long long n2 = N / 2;
    double2* x2 = reinterpret_cast<double2*>(x);
    double2* r2 = reinterpret_cast<double2*>(r);
    const double2* p2 = reinterpret_cast<const double2*>(p);
    const double2* q2 = reinterpret_cast<const double2*>(q);
#pragma unroll 2
    for (long long i = t0; i < n2; i += stride) {
      const double2 pv = ldd<CG>(p2 + i), xv = ldd<CG>(x2 + i), qv = ldd<CG>(q2 + i), rv = ldd<CG>(r2 + i);
      x2[i] = double2{fma(alpha, pv.x, xv.x), fma(alpha, pv.y, xv.y)};
      const double2 rn{fma(-alpha, qv.x, rv.x), fma(-alpha, qv.y, rv.y)};
      r2[i] = rn;
      s = fma(rn.x, rn.x, s);
      s = fma(rn.y, rn.y, s);
    }
    i0 = 2 * n2;  // an odd N leaves one value
  }
  for (long long i = i0 + t0; i < N; i += stride) {
    x[i] = fma(alpha, ldd<CG>(p + i), ldd<CG>(x + i));
    const double rv = fma(-alpha, ldd<CG>(q + i), ldd<CG>(r + i));
    r[i] = rv;
    s = fma(rv, rv, s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blk] = s;
}

// status codes mirror iffd_status in include/iffd.h
constexpr int kStOk = 0, kStNotConverged = 6, kStBreakdown = 7;

// The reduction order is that of kFinThreads threads whatever the block size
// (a divisor of it): virtual thread v sums parts v, v + kFinThreads, ...; each
// virtual warp reduces by the xor-shuffle tree; thread 0 adds the warp sums in
// order. A 1024-thread CTA runs one virtual thread per thread; a 256-thread
// CTA (the persistent engine launch) runs four, in slots that keep each
// virtual warp inside one physical warp, so both give bitwise the same sums.
constexpr int kFinThreads = 1024;

template <bool CG = false>
__device__ __forceinline__ void finalize_body(SolveState* st, const double* __restrict__ partial, int nparts, int phase,
                                              double tol2, int maxit) {
  __shared__ double red[2][kFinThreads / 32];
  if (phase != FP_FF && phase != FP_TRUE && ldd<CG>(&st->done)) return;
  // The flexible beta also needs the second set partial[nparts..2 nparts).
  const bool two = (phase == FP_RZ_FLEX);
  const int slots = kFinThreads / blockDim.x;
  for (int j = 0; j < slots; ++j) {
    const int v = threadIdx.x + j * blockDim.x;  // virtual thread
    double s = 0.0, s2 = 0.0;
    for (int i = v; i < nparts; i += kFinThreads) {
      s += ldd<CG>(partial + i);
      if (two) s2 += ldd<CG>(partial + nparts + i);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, off);
      s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    }
    if ((v & 31) == 0) {
      red[0][v >> 5] = s;
      red[1][v >> 5] = s2;
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double tot = 0.0, tot2 = 0.0;
  for (int w = 0; w < kFinThreads / 32; ++w) {
    tot += red[0][w];
    tot2 += red[1][w];
  }
  switch (phase) {
    case FP_FF:
      st->ff = tot;
      st->iters = 0;
      st->status = kStOk;
      st->done = (tot == 0.0) ? 1 : 0;
      st->rr = tot;
      break;
    case FP_RZ0:
      st->rz = tot;
      if (!(tot > 0.0)) { st->status = kStBreakdown; st->done = 1; }
      break;
    case FP_PQ:
      st->pq = tot;
      if (!(tot > 0.0) || !isfinite(tot)) { st->status = kStBreakdown; st->done = 1; }
      else st->alpha = ldd<CG>(&st->rz) / tot;
      break;
    case FP_RR:
      st->rr = tot;
      st->iters = ldd<CG>(&st->iters) + 1;
      if (!isfinite(tot)) { st->status = kStBreakdown; st->done = 1; }
      else if (tot <= tol2 * ldd<CG>(&st->ff)) { st->status = kStOk; st->done = 1; }
      else if (st->iters >= maxit) { st->status = kStNotConverged; st->done = 1; }
      break;
    case FP_RZ:
      if (!(tot > 0.0) || !isfinite(tot)) { st->status = kStBreakdown; st->done = 1; }
      else {
        const double rz = ldd<CG>(&st->rz);
        st->beta = tot / rz;
        st->rz_old = rz;
        st->rz = tot;
      }
      break;
    case FP_RZ_FLEX:
      // flexible (Polak-Ribiere) beta = (z_new, r_new - r_old) / (z_old, r_old)
      //                              = -alpha (z_new, q) / rz_old;
      // partial[0..nparts) holds (r,z), partial[nparts..2 nparts) holds (q,z)
      st->zq = tot2;
      if (!(tot > 0.0) || !isfinite(tot)) { st->status = kStBreakdown; st->done = 1; }
      else {
        const double rz = ldd<CG>(&st->rz);
        st->beta = -ldd<CG>(&st->alpha) * tot2 / rz;
        st->rz_old = rz;
        st->rz = tot;
      }
      break;
    case FP_TRUE:
      st->zq = tot;  // ||f - A u||^2 of the final iterate
      break;
  }
}

}  // namespace iffd
