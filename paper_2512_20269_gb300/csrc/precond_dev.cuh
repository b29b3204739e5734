// Device helpers shared by the block-wide transform passes (precond.cu) and
// the warp-FFT passes (precond_warp.cuh): small register DFTs, the V_reg^T
// gather of one pencil, a warp sum.
#pragma once

#include <type_traits>

#include "device_common.cuh"

namespace iffd {

template <typename T>
__device__ __forceinline__ Cplx<T> ldc(const T* p) {
  return {ldg(p), ldg(p + 1)};
}

// ------------------------------------------------------------- small DFTs
// Forward DFTs y_t = sum_q v_q exp(-2 pi i q t / R) in registers.
template <typename T>
__device__ __forceinline__ void dft2(Cplx<T>* v) {
  const Cplx<T> a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <typename T>
__device__ __forceinline__ void dft4(Cplx<T>* v) {
  const Cplx<T> t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
  const Cplx<T> t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = cadd(t1, mul_mi(t3));
  v[3] = csub(t1, mul_mi(t3));
}

// plus = e + r s and minus = e - r s: two fused multiply-adds (float,
// double); for double-float one product and two sums (23 instead of 30
// FP32 instructions)
template <typename T>
__device__ __forceinline__ void pm_fma(T r, T s, T e, T& plus, T& minus) {
  if constexpr (std::is_same<T, df>::value) {
    const T t = r * s;
    plus = e + t;
    minus = e - t;
  } else {
    plus = fma(r, s, e);
    minus = fma(-r, s, e);
  }
}

template <typename T>
__device__ __forceinline__ void dft8(Cplx<T>* v) {
  const T r = T(0.70710678118654752440084436210484903928);
  Cplx<T> e[4] = {v[0], v[2], v[4], v[6]};
  Cplx<T> o[4] = {v[1], v[3], v[5], v[7]};
  dft4(e);
  dft4(o);
  // o_t *= exp(-2 pi i t / 8): o_1 = r (s1x, s1y), o_3 = r (s3x, -s3y) with
  // r = 1/sqrt(2), the factor r folded into the output FMAs
  const T s1x = o[1].x + o[1].y, s1y = o[1].y - o[1].x;
  const T s3x = o[3].y - o[3].x, s3y = o[3].x + o[3].y;
  const Cplx<T> o2 = mul_mi(o[2]);
  v[0] = cadd(e[0], o[0]);
  v[4] = csub(e[0], o[0]);
  pm_fma(r, s1x, e[1].x, v[1].x, v[5].x);
  pm_fma(r, s1y, e[1].y, v[1].y, v[5].y);
  v[2] = cadd(e[2], o2);
  v[6] = csub(e[2], o2);
  pm_fma(r, s3x, e[3].x, v[3].x, v[7].x);
  pm_fma(r, s3y, e[3].y, v[7].y, v[3].y);
}

// y_reg[i] = (V_reg^T r)_i for the pencil held in row[0..m-1] (row values of
// type T, tables of type TT: the same type, or FP32 tables for a pair).
template <typename T, typename TT>
__device__ __forceinline__ T reg_gather(const T* row, int i, const AxisTab<TT>& ax) {
  if (i < ax.nL) {
    T s = T(0);
    for (int r = 0; r < ax.rowsL; ++r) s = fma(ldg(ax.VL + r * ax.nL + i), row[r], s);
    return s;
  }
  if (i >= ax.n_reg - ax.nR) {
    const int c = ax.n_reg - 1 - i;
    T s = T(0);
    for (int r = 0; r < ax.rowsR; ++r) s = fma(ldg(ax.VR + r * ax.nR + c), row[ax.m - 1 - r], s);
    return s;
  }
  int o = ax.o;
  for (int b = 0; b < ax.nblk; ++b) {  // interior blocks (repeated knots only)
    const int* B = ax.blk + 6 * b;
    const int c0 = ldg(B), c1 = ldg(B + 1);
    if (i < c0) break;
    if (i < c1) {
      const int r0 = ldg(B + 2), r1 = ldg(B + 3), w = c1 - c0;
      const TT* V = ax.VB + ldg(B + 5) + (i - c0);
      T s = T(0);
      for (int r = r0; r < r1; ++r) s = fma(ldg(V + (r - r0) * w), row[r], s);
      return s;
    }
    o = ldg(B + 4);
  }
  return row[i + o];
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

}  // namespace iffd
