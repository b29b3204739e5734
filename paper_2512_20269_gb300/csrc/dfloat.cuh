// Double-float ("df") arithmetic: a value is the unevaluated sum hi + lo of two
// float32 numbers with |lo| <= ulp(hi) / 2, carrying about 48 significant
// bits. It runs the FP64-accurate transform passes on the FP32 pipe, which on
// this GPU retires about 60 times as many instructions per clock as the FP64
// pipe.
//
// The operations are the classical error-free transformations:
//  - two_sum (Knuth, The Art of Computer Programming vol. 2, 4.2.2; Moller
//    1965): s = fl(a + b) and the exact error e = (a + b) - s in 6 additions;
//  - fast_two_sum (Dekker 1971): the same in 3 additions when |a| >= |b|;
//  - two_prod through a fused multiply-add: p = fl(a b), e = fma(a, b, -p)
//    is the exact error of the product.
// On top of them (Dekker 1971, "A floating-point technique for extending the
// available precision"; Shewchuk 1997): the double-float sum adds the exact
// error of hi + hi to the low parts and renormalises; the product forms the
// exact high product and adds the cross terms hi * lo; both have relative error
// near 2^-47 (2^-44 for the sum under cancellation of the high parts, where
// the error is still below 2^-47 of |a| + |b| -- the normwise bound that an
// FFT's error analysis needs).
//
// Every step uses the round-to-nearest intrinsics (__fadd_rn, __fmul_rn,
// __fmaf_rn), which the compiler never contracts into fused multiply-adds or
// reassociates: the error-free transformations depend on each rounding.
#pragma once

#include <cuda_runtime.h>

namespace iffd {

struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  // exact for constants and table entries: the split is done in double,
  // folded at compile time for literals
  __host__ __device__ constexpr explicit df(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ constexpr explicit df(int x) : hi((float)x), lo(0.f) {}
};

// one complex value (16 bytes, one 128-bit shared-memory access)
struct __align__(16) df2 {
  df x, y;
};

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fadd_rn(b, -__fadd_rn(s, -a));
  return {s, e};
}

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fadd_rn(s, -a);
  const float e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
  return {s, e};
}

__device__ __forceinline__ df operator+(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df operator-(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// a * b + c with the exact high product folded into the sum
__device__ __forceinline__ df fma(df a, df b, df c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const df s = two_sum(p, c.hi);
  const float t = __fadd_rn(s.lo, __fadd_rn(e, c.lo));
  return fast_two_sum(s.hi, t);
}

__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }

// 1 / b: the float reciprocal refined by one Newton step x + x (1 - b x)
// evaluated with the exact product b.hi x
__device__ __forceinline__ df recip(df b) {
  const float x = __frcp_rn(b.hi);
  const float p = __fmul_rn(b.hi, x);
  const float pe = __fmaf_rn(b.hi, x, -p);  // b.hi x = p + pe exactly
  // r = 1 - b x = (1 - p) - pe - b.lo x  (1 - p is exact: p is within an ulp of 1)
  const float r = __fadd_rn(__fadd_rn(__fadd_rn(1.f, -p), -pe), -__fmul_rn(b.lo, x));
  return fast_two_sum(x, __fmul_rn(x, r));
}

// sign flip on the integer pipe (as neg_if for float / double)
__device__ __forceinline__ df neg_if(df v, bool neg) {
  const int m = (int)neg << 31;
  return {__int_as_float(__float_as_int(v.hi) ^ m), __int_as_float(__float_as_int(v.lo) ^ m)};
}

__device__ __forceinline__ df to_df(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double to_double(df v) { return (double)v.hi + (double)v.lo; }

__device__ __forceinline__ df ldg(const df* p) {
  const float2 t = __ldg(reinterpret_cast<const float2*>(p));
  return {t.x, t.y};
}
__device__ __forceinline__ df2 ldg(const df2* p) {
  const float4 t = __ldg(reinterpret_cast<const float4*>(p));
  return {{t.x, t.y}, {t.z, t.w}};
}

__device__ __forceinline__ df shfl_xor(df v, int off) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off)};
}

}  // namespace iffd
