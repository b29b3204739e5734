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

template <typename T>
struct Vec2Of;
template <>
struct Vec2Of<df> {
  using type = df2;
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

// The sum leaves the pair unnormalised: lo = (error of hi + hi) + a.lo + b.lo
// may exceed ulp(hi) / 2 by a few units. The next product (or fma)
// renormalises (its fast_two_sum), which happens at least once per FFT stage
// (the twiddle products) and in every separation step; the error bound of the
// sum stays near 2^-47 of |a| + |b|. Saves 3 of 11 instructions per addition.
__device__ __forceinline__ df operator+(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return {s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))};
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

// the float / double overloads stay visible next to the df one inside the namespace
using ::fma;

// a * b + c * d with one sum of the two exact high products: their errors
// and cross terms join the low part, left unnormalised as in the sum (the
// next product renormalises). 16 instructions against 22 for a product and a
// fused multiply-add; the error stays near 2^-47 of |a b| + |c d|.
__device__ __forceinline__ df dot2(df a, df b, df c, df d) {
  const float p1 = __fmul_rn(a.hi, b.hi);
  float e1 = __fmaf_rn(a.hi, b.hi, -p1);
  e1 = __fmaf_rn(a.hi, b.lo, e1);
  e1 = __fmaf_rn(a.lo, b.hi, e1);
  const float p2 = __fmul_rn(c.hi, d.hi);
  float e2 = __fmaf_rn(c.hi, d.hi, -p2);
  e2 = __fmaf_rn(c.hi, d.lo, e2);
  e2 = __fmaf_rn(c.lo, d.hi, e2);
  const df s = two_sum(p1, p2);
  return {s.hi, __fadd_rn(s.lo, __fadd_rn(e1, e2))};
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

// ------------------------------------------------------------ conversions
// FP64 <-> double-float at the first and last transform pass. On this GPU a
// float64 conversion or addition runs on the FP64 pipe, so both directions
// work on the bit patterns with integer instructions and leave the FP64 pipe
// one addition (df -> double) or nothing (double -> df) per value; values
// outside the range where the integer route is exact take the FP64 route.
__host__ __device__ __forceinline__ unsigned long long bits_of(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long u;
  __builtin_memcpy(&u, &x, sizeof u);
  return u;
#endif
}
__host__ __device__ __forceinline__ double double_of(unsigned long long u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  __builtin_memcpy(&x, &u, sizeof x);
  return x;
#endif
}
__host__ __device__ __forceinline__ unsigned bits_of(float x) {
#ifdef __CUDA_ARCH__
  return (unsigned)__float_as_int(x);
#else
  unsigned u;
  __builtin_memcpy(&u, &x, sizeof u);
  return u;
#endif
}
__host__ __device__ __forceinline__ float float_of(unsigned u) {
#ifdef __CUDA_ARCH__
  return __int_as_float((int)u);
#else
  float x;
  __builtin_memcpy(&x, &u, sizeof x);
  return x;
#endif
}
__host__ __device__ __forceinline__ int clz32(unsigned x) {
#ifdef __CUDA_ARCH__
  return __clz((int)x);
#else
  return x ? __builtin_clz(x) : 32;
#endif
}

// The rare values outside the integer route: a real branch to a function of
// its own (kept out of line so that the common path carries no float64
// instruction).
static __device__ __noinline__ df to_df_fp64(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
static __device__ __noinline__ double float_to_double_fp64(float f) { return (double)f; }

// x = hi + lo with hi the first 24 significant bits of x (truncated) and lo
// the next 29 bits rounded to 24 (relative error <= 2^-48 of |x|), from the
// bit pattern of x. The binary exponent of x must lie in [-74, 127] (float
// exponent field 53..254) so that hi and lo are normal floats; zero, smaller,
// larger and non-finite values take the float64 route.
__host__ __device__ __forceinline__ df to_df(double x) {
  const unsigned long long b = bits_of(x);
  const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
  const unsigned sign = h32 & 0x80000000u;
  const int fe = (int)((h32 >> 20) & 0x7FFu) - 896;  // float exponent field of hi
  if (((h32 << 1) | l32) == 0) return {float_of(sign), 0.f};  // +-0, tested on the 32-bit halves
  if (fe < 53 || fe > 254) {
#ifdef __CUDA_ARCH__
    return to_df_fp64(x);
#else
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
#endif
  }
  const float h = float_of(sign | ((unsigned)fe << 23) | ((h32 & 0xFFFFFu) << 3) | (l32 >> 29));
  const unsigned r = l32 & 0x1FFFFFFFu;  // x - hi = r 2^(fe - 179)
  if (r == 0) return {h, 0.f};
  const int lz = clz32(r) - 3;   // leading zeros inside the 29-bit field
  const unsigned rn = r << lz;   // leading one at bit 28
  // 23 fraction bits, rounded half up (a carry moves into the exponent field)
  const unsigned lb = ((unsigned)(fe - 24 - lz) << 23) + ((rn >> 5) & 0x7FFFFFu) + ((rn >> 4) & 1u);
  return {h, float_of(sign | lb)};
}

// exact float -> double on the integer pipe (normal floats and zeros)
__host__ __device__ __forceinline__ double float_to_double_bits(float f) {
  const unsigned u = bits_of(f);
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  if ((u & 0x7FFFFFFFu) == 0) return double_of(s);
  if (e == 0 || e == 255) {  // subnormal, inf, nan
#ifdef __CUDA_ARCH__
    return float_to_double_fp64(f);
#else
    return (double)f;
#endif
  }
  return double_of(s | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29));
}

// hi + lo rounded to float64: one FP64 addition
__host__ __device__ __forceinline__ double to_double(df v) {
  return float_to_double_bits(v.hi) + float_to_double_bits(v.lo);
}

template <typename To>
struct Cvt;
template <>
struct Cvt<df> {
  __device__ __forceinline__ static df from(double v) { return to_df(v); }
  __device__ __forceinline__ static df from(df v) { return v; }
};
template <>
struct Cvt<double> {
  __device__ __forceinline__ static double from(double v) { return v; }
  __device__ __forceinline__ static double from(float v) { return (double)v; }
  __device__ __forceinline__ static double from(df v) { return to_double(v); }
};

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
