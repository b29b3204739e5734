// Two FP32 values handled as one (f2): the arithmetic type of the paired
// FP32 warp-FFT passes, where every lane carries the same step of two
// independent complex sequences (four pencils) at once. Each operation acts
// on the two components separately with the same FP32 operation a single
// sequence would use, so a pencil's result is bitwise that of the unpaired
// pass; what the pairing saves is the work around the arithmetic: one
// 128-bit shared-memory access moves a value of both sequences, and one
// twiddle, table entry or index computation serves both.
#pragma once

#include "device_common.cuh"

namespace iffd {

struct __align__(8) f2 {
  float a, b;
  f2() = default;
  __host__ __device__ constexpr f2(float s) : a(s), b(s) {}
  __host__ __device__ constexpr f2(float x, float y) : a(x), b(y) {}
};

// one complex value of both sequences: one 128-bit shared-memory access
struct __align__(16) f2x2 {
  f2 x, y;
};
template <>
struct Vec2Of<f2> {
  using type = f2x2;
};

// the type of the tables (twiddles, V_reg blocks, W, eigenvalues) that
// serve an arithmetic type: its own, except FP32 for the pair
template <typename T>
struct TabOf {
  using type = T;
};
template <>
struct TabOf<f2> {
  using type = float;
};
template <typename T>
using tab_t = typename TabOf<T>::type;

template <typename T>
struct IsPair {
  static constexpr bool value = false;
};
template <>
struct IsPair<f2> {
  static constexpr bool value = true;
};

__device__ __forceinline__ f2 operator+(f2 x, f2 y) { return {x.a + y.a, x.b + y.b}; }
__device__ __forceinline__ f2 operator-(f2 x, f2 y) { return {x.a - y.a, x.b - y.b}; }
__device__ __forceinline__ f2 operator-(f2 x) { return {-x.a, -x.b}; }
__device__ __forceinline__ f2 operator*(f2 x, f2 y) { return {x.a * y.a, x.b * y.b}; }
__device__ __forceinline__ f2 operator/(f2 x, f2 y) { return {x.a / y.a, x.b / y.b}; }
__device__ __forceinline__ f2 operator+(float s, f2 y) { return {s + y.a, s + y.b}; }
__device__ __forceinline__ f2 operator*(float s, f2 y) { return {s * y.a, s * y.b}; }
__device__ __forceinline__ f2 operator*(f2 x, float s) { return {x.a * s, x.b * s}; }
__device__ __forceinline__ f2& operator+=(f2& x, f2 y) {
  x = x + y;
  return x;
}
__device__ __forceinline__ f2 fma(f2 x, f2 y, f2 z) { return {fmaf(x.a, y.a, z.a), fmaf(x.b, y.b, z.b)}; }
__device__ __forceinline__ f2 fma(float s, f2 y, f2 z) { return {fmaf(s, y.a, z.a), fmaf(s, y.b, z.b)}; }
__device__ __forceinline__ f2 fma(f2 x, float s, f2 z) { return {fmaf(x.a, s, z.a), fmaf(x.b, s, z.b)}; }
__device__ __forceinline__ f2 neg_if(f2 v, bool neg) { return {neg_if(v.a, neg), neg_if(v.b, neg)}; }
__device__ __forceinline__ f2 shfl_xor(f2 v, int off) { return {shfl_xor(v.a, off), shfl_xor(v.b, off)}; }

// a * w with one twiddle for both sequences (the operations of cmul)
__device__ __forceinline__ Cplx<f2> cmul(Cplx<f2> a, Cplx<float> w) {
  return {fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x)};
}

}  // namespace iffd
