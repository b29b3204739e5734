// Compile-time geometry of the warp-FFT passes (precond_warp.cuh), shared
// with the host code that sizes their launches (precond.cu).
#pragma once

#include <type_traits>

#include "device_common.cuh"

namespace iffd {

// Complex values per lane (R) and lanes per sequence (LS) for length N; a warp
// holds 32 / LS sequences, a CTA of 8 warps 8 * 32 / LS pencil pairs.
template <int N>
struct WarpFft;
template <>
struct WarpFft<64> {
  static constexpr int R = 8, LS = 8;
};
template <>
struct WarpFft<128> {
  static constexpr int R = 8, LS = 16;
};
template <>
struct WarpFft<256> {
  static constexpr int R = 8, LS = 32;
};
template <>
struct WarpFft<512> {
  static constexpr int R = 16, LS = 32;
};

// Pencils per CTA: two per sequence (real and imaginary part), one sequence
// per LS lanes; the paired pass (FP32, two sequences per lane group) twice that.
template <int N, bool PAIR = false>
__host__ __device__ constexpr int warp_pencils() {
  return (PAIR ? 4 : 2) * (kThreads / 32) * (32 / WarpFft<N>::LS);
}

// Sequence buffers skip one complex slot after every 8, so that the strided
// stores of the early stages spread over the banks.
__host__ __device__ constexpr int wpad(int i) { return i + (i >> 3); }
template <int N>
__host__ __device__ constexpr int wbuf_len() {
  return N + N / 8;
}
inline int wbuf_len_host(int N) { return N + N / 8; }

// Whether the warp pass of arithmetic T keeps each pencil pair's sequence
// buffer inside the pair's tile rows (double-float: a fourth resident CTA per
// SM, measured faster; FP32 kept the separate buffers, measured faster there).
template <typename T>
__host__ __device__ constexpr bool walias() {
  return std::is_same<T, df>::value;
}

}  // namespace iffd
