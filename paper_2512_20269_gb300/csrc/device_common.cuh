// Device-side types shared by the IFFD kernels (preconditioner passes,
// stiffness sweeps, PCG vector kernels). sm_103a only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace iffd {

constexpr int kMaxStages = 12;
constexpr int kMaxNout = 16;
constexpr int kThreads = 256;  // threads per CTA of every pass kernel

template <typename T>
struct Cplx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ Cplx<T> cadd(Cplx<T> a, Cplx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ Cplx<T> csub(Cplx<T> a, Cplx<T> b) { return {a.x - b.x, a.y - b.y}; }
// a * w
template <typename T>
__device__ __forceinline__ Cplx<T> cmul(Cplx<T> a, Cplx<T> w) {
  return {fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x)};
}
// -i * a
template <typename T>
__device__ __forceinline__ Cplx<T> mul_mi(Cplx<T> a) { return {a.y, -a.x}; }
// +i * a
template <typename T>
__device__ __forceinline__ Cplx<T> mul_pi(Cplx<T> a) { return {-a.y, a.x}; }

// Logical shape of a tensor-product coefficient array: x (direction 1) fastest.
struct Dims {
  int d;
  int m[3];
  long long N;
};

// Per-direction tables consumed by the transform passes (device pointers).
template <typename T>
struct AxisTab {
  int m, n_reg, n_out, p, o, nL, rowsL, wlo, whi, kind;
  int L, nst;
  int radix[kMaxStages];
  int twoff[kMaxStages];
  const T* VL;    // rowsL * nL (row-major); the right block is its mirror image
  const T* W;     // m * n_out (row-major) = V_out Q_out
  const T* lam;   // m: Lambda_reg then Lambda_out
  const T* post;  // DST-II/III: 4 per k = 0..N/2;  DST-I: n_reg values 1/(2 D~)
  const T* tw;    // complex FFT twiddles (interleaved), per stage offsets twoff
};

// Global run status shared by the kernels of one solve (device memory).
struct SolveState {
  double rz, rz_old, pq, rr, ff, alpha, beta, zq;
  int iters, done, status, pad;
};

}  // namespace iffd
