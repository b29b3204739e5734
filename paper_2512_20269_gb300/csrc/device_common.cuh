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

// The vector type of one complex value in shared-memory sequence buffers and
// twiddle tables (one 64- or 128-bit access).
template <typename T>
struct Vec2Of;
template <>
struct Vec2Of<float> {
  using type = float2;
};
template <>
struct Vec2Of<double> {
  using type = double2;
};
template <typename T>
using vec2_t = typename Vec2Of<T>::type;

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

// Read-only loads through the non-coherent cache, for any type __ldg takes;
// the double-float types (dfloat.cuh) add their own overloads.
template <typename T>
__device__ __forceinline__ T ldg(const T* p) {
  return __ldg(p);
}

// Loads of solver data (vectors, partial sums, solve states). With CG set
// they go through the L2-coherent path (ld.global.cg): in one persistent
// launch, data written by other CTAs after this SM cached a line must not be
// read from L1 or the read-only cache. ldd: plain load otherwise; ldr: the
// read-only cache otherwise (data that no kernel of the launch writes).
template <bool CG, typename T>
__device__ __forceinline__ T ldd(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}
template <bool CG, typename T>
__device__ __forceinline__ T ldr(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return __ldg(p);
}

__device__ __forceinline__ float shfl_xor(float v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
__device__ __forceinline__ double shfl_xor(double v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }

// Value conversion between the storage and arithmetic types (identity, or a
// float <-> double cast; dfloat.cuh adds the double-float conversions).
template <typename To>
struct Cvt {
  template <typename From>
  __device__ __forceinline__ static To from(From v) {
    return (To)v;
  }
};
}  // namespace iffd

#include "dfloat.cuh"

namespace iffd {
template <typename To, typename From>
__device__ __forceinline__ To cvt(From v) {
  return Cvt<To>::from(v);
}

// a * b + c * d: a fused multiply-add onto a product (double-float: one sum of
// the two exact products, dfloat.cuh)
template <typename S, typename T>
__device__ __forceinline__ T dot2(S a, T b, S c, T d) {
  return fma(a, b, c * d);
}

// a * w for double-float values, through dot2 (the generic cmul's operations
// for float and double)
__device__ __forceinline__ Cplx<df> cmul(Cplx<df> a, Cplx<df> w) {
  return {dot2(a.x, w.x, -a.y, w.y), dot2(a.x, w.y, a.y, w.x)};
}

// Quotient of a non-negative n < 2^31 by an invariant divisor d >= 1 through
// one 64-bit multiply and a shift -- division by invariant integers using
// multiplication (Granlund and Montgomery, PLDI 1994). With l = ceil(log2 d),
// s = 31 + l and M = ceil(2^s / d) (< 2^32): M d = 2^s + e with 0 <= e < d,
// so n M / 2^s = n / d + n e / (d 2^s), and the last term is below
// n / 2^s < 2^-l <= 1/d, too small to reach the next integer:
// floor(n M / 2^s) = floor(n / d).
struct FastDiv {
  unsigned M;
  int s, d;
  __host__ __device__ __forceinline__ int div(int n) const {
    return (int)(((unsigned long long)(unsigned)n * M) >> s);
  }
  __host__ __device__ __forceinline__ int mod(int n) const { return n - div(n) * d; }
};

inline FastDiv make_fastdiv(int d) {
  FastDiv f;
  f.d = d < 1 ? 1 : d;
  int l = 0;
  while ((1LL << l) < f.d) ++l;
  f.s = 31 + l;
  f.M = (unsigned)(((1ULL << f.s) + (unsigned long long)f.d - 1) / (unsigned long long)f.d);
  return f;
}

// Logical shape of a tensor-product coefficient array: x (direction 1) fastest.
struct Dims {
  int d;
  int m[3];
  long long N;
};

// Per-direction tables consumed by the transform passes (device pointers).
template <typename T>
struct AxisTab {
  int m, n_reg, n_out, p, o, nL, rowsL, nR, rowsR, wlo, whi, kind;
  int gq, gqc, gqe;  // generic transform (kind 2): frequencies gq j - gqe (FWD), gq i - gqc (BWD)
  // L: length of the complex DFT that carries the DST (two pencils per
  // sequence). F: length of the FFT actually run, = L, or, when blu is set, the
  // 5-smooth Bluestein length F >= 2L - 1; shared-memory sequences have stride F.
  int L, F, blu, nst;
  int radix[kMaxStages];  // stages of the length-F FFT
  int twoff[kMaxStages];
  const T* VL;     // rowsL * nL (row-major), left edge block
  const T* VR;     // rowsR * nR (row-major), right edge block in mirrored form:
                   // V_reg[m-1-r][n_reg-1-c] = VR[r][c]
  // interior blocks of V_reg around repeated knots (reduced regularity; nblk
  // = 0 without): 6 ints per block (columns c0..c1-1, rows r0..r1-1, identity
  // offset after the block, offset of its row-major values in VB)
  int nblk;
  const int* blk;
  const T* VB;
  const T* W;      // m * n_out (row-major) = V_out Q_out
  const T* lam;    // m: Lambda_reg then Lambda_out
  const T* post;   // DST-II/III: 4 per k = 0..N/2;  DST-I: n_reg values 1/(2 D~);
                   // generic: w_j/D~_j (2 N), v_i (2 N), 1/D~_j (N)
  const T* tw;     // complex FFT twiddles (interleaved), per stage offsets twoff
  // invariant divisors of the index arithmetic: m, L, F, n_reg, n_reg/2 + 1,
  // n_out, and per FFT stage F / radix and the stage's Ns
  FastDiv fm, fL, fF, fN, fK, fnout;
  FastDiv fnb[kMaxStages], fNs[kMaxStages];
  const T* chirp;  // Bluestein: c_j = exp(i pi j^2 / L), j < L (interleaved)
  const T* bhat;   // Bluestein: DFT_F of the chirp kernel, divided by F
  // FP64 plans, last direction: 1 / (sum of the eigenvalues of all directions)
  // per DoF (same layout as the data), used by the FUSED pass instead of a
  // division; NULL elsewhere.
  const double* rden;
};

// Pencil tiles. The pencils along direction `axis` are numbered q = 0..Q-1:
// for axis 0, q is the row index (the (y, z) pair, y fastest); for axis a > 0,
// q = x + m0 * rest with rest the remaining coordinate (z for axis 1, y for
// axis 2), so consecutive pencils of a tile are consecutive in x (coalesced)
// and a tile may continue across the edge of the x range instead of leaving
// part of a CTA idle. A CTA owns PP consecutive pencils; pencil pc starts at
// pbase[pc] and its entries are pbase[pc] + i * S. ia/ib are the pencil's
// coordinates in the other two directions (x, rest for axis > 0; y, z for
// axis 0). Padding pencils (q >= Q) alias the last pencil and are never stored.
struct TileInfo {
  long long S;
  int nvalid;
};

__device__ __forceinline__ long long num_pencils(const Dims& dims, int axis) { return dims.N / dims.m[axis]; }

__device__ __forceinline__ TileInfo tile_setup(const Dims& dims, int axis, int PP, long long tile, long long* pbase,
                                               int* pia, int* pib) {
  const int m0 = dims.m[0], m1 = dims.m[1];
  const long long Q = num_pencils(dims, axis);
  const long long q0 = tile * PP;
  TileInfo t;
  t.nvalid = (int)min((long long)PP, Q - q0);
  t.S = (axis == 0) ? 1 : ((axis == 1) ? (long long)m0 : (long long)m0 * m1);
  for (int pc = threadIdx.x; pc < PP; pc += blockDim.x) {
    long long q = q0 + pc;
    if (q >= Q) q = Q - 1;
    long long base;
    int ia, ib;
    if (axis == 0) {
      base = q * m0;
      ia = (int)(q % m1);
      ib = (int)(q / m1);
    } else {
      const long long x = q % m0, rest = q / m0;
      ia = (int)x;
      ib = (int)rest;
      base = x + rest * ((axis == 1) ? (long long)m0 * m1 : (long long)m0);
    }
    pbase[pc] = base;
    if (pia) pia[pc] = ia;
    if (pib) pib[pc] = ib;
  }
  return t;
}

inline long long host_num_tiles(const Dims& dims, int axis, int PP) {
  const long long Q = dims.N / dims.m[axis];
  return (Q + PP - 1) / PP;
}

// v or -v without an FP64 (or FP32) instruction: flips the sign bit on the
// integer pipe.
__device__ __forceinline__ double neg_if(double v, bool neg) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)neg << 63));
}
__device__ __forceinline__ float neg_if(float v, bool neg) {
  return __int_as_float(__float_as_int(v) ^ ((int)neg << 31));
}

// Global run status shared by the kernels of one solve (device memory).
struct SolveState {
  double rz, rz_old, pq, rr, ff, alpha, beta, zq;
  int iters, done, status, pad;
};

}  // namespace iffd
