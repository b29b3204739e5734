// Exact Fast Diagonalization (eq. "exact_diagonalization" of the paper):
//   A^{-1} r = (Q_d x .. x Q_1) (sum_k Lambda_k)^{-1} (Q_d^T x .. x Q_1^T) r,
// with dense m x m generalized eigenvector matrices Q_k (Q^T M Q = I). It is the
// comparator of the IFFD preconditioner: every direction costs a dense
// contraction (2 m flops per entry), O(N^{1+1/d}) per apply.
//
// One launch contracts all pencils along one direction with A = Q^T (FWD) or
// A = Q (BWD); FUSED does Q^T, the eigenvalue scaling and Q on the last
// direction. A CTA holds PP pencils in shared memory (32, or 16 where two
// tiles of 32 pencils would not fit: m > ~340) and computes the
// (4 * 256 / (PP / 4)) x PP output blocks of C = A B with a 4 x 4 register
// block per thread, staging 32-column slabs of A through shared memory. FP64
// FMA throughput bounds it.
#include "device_common.cuh"
#include "kernels.h"
#include "fd.h"

namespace iffd {

constexpr int kFdBJ = 32;  // A slab width
// output rows per block for PP pencils per CTA (PP / 4 pencil groups of 4)
template <int PP>
__host__ __device__ constexpr int fd_bi() {
  return 4 * (kThreads / (PP / 4));
}

// C[i][pc] = sum_j A[i][j] * B[pc][j] for the tile (B rows = pencils), in place
// into Cout (separate smem array).
template <int PP>
__device__ void fd_contract(const double* __restrict__ A, int m, const double* Bt, int ldb, double* Ct,
                            double* As) {
  constexpr int kFdBI = fd_bi<PP>();
  constexpr int TP = PP / 4;
  const int tid = threadIdx.x;
  const int ti = tid / TP;        // rows 4*ti .. 4*ti+3
  const int tp = tid % TP;        // pencils 4*tp .. 4*tp+3
  for (int i0 = 0; i0 < m; i0 += kFdBI) {
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int j0 = 0; j0 < m; j0 += kFdBJ) {
      __syncthreads();
      // stage A[i0 .. i0+127][j0 .. j0+31] as As[jj][ii] (ii fastest)
      for (int e = tid; e < kFdBI * kFdBJ; e += blockDim.x) {
        const int ii = e / kFdBJ, jj = e - ii * kFdBJ;
        const int i = i0 + ii, j = j0 + jj;
        As[jj * (kFdBI + 1) + ii] = (i < m && j < m) ? __ldg(A + (size_t)i * m + j) : 0.0;
      }
      __syncthreads();
      const int jn = min(kFdBJ, m - j0);
      for (int jj = 0; jj < jn; ++jj) {
        double a[4], b[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = As[jj * (kFdBI + 1) + 4 * ti + r];
#pragma unroll
        for (int c = 0; c < 4; ++c) b[c] = Bt[(4 * tp + c) * ldb + j0 + jj];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = i0 + 4 * ti + r;
      if (i < m) {
#pragma unroll
        for (int c = 0; c < 4; ++c) Ct[(4 * tp + c) * ldb + i] = acc[r][c];
      }
    }
  }
  __syncthreads();
}

template <int MODE, int kFdPP>
__global__ void __launch_bounds__(kThreads)
fd_pass(const double* in, double* out, Dims dims, int axis, int ldb, const double* __restrict__ QT,
        const double* __restrict__ Q, const double* __restrict__ lam, const double* __restrict__ lamA,
        const double* __restrict__ lamB, const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int m = dims.m[axis];
  double* B = reinterpret_cast<double*>(smem);
  double* C = B + (size_t)kFdPP * ldb;
  double* As = C + (size_t)kFdPP * ldb;
  __shared__ long long pbase[kFdPP];
  __shared__ int pia[kFdPP], pib[kFdPP];
  const TileInfo g = tile_setup(dims, axis, kFdPP, blockIdx.x, pbase, pia, pib);
  __syncthreads();
  for (int e = threadIdx.x; e < kFdPP * m; e += blockDim.x) {
    int pc, i;
    if (axis == 0) { pc = e / m; i = e - pc * m; }
    else { i = e / kFdPP; pc = e - i * kFdPP; }
    B[pc * ldb + i] = in[pbase[pc] + i * g.S];
  }
  __syncthreads();
  double* res = B;
  if (MODE == PM_FWD || MODE == PM_FUSED) {
    fd_contract<kFdPP>(QT, m, B, ldb, C, As);
    res = C;
  }
  if (MODE == PM_FUSED) {
    for (int e = threadIdx.x; e < kFdPP * m; e += blockDim.x) {
      const int pc = e / m, i = e - pc * m;
      if (pc >= g.nvalid) continue;  // padding pencils
      double den = __ldg(lam + i) + __ldg(lamA + pia[pc]);
      if (dims.d == 3) den += __ldg(lamB + pib[pc]);
      C[pc * ldb + i] = C[pc * ldb + i] / den;
    }
    __syncthreads();
    fd_contract<kFdPP>(Q, m, C, ldb, B, As);
    res = B;
  }
  if (MODE == PM_BWD) {
    fd_contract<kFdPP>(Q, m, B, ldb, C, As);
    res = C;
  }
  for (int e = threadIdx.x; e < kFdPP * m; e += blockDim.x) {
    int pc, i;
    if (axis == 0) { pc = e / m; i = e - pc * m; }
    else { i = e / kFdPP; pc = e - i * kFdPP; }
    if (pc < g.nvalid) out[pbase[pc] + i * g.S] = res[pc * ldb + i];
  }
}

static size_t fd_smem_pp(int m, int PP) {
  const int ldb = m | 1;
  const int bi = 4 * (kThreads / (PP / 4));
  return (size_t)2 * PP * ldb * sizeof(double) + (size_t)kFdBJ * (bi + 1) * sizeof(double);
}

// 32 pencils per CTA while two tiles fit in 200 KB of shared memory, else 16
static int fd_pp(int m) { return fd_smem_pp(m, 32) <= 200 * 1024 ? 32 : 16; }

int fd_tiles(const Dims& dims, int axis) {
  return (int)host_num_tiles(dims, axis, fd_pp(dims.m[axis]));
}

size_t fd_smem(int m) { return fd_smem_pp(m, fd_pp(m)); }

template <int MODE, int PP>
static cudaError_t launch_fd_t(const double* in, double* out, const Dims& dims, int axis, const double* QT,
                               const double* Q, const double* lam, const double* lamA, const double* lamB,
                               const int* done, cudaStream_t st) {
  const int m = dims.m[axis];
  const int ldb = m | 1;
  const size_t sm = fd_smem_pp(m, PP);
  const int tiles = (int)host_num_tiles(dims, axis, PP);
  cudaError_t e = cudaFuncSetAttribute(fd_pass<MODE, PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  fd_pass<MODE, PP><<<tiles, kThreads, sm, st>>>(in, out, dims, axis, ldb, QT, Q, lam, lamA, lamB, done);
  return cudaGetLastError();
}

cudaError_t launch_fd_pass(int mode, const double* in, double* out, const Dims& dims, int axis,
                           const double* QT, const double* Q, const double* lam, const double* lamA,
                           const double* lamB, const int* done, cudaStream_t st) {
  const bool big = fd_pp(dims.m[axis]) == 16;
  if (mode == PM_FWD)
    return big ? launch_fd_t<PM_FWD, 16>(in, out, dims, axis, QT, Q, lam, lamA, lamB, done, st)
               : launch_fd_t<PM_FWD, 32>(in, out, dims, axis, QT, Q, lam, lamA, lamB, done, st);
  if (mode == PM_BWD)
    return big ? launch_fd_t<PM_BWD, 16>(in, out, dims, axis, QT, Q, lam, lamA, lamB, done, st)
               : launch_fd_t<PM_BWD, 32>(in, out, dims, axis, QT, Q, lam, lamA, lamB, done, st);
  return big ? launch_fd_t<PM_FUSED, 16>(in, out, dims, axis, QT, Q, lam, lamA, lamB, done, st)
             : launch_fd_t<PM_FUSED, 32>(in, out, dims, axis, QT, Q, lam, lamA, lamB, done, st);
}

}  // namespace iffd
