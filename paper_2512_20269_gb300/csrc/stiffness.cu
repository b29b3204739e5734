// Kronecker stiffness apply (eq. "system_matrix", written for d directions):
//   A^ u = sum_k (M x .. x K_k x .. x M) u,
// factorised into one banded (2p+1) sweep per direction (3D):
//   slowest direction z:  T1 = M_z u,           T2 = K_z u
//   direction y:          T1 <- M_y T1,        T2 <- K_y T1 + M_y T2
//   direction x:          A^ u = K_x T1 + M_x T2
// (2D: the first stage runs on y and the last on x.) Seven banded products in
// 3D, four in 2D. Interior rows of M and K are symmetric Toeplitz (uniform
// knots), so one set of pair sums u_{i-k} + u_{i+k} feeds both M and K; the
// boundary rows (2p-1 at a Dirichlet end, 2p at a natural end) use the stored band.
#include "device_common.cuh"
#include "kernels.h"
#include "stiff_dev.cuh"

namespace iffd {

int stiff_tiles(const Dims& dims, int axis, int PP) { return (int)host_num_tiles(dims, axis, PP); }

template <int P>
__global__ void __launch_bounds__(kThreads)
stiff_first(Dims dims, int axis, int PP, int ldt, BandTab bt, const double* __restrict__ u,
            const double* __restrict__ z, double* __restrict__ p_io, const double* __restrict__ betap, int pmode,
            double* __restrict__ T1, double* __restrict__ T2, const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  first_body<P>(dims, axis, PP, ldt, bt, u, z, p_io, betap, pmode, T1, T2, blockIdx.x, smem);
}

template <int P>
__global__ void __launch_bounds__(kThreads)
stiff_mid(Dims dims, int axis, int PP, int ldt, BandTab bt, double* __restrict__ T1, double* __restrict__ T2,
          const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  mid_body<P>(dims, axis, PP, ldt, bt, T1, T2, blockIdx.x, smem);
}

template <int P>
__global__ void __launch_bounds__(kThreads)
stiff_last(Dims dims, int axis, int PP, int ldt, BandTab bt, const double* __restrict__ T1,
           const double* __restrict__ T2, double* __restrict__ out, const double* __restrict__ dotv,
           double* __restrict__ partial, const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  last_body<P>(dims, axis, PP, ldt, bt, T1, T2, out, dotv, partial, blockIdx.x, blockIdx.x, smem);
}

// Batched sweep over many systems of the same degree P (see precond_pass_batched).
template <int P, int STAGE>
__global__ void __launch_bounds__(kThreads)
stiff_batched(const StiffDesc* __restrict__ sys, const long long* __restrict__ tile_prefix, int nsys) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ StiffDesc sd;
  __shared__ int s_sys;
  if (threadIdx.x == 0) {
    const long long b = blockIdx.x;
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile_prefix[mid] <= b) lo = mid;
      else hi = mid - 1;
    }
    s_sys = lo;
    sd = sys[lo];
  }
  __syncthreads();
  if (sd.done != nullptr && *((volatile const int*)sd.done)) return;
  const long long tile = (long long)blockIdx.x - tile_prefix[s_sys];
  if (STAGE == SS_FIRST)
    first_body<P>(sd.dims, sd.axis, sd.PP, sd.ldt, sd.bt, sd.u, sd.z, sd.p_io, sd.beta, sd.pmode, sd.T1, sd.T2,
                  tile, smem);
  else if (STAGE == SS_MID)
    mid_body<P>(sd.dims, sd.axis, sd.PP, sd.ldt, sd.bt, sd.T1, sd.T2, tile, smem);
  else
    last_body<P>(sd.dims, sd.axis, sd.PP, sd.ldt, sd.bt, sd.T1, sd.T2, sd.out, sd.dotv, sd.partial, tile, (int)tile,
                 smem);
}

static size_t stiff_smem(const StiffLaunch& S, int arrays) { return (size_t)arrays * S.PP * S.ldt * sizeof(double); }

template <int P>
static cudaError_t first_p(const StiffLaunch& S, const double* u, const double* z, double* p_io, const double* beta,
                           int pmode, double* T1, double* T2, const int* done, cudaStream_t st) {
  const size_t sm = stiff_smem(S, 1);
  cudaError_t e = cudaFuncSetAttribute(stiff_first<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  stiff_first<P><<<stiff_tiles(S.dims, S.axis, S.PP), kThreads, sm, st>>>(S.dims, S.axis, S.PP, S.ldt, S.bt, u, z,
                                                                          p_io, beta, pmode, T1, T2, done);
  return cudaGetLastError();
}

template <int P>
static cudaError_t mid_p(const StiffLaunch& S, double* T1, double* T2, const int* done, cudaStream_t st) {
  const size_t sm = stiff_smem(S, 2);
  cudaError_t e = cudaFuncSetAttribute(stiff_mid<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  stiff_mid<P><<<stiff_tiles(S.dims, S.axis, S.PP), kThreads, sm, st>>>(S.dims, S.axis, S.PP, S.ldt, S.bt, T1, T2,
                                                                        done);
  return cudaGetLastError();
}

template <int P>
static cudaError_t last_p(const StiffLaunch& S, const double* T1, const double* T2, double* out, const double* dotv,
                          double* partial, const int* done, cudaStream_t st) {
  const size_t sm = stiff_smem(S, 2);
  cudaError_t e = cudaFuncSetAttribute(stiff_last<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  stiff_last<P><<<stiff_tiles(S.dims, S.axis, S.PP), kThreads, sm, st>>>(S.dims, S.axis, S.PP, S.ldt, S.bt, T1, T2,
                                                                         out, dotv, partial, done);
  return cudaGetLastError();
}

#define IFFD_DISPATCH_P(p, CALL)                                   \
  switch (p) {                                                     \
    case 1: return CALL(1); case 2: return CALL(2);                \
    case 3: return CALL(3); case 4: return CALL(4);                \
    case 5: return CALL(5); case 6: return CALL(6);                \
    case 7: return CALL(7); case 8: return CALL(8);                \
    case 9: return CALL(9); case 10: return CALL(10);              \
    case 11: return CALL(11); case 12: return CALL(12);            \
    case 13: return CALL(13); case 14: return CALL(14);            \
    case 15: return CALL(15); case 16: return CALL(16);            \
    default: return cudaErrorInvalidValue;                         \
  }

template <int P>
static cudaError_t batched_p(int stage, const StiffDesc* sys, const long long* tile_prefix, int nsys,
                             long long total_tiles, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (stage == SS_FIRST) {
    static size_t set_SS_FIRST = 0;
    if (smem > set_SS_FIRST) {
      e = cudaFuncSetAttribute(stiff_batched<P, SS_FIRST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      set_SS_FIRST = smem;
    }
    if (total_tiles <= 0) return cudaSuccess;
    stiff_batched<P, SS_FIRST><<<(unsigned)total_tiles, kThreads, smem, st>>>(sys, tile_prefix, nsys);
  } else if (stage == SS_MID) {
    static size_t set_SS_MID = 0;
    if (smem > set_SS_MID) {
      e = cudaFuncSetAttribute(stiff_batched<P, SS_MID>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      set_SS_MID = smem;
    }
    if (total_tiles <= 0) return cudaSuccess;
    stiff_batched<P, SS_MID><<<(unsigned)total_tiles, kThreads, smem, st>>>(sys, tile_prefix, nsys);
  } else {
    static size_t set_SS_LAST = 0;
    if (smem > set_SS_LAST) {
      e = cudaFuncSetAttribute(stiff_batched<P, SS_LAST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      set_SS_LAST = smem;
    }
    if (total_tiles <= 0) return cudaSuccess;
    stiff_batched<P, SS_LAST><<<(unsigned)total_tiles, kThreads, smem, st>>>(sys, tile_prefix, nsys);
  }
  return cudaGetLastError();
}

cudaError_t launch_stiff_batched(int p, int stage, const StiffDesc* sys, const long long* tile_prefix, int nsys,
                                 long long total_tiles, size_t smem, cudaStream_t st) {
#define CALL_B(P) batched_p<P>(stage, sys, tile_prefix, nsys, total_tiles, smem, st)
  IFFD_DISPATCH_P(p, CALL_B)
#undef CALL_B
}

cudaError_t launch_stiff_first(const StiffLaunch& S, const double* u, const double* z, double* p_io,
                               const double* beta, int pmode, double* T1, double* T2, const int* done,
                               cudaStream_t st) {
#define CALL_FIRST(P) first_p<P>(S, u, z, p_io, beta, pmode, T1, T2, done, st)
  IFFD_DISPATCH_P(S.bt.p, CALL_FIRST)
#undef CALL_FIRST
}

cudaError_t launch_stiff_mid(const StiffLaunch& S, double* T1, double* T2, const int* done, cudaStream_t st) {
#define CALL_MID(P) mid_p<P>(S, T1, T2, done, st)
  IFFD_DISPATCH_P(S.bt.p, CALL_MID)
#undef CALL_MID
}

cudaError_t launch_stiff_last(const StiffLaunch& S, const double* T1, const double* T2, double* out,
                              const double* dotv, double* partial, const int* done, cudaStream_t st) {
#define CALL_LAST(P) last_p<P>(S, T1, T2, out, dotv, partial, done, st)
  IFFD_DISPATCH_P(S.bt.p, CALL_LAST)
#undef CALL_LAST
}

}  // namespace iffd
