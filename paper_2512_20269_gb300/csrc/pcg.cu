// PCG vector kernels and deterministic reductions (Section 3 of the paper;
// zero initial guess and relative-residual stopping rule of Section 7).
//
// Every kernel writes one partial sum per CTA; `finalize` reduces them in a
// fixed order (one CTA, fixed tree), so a solve is bitwise reproducible for a
// given problem shape. All scalars of the iteration live in device memory
// (SolveState) and every kernel returns immediately once `done` is set, so the
// host can enqueue iterations ahead without synchronising.
#include "device_common.cuh"
#include "kernels.h"
#include "pcg_dev.cuh"

namespace iffd {

int vec_grid(long long N) {
  long long g = (N + 1023) / 1024;
  const long long cap = 4LL * device_sm_count();  // four 256-thread CTAs per SM
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

__global__ void __launch_bounds__(kThreads)
pcg_init(const double* __restrict__ f, double* __restrict__ x, double* __restrict__ r, long long N,
         double* __restrict__ partial, SolveState* __restrict__ state) {
  // the solve state starts from zero (a kernel store rather than a memset
  // node, which in a captured graph can queue behind the caller's copies)
  if (state != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *state = SolveState{};
  init_body(f, x, r, N, partial, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kThreads)
pcg_update(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p, const double* __restrict__ q,
           const SolveState* __restrict__ st, long long N, double* __restrict__ partial, const int* __restrict__ done) {
  if (*((volatile const int*)done)) return;
  update_body(x, r, p, q, st, N, partial, blockIdx.x, gridDim.x);
}

// Batched vector kernels: block b serves local block b - block_prefix[s] of
// system s (which has vec_grid(N_s) blocks, as when solved alone).
__device__ __forceinline__ int find_system(const long long* __restrict__ prefix, int nsys, long long b) {
  int lo = 0, hi = nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kThreads)
pcg_init_batched(const VecDesc* __restrict__ sys, const long long* __restrict__ prefix, int nsys) {
  const int s = find_system(prefix, nsys, blockIdx.x);
  const VecDesc& d = sys[s];
  const int blk = (int)(blockIdx.x - prefix[s]);
  const int nblk = (int)(prefix[s + 1] - prefix[s]);
  if (blk == 0 && threadIdx.x == 0) *d.st = SolveState{};
  init_body(d.f, d.x, d.r, d.N, d.part_rr, blk, nblk);
  if (d.p_zero != nullptr)
    for (long long i = blk * (long long)blockDim.x + threadIdx.x; i < d.N; i += (long long)nblk * blockDim.x)
      d.p_zero[i] = 0.0;
}

// Copies the solve state of every system into one array (one D2H copy).
__global__ void gather_states(SolveState* const* __restrict__ src, SolveState* __restrict__ dst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = *src[i];
}

cudaError_t launch_gather_states(SolveState* const* src, SolveState* dst, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  gather_states<<<(n + 127) / 128, 128, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kThreads)
pcg_update_batched(const VecDesc* __restrict__ sys, const long long* __restrict__ prefix, int nsys) {
  const int s = find_system(prefix, nsys, blockIdx.x);
  const VecDesc& d = sys[s];
  if (*((volatile const int*)&d.st->done)) return;
  const int blk = (int)(blockIdx.x - prefix[s]);
  const int nblk = (int)(prefix[s + 1] - prefix[s]);
  update_body(d.x, d.r, d.p, d.q, d.st, d.N, d.part_rr, blk, nblk);
}

// partial ||f - Au||^2
__global__ void __launch_bounds__(kThreads)
residual_kernel(const double* __restrict__ f, const double* __restrict__ Au, long long N, double* __restrict__ partial) {
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double d = f[i] - Au[i];
    s = fma(d, d, s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024)
finalize_kernel(SolveState* st, const double* __restrict__ partial, int nparts, int phase, double tol2, int maxit) {
  finalize_body(st, partial, nparts, phase, tol2, maxit);
}

// One CTA per system; the reduction order equals finalize_kernel's.
__global__ void __launch_bounds__(1024)
finalize_batched(const FinDesc* __restrict__ sys, int phase, double tol2, int maxit) {
  const FinDesc& d = sys[blockIdx.x];
  finalize_body(d.st, d.partial, d.nparts, phase, tol2, maxit);
}

cudaError_t launch_pcg_init(const double* f, double* x, double* r, long long N, double* partial, cudaStream_t st,
                            SolveState* state) {
  pcg_init<<<vec_grid(N), kThreads, 0, st>>>(f, x, r, N, partial, state);
  return cudaGetLastError();
}

cudaError_t launch_pcg_update(double* x, double* r, const double* p, const double* q, const SolveState* s,
                              long long N, double* partial, const int* done, cudaStream_t st) {
  pcg_update<<<vec_grid(N), kThreads, 0, st>>>(x, r, p, q, s, N, partial, done);
  return cudaGetLastError();
}

cudaError_t launch_residual(const double* f, const double* Au, long long N, double* partial, cudaStream_t st) {
  residual_kernel<<<vec_grid(N), kThreads, 0, st>>>(f, Au, N, partial);
  return cudaGetLastError();
}

cudaError_t launch_pcg_init_batched(const VecDesc* sys, const long long* prefix, int nsys, long long total_blocks,
                                    cudaStream_t st) {
  pcg_init_batched<<<(unsigned)total_blocks, kThreads, 0, st>>>(sys, prefix, nsys);
  return cudaGetLastError();
}

cudaError_t launch_pcg_update_batched(const VecDesc* sys, const long long* prefix, int nsys, long long total_blocks,
                                      cudaStream_t st) {
  pcg_update_batched<<<(unsigned)total_blocks, kThreads, 0, st>>>(sys, prefix, nsys);
  return cudaGetLastError();
}

cudaError_t launch_finalize_batched(const FinDesc* sys, int nsys, int phase, double tol2, int maxit, cudaStream_t st) {
  finalize_batched<<<nsys, 1024, 0, st>>>(sys, phase, tol2, maxit);
  return cudaGetLastError();
}

cudaError_t launch_finalize(SolveState* s, const double* partial, int nparts, int phase, double tol2, int maxit,
                            cudaStream_t st) {
  finalize_kernel<<<1, 1024, 0, st>>>(s, partial, nparts, phase, tol2, maxit);
  return cudaGetLastError();
}

}  // namespace iffd
