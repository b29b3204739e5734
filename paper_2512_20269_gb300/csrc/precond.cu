// IFFD preconditioner passes (eq. "preconditioner" of the paper):
//   P^{-1} r = (Q~_d x .. x Q~_1) (sum_k Lambda~_k)^{-1} (Q~_d^T x .. x Q~_1^T) r,
//   Q~ = [V_reg U_reg D~^{-1}, V_out Q_out]   (Sections 4 and 6).
//
// One kernel launch applies Q~^T (FWD), Q~ (BWD), or Q~^T, the eigenvalue
// scaling and Q~ (FUSED, used on the last direction) to every pencil along one
// direction. A CTA owns a tile of PP pencils: it loads them (coalesced along x)
// into shared memory and, per pencil pair, runs
//   FWD: remainder projections y_out = W^T r (W = V_out Q_out), the V_reg^T edge
//        gather, Makhoul's reordering, a two-for-one complex Stockham FFT of
//        length L and the separation / twiddle / D~^{-1} step, giving
//        [D~^{-1} U^T V_reg^T r | Q_out^T V_out^T r];
//   BWD: the transpose of the same steps (DST-III for even p, DST-I for odd p,
//        Table 1) followed by the V_reg edge scatter and the rank-n_out update
//        V_out Q_out z_out.
// All arithmetic is in Tc (double, or float for the reduced-precision
// transform variant); Tin/Tout are the global storage types.
#include <cuda_pipeline.h>

#include <algorithm>

#include <type_traits>

#include "device_common.cuh"
#include "kernels.h"
#include "precond_block.cuh"
#include "precond_dev.cuh"
#include "precond_warp_geom.h"

namespace iffd {

template <typename Tc, typename Tin, typename Tout, int MODE, int NDOT>
__global__ void __launch_bounds__(kThreads)
precond_pass(const Tin* in, Tout* out, Dims dims, int axis, int PP, int ldt, AxisTab<Tc> ax,
             const Tc* __restrict__ lamA, const Tc* __restrict__ lamB,
             const double* __restrict__ dotv0, const double* __restrict__ dotv1,
             double* __restrict__ partial, const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  precond_body<Tc, Tin, Tout, MODE, NDOT>(in, out, dims, axis, PP, ldt, ax, lamA, lamB, dotv0, dotv1, partial,
                                          blockIdx.x, blockIdx.x, gridDim.x, smem);
}

// Asynchronous tile load: one cp.async element copy per DoF (padding pencils
// are written as zeros); the caller commits the copy group.
template <typename Tc>
__device__ __forceinline__ void load_tile_async(const Tc* __restrict__ in, Tc* tile, int axis, int PP, int ldt,
                                                const AxisTab<Tc>& ax, const long long* pbase, const TileInfo& g) {
  const int lpp = 31 - __clz(PP);
  const int m = ax.m;
  for (int e = threadIdx.x; e < PP * m; e += blockDim.x) {
    int pc, i;
    if (axis == 0) { pc = ax.fm.div(e); i = e - pc * m; }
    else { i = e >> lpp; pc = e & (PP - 1); }
    Tc* dst = tile + pc * ldt + i;
    if (pc < g.nvalid) __pipeline_memcpy_async(dst, in + pbase[pc] + i * g.S, sizeof(Tc));
    else *dst = Tc(0);
  }
}

// Persistent transform pass with a two-stage pipeline: each CTA walks the
// tiles t = blockIdx.x, + gridDim.x, ...; while it transforms tile t the
// copies of its next tile are already in flight into the second tile buffer.
// Same arithmetic and partial sums as precond_pass (only the loading differs).
template <typename Tc, int MODE, int NDOT>
__global__ void __launch_bounds__(kThreads)
precond_pass_pipe(const Tc* in, Tc* out, Dims dims, int axis, int PP, int ldt, AxisTab<Tc> ax,
                  const Tc* __restrict__ lamA, const Tc* __restrict__ lamB, const double* __restrict__ dotv0,
                  const double* __restrict__ dotv1, double* __restrict__ partial, int ntiles,
                  const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int npairs = PP / 2, F = ax.F;
  Cplx<Tc>* bufA = reinterpret_cast<Cplx<Tc>*>(smem);
  Cplx<Tc>* bufB = bufA + (size_t)npairs * F;
  Tc* tiles = reinterpret_cast<Tc*>(bufB + (size_t)npairs * F);  // two tile buffers
  Tc* outv = tiles + (size_t)2 * PP * ldt;                          // PP * kMaxNout
  __shared__ long long pbase[2][64];
  __shared__ int pia[2][64], pib[2][64];
  int t = blockIdx.x;
  if (t >= ntiles) return;  // the same for every thread of the CTA
  TileInfo g = tile_setup(dims, axis, PP, t, pbase[0], pia[0], pib[0]);
  __syncthreads();
  load_tile_async<Tc>(in, tiles, axis, PP, ldt, ax, pbase[0], g);
  __pipeline_commit();
  int cur = 0;
  for (; t < ntiles; t += gridDim.x) {
    const int tn = t + gridDim.x;
    const int nx = cur ^ 1;
    TileInfo gn = g;
    if (tn < ntiles) gn = tile_setup(dims, axis, PP, tn, pbase[nx], pia[nx], pib[nx]);
    __syncthreads();  // pbase[nx] written
    if (tn < ntiles) load_tile_async<Tc>(in, tiles + (size_t)nx * PP * ldt, axis, PP, ldt, ax, pbase[nx], gn);
    __pipeline_commit();
    __pipeline_wait_prior(1);  // this thread's copies of tile t have landed
    __syncthreads();           // and every thread's
    Tc* tile = tiles + (size_t)cur * PP * ldt;
    compute_tile<Tc, MODE>(tile, bufA, bufB, outv, dims, axis, PP, ldt, ax, lamA, lamB, pbase[cur], pia[cur],
                           pib[cur], g);
    store_tile<Tc, Tc, NDOT>(tile, out, axis, PP, ldt, ax, pbase[cur], g, dotv0, dotv1, partial, t, ntiles);
    __syncthreads();  // tile buffer and pbase of `cur` are free for tile t + 2 gridDim.x
    g = gn;
    cur = nx;
  }
  __pipeline_wait_prior(0);
}

// Batched pass: the grid covers the tiles of many independent systems; CTA b
// serves tile b - tile_prefix[s] of system s with tile_prefix[s] <= b <
// tile_prefix[s+1]. Each system's work and reductions are exactly those of the
// single-system kernel, so a result does not depend on the rest of the batch.
template <typename Tc, typename Tin, typename Tout, int MODE, int NDOT>
__global__ void __launch_bounds__(kThreads)
precond_pass_batched(const PassDesc<Tc, Tin, Tout>* __restrict__ sys, const long long* __restrict__ tile_prefix,
                     int nsys) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ PassDesc<Tc, Tin, Tout> sd;
  __shared__ int s_sys;
  if (threadIdx.x == 0) {
    const long long b = blockIdx.x;
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {  // last s with tile_prefix[s] <= b
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
  const int ntiles = (int)(tile_prefix[s_sys + 1] - tile_prefix[s_sys]);
  precond_body<Tc, Tin, Tout, MODE, NDOT>(sd.in, sd.out, sd.dims, sd.axis, sd.PP, sd.ldt, sd.ax, sd.lamA, sd.lamB,
                                          sd.dot0, sd.dot1, sd.partial, tile, (int)tile, ntiles, smem);
}

// rden[x + m0 (y + m1 z)] = 1 / (lam_F[i_F] + lam_0[x] (+ lam_1[y])): the
// reciprocal of the summed eigenvalues, added in the order of the FUSED pass
// (last direction F = d-1 first, then direction 0, then direction 1).
__global__ void rden_fill(double* __restrict__ rden, Dims dims, const double* __restrict__ lamF,
                          const double* __restrict__ lam0, const double* __restrict__ lam1) {
  const long long m0 = dims.m[0], m1 = dims.m[1];
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < dims.N;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long x = idx % m0, rest = idx / m0;
    double den;
    if (dims.d == 3) den = (__ldg(lamF + rest / m1) + __ldg(lam0 + x)) + __ldg(lam1 + rest % m1);
    else den = __ldg(lamF + rest) + __ldg(lam0 + x);
    rden[idx] = 1.0 / den;
  }
}

cudaError_t launch_rden_fill(double* rden, const Dims& dims, const double* lamF, const double* lam0,
                             const double* lam1, cudaStream_t st) {
  long long g = (dims.N + kThreads - 1) / kThreads;
  if (g > 8 * 152) g = 8 * 152;
  rden_fill<<<(unsigned)g, kThreads, 0, st>>>(rden, dims, lamF, lam0, lam1);
  return cudaGetLastError();
}

// ------------------------------------------------------------ host launchers
// F: FFT length (stride of a sequence); two ping-pong buffers of PP/2 complex
// sequences, the tile and the remainder coefficients.
size_t precond_smem_bytes(int PP, int ldt, int F, size_t elt) {
  return (size_t)2 * (PP / 2) * F * 2 * elt + (size_t)PP * ldt * elt + (size_t)PP * kMaxNout * elt;
}

int precond_tiles(const Dims& dims, int axis, int PP) { return (int)host_num_tiles(dims, axis, PP); }

int device_sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 152;
  }
  return n;
}

size_t precond_smem_bytes_pipe(int PP, int ldt, int F, size_t elt) {
  return precond_smem_bytes(PP, ldt, F, elt) + (size_t)PP * ldt * elt;
}

template <typename Tc, int MODE, int NDOT>
static cudaError_t launch_pipe_t(const PassLaunch<Tc>& P, const Tc* in, Tc* out, cudaStream_t st) {
  auto kern = precond_pass_pipe<Tc, MODE, NDOT>;
  const size_t sm = precond_smem_bytes_pipe(P.PP, P.ldt, P.ax.F, sizeof(Tc));
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int tiles = precond_tiles(P.dims, P.axis, P.PP);
  const int grid = std::min(tiles, per_sm * device_sm_count());
  kern<<<grid, kThreads, sm, st>>>(in, out, P.dims, P.axis, P.PP, P.ldt, P.ax, P.lamA, P.lamB, P.dot0, P.dot1,
                                   P.partial, tiles, P.done);
  return cudaGetLastError();
}

template <typename T>
static int wpass_len_t(const AxisTab<T>& ax, int nmax) {
  int N = 0;
  if (ax.kind == 1) N = ax.n_reg;                 // DST-II/III: Makhoul, length n_reg
  else if (ax.kind == 0) N = 2 * (ax.n_reg + 1);  // DST-I: odd extension
  else return 0;
  if (ax.blu || ax.L != N || ax.F != N || N > nmax || ax.m > N + kMaxNout) return 0;
  return (N == 64 || N == 128 || N == 256 || N == 512) ? N : 0;
}
int wpass_len(const AxisTab<float>& ax) { return wpass_len_t(ax, 512); }
// FP64: a length-512 tile (141 KB of shared memory) would leave one CTA per SM
int wpass_len(const AxisTab<double>& ax) { return wpass_len_t(ax, 256); }
int wpass_len(const AxisTab<df>& ax) { return wpass_len_t(ax, 256); }

template <typename Tc, typename Tin, typename Tout, int MODE, int NDOT>
cudaError_t launch_pass_t(const PassLaunch<Tc>& P, const Tin* in, Tout* out, cudaStream_t st);

template <typename Tin, typename Tout>
cudaError_t launch_pass_df(const PassLaunch<df>& P, int mode, int ndot, const Tin* in, Tout* out, cudaStream_t st) {
  if (P.wN == 0) {  // the block kernel (the combinations the preconditioner uses)
    if (P.ax.blu || P.pipe) return cudaErrorInvalidValue;
    if constexpr (std::is_same<Tin, double>::value) {
      if (mode != PM_FWD) return cudaErrorInvalidValue;
      return launch_pass_t<df, double, df, PM_FWD, 0>(P, in, out, st);
    } else if constexpr (std::is_same<Tout, double>::value) {
      if (mode != PM_BWD) return cudaErrorInvalidValue;
      if (ndot == 0) return launch_pass_t<df, df, double, PM_BWD, 0>(P, in, out, st);
      if (ndot == 1) return launch_pass_t<df, df, double, PM_BWD, 1>(P, in, out, st);
      return launch_pass_t<df, df, double, PM_BWD, 2>(P, in, out, st);
    } else {
      if (ndot != 0) return cudaErrorInvalidValue;
      if (mode == PM_FWD) return launch_pass_t<df, df, df, PM_FWD, 0>(P, in, out, st);
      if (mode == PM_FUSED) return launch_pass_t<df, df, df, PM_FUSED, 0>(P, in, out, st);
      return launch_pass_t<df, df, df, PM_BWD, 0>(P, in, out, st);
    }
  }
  if (P.PP != wpass_pencils(P.wN) || P.ldt < wpass_ldt(P.wN, P.ax.m, true)) return cudaErrorInvalidConfiguration;
  switch (P.wN) {
    case 64: return launch_wpass<64, df, Tin, Tout>(P, mode, ndot, in, out, st);
    case 128: return launch_wpass<128, df, Tin, Tout>(P, mode, ndot, in, out, st);
    case 256: return launch_wpass<256, df, Tin, Tout>(P, mode, ndot, in, out, st);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_pass_df<double, df>(const PassLaunch<df>&, int, int, const double*, df*, cudaStream_t);
template cudaError_t launch_pass_df<df, df>(const PassLaunch<df>&, int, int, const df*, df*, cudaStream_t);
template cudaError_t launch_pass_df<df, double>(const PassLaunch<df>&, int, int, const df*, double*, cudaStream_t);

int wpass_pencils(int N, bool pair) {
  switch (N) {
    case 64: return pair ? warp_pencils<64, true>() : warp_pencils<64>();
    case 128: return pair ? warp_pencils<128, true>() : warp_pencils<128>();
    case 256: return pair ? warp_pencils<256, true>() : warp_pencils<256>();
    default: return warp_pencils<512>();
  }
}

// tile (PP pencil rows of ldt values), PP / 2 sequence buffers of wpad(N)
// complex values (none with alias: they live in the pairs' rows) and PP rows
// of kMaxNout remainder coefficients -- for the paired pass the same bytes
// per pencil (rows and buffers hold two pencils' or two sequences' values)
size_t wpass_smem_bytes(int N, int ldt, size_t elt, bool pair, bool alias) {
  const int PP = wpass_pencils(N, pair);
  return (size_t)PP * ldt * elt + (alias ? 0 : (size_t)(PP / 2) * wpad(N) * 2 * elt) +
         (size_t)PP * kMaxNout * elt;
}

int wpass_ldt(int N, int m, bool alias) { return (alias ? std::max(m, wbuf_len_host(N)) : m) | 1; }

template <typename Tc, typename Tin, typename Tout, int MODE, int NDOT>
cudaError_t launch_pass_t(const PassLaunch<Tc>& P, const Tin* in, Tout* out, cudaStream_t st) {
  if (P.wN != 0) {
    if (P.PP != wpass_pencils(P.wN, P.pair != 0) || P.ldt < wpass_ldt(P.wN, P.ax.m, false))
      return cudaErrorInvalidConfiguration;
    switch (P.wN) {
      case 64: return launch_wpass<64, Tc, Tin, Tout>(P, MODE, NDOT, in, out, st);
      case 128: return launch_wpass<128, Tc, Tin, Tout>(P, MODE, NDOT, in, out, st);
      case 256: return launch_wpass<256, Tc, Tin, Tout>(P, MODE, NDOT, in, out, st);
      case 512:
        if constexpr (std::is_same<Tc, float>::value) return launch_wpass<512, Tc, Tin, Tout>(P, MODE, NDOT, in, out, st);
        else return cudaErrorInvalidValue;
      default: return cudaErrorInvalidValue;
    }
  }
  if constexpr (std::is_same<Tin, Tc>::value && std::is_same<Tout, Tc>::value && !std::is_same<Tc, df>::value) {
    if (P.pipe) return launch_pipe_t<Tc, MODE, NDOT>(P, in, out, st);
  }
  auto kern = precond_pass<Tc, Tin, Tout, MODE, NDOT>;
  const size_t sm = precond_smem_bytes(P.PP, P.ldt, P.ax.F, sizeof(Tc));
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int tiles = precond_tiles(P.dims, P.axis, P.PP);
  kern<<<tiles, kThreads, sm, st>>>(in, out, P.dims, P.axis, P.PP, P.ldt, P.ax, P.lamA, P.lamB, P.dot0,
                                     P.dot1, P.partial, P.done);
  return cudaGetLastError();
}

// Only the (arithmetic, input, output) type and mode combinations the
// preconditioners use are instantiated: FP64 throughout (every mode); FP32
// transforms with FP64 input (forward passes of the first direction), FP32
// in and out (forward, fused, backward without dot products), FP64 output
// (backward passes of the first direction, with 0..2 dot products).
template <typename Tc, typename Tin, typename Tout>
cudaError_t launch_pass(const PassLaunch<Tc>& P, int mode, int ndot, const Tin* in, Tout* out, cudaStream_t st) {
  constexpr bool in64 = std::is_same<Tc, float>::value && std::is_same<Tin, double>::value;
  constexpr bool out64 = std::is_same<Tc, float>::value && std::is_same<Tout, double>::value;
  constexpr bool f32 = std::is_same<Tc, float>::value && !in64 && !out64;
  if constexpr (in64) {
    if (mode != PM_FWD) return cudaErrorInvalidValue;
    return launch_pass_t<Tc, Tin, Tout, PM_FWD, 0>(P, in, out, st);
  } else if constexpr (out64) {
    if (mode != PM_BWD) return cudaErrorInvalidValue;
    if (ndot == 0) return launch_pass_t<Tc, Tin, Tout, PM_BWD, 0>(P, in, out, st);
    if (ndot == 1) return launch_pass_t<Tc, Tin, Tout, PM_BWD, 1>(P, in, out, st);
    return launch_pass_t<Tc, Tin, Tout, PM_BWD, 2>(P, in, out, st);
  } else if constexpr (f32) {
    if (ndot != 0) return cudaErrorInvalidValue;
    if (mode == PM_FWD) return launch_pass_t<Tc, Tin, Tout, PM_FWD, 0>(P, in, out, st);
    if (mode == PM_FUSED) return launch_pass_t<Tc, Tin, Tout, PM_FUSED, 0>(P, in, out, st);
    return launch_pass_t<Tc, Tin, Tout, PM_BWD, 0>(P, in, out, st);
  } else {
    if (mode == PM_FWD) return launch_pass_t<Tc, Tin, Tout, PM_FWD, 0>(P, in, out, st);
    if (mode == PM_FUSED) return launch_pass_t<Tc, Tin, Tout, PM_FUSED, 0>(P, in, out, st);
    if (ndot == 0) return launch_pass_t<Tc, Tin, Tout, PM_BWD, 0>(P, in, out, st);
    if (ndot == 1) return launch_pass_t<Tc, Tin, Tout, PM_BWD, 1>(P, in, out, st);
    return launch_pass_t<Tc, Tin, Tout, PM_BWD, 2>(P, in, out, st);
  }
}

template <typename Tc, typename Tin, typename Tout, int MODE, int NDOT>
static cudaError_t launch_batched_t(const PassDesc<Tc, Tin, Tout>* sys, const long long* tile_prefix, int nsys,
                                   long long total_tiles, size_t smem, cudaStream_t st) {
  auto kern = precond_pass_batched<Tc, Tin, Tout, MODE, NDOT>;
  static size_t smem_set = 0;  // attribute is raised only when needed (not inside a graph capture)
  if (smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    smem_set = smem;
  }
  if (total_tiles <= 0) return cudaSuccess;
  kern<<<(unsigned)total_tiles, kThreads, smem, st>>>(sys, tile_prefix, nsys);
  return cudaGetLastError();
}

template <typename Tc, typename Tin, typename Tout>
cudaError_t launch_pass_batched(const PassDesc<Tc, Tin, Tout>* sys, const long long* tile_prefix, int nsys,
                                long long total_tiles, size_t smem, int mode, int ndot, cudaStream_t st) {
  constexpr bool in64 = std::is_same<Tc, float>::value && std::is_same<Tin, double>::value;
  constexpr bool out64 = std::is_same<Tc, float>::value && std::is_same<Tout, double>::value;
  constexpr bool f32 = std::is_same<Tc, float>::value && !in64 && !out64;
  if constexpr (in64) {  // the same combinations as launch_pass
    if (mode != PM_FWD) return cudaErrorInvalidValue;
    return launch_batched_t<Tc, Tin, Tout, PM_FWD, 0>(sys, tile_prefix, nsys, total_tiles, smem, st);
  } else if constexpr (out64) {
    if (mode != PM_BWD) return cudaErrorInvalidValue;
    if (ndot == 0) return launch_batched_t<Tc, Tin, Tout, PM_BWD, 0>(sys, tile_prefix, nsys, total_tiles, smem, st);
    if (ndot == 1) return launch_batched_t<Tc, Tin, Tout, PM_BWD, 1>(sys, tile_prefix, nsys, total_tiles, smem, st);
    return launch_batched_t<Tc, Tin, Tout, PM_BWD, 2>(sys, tile_prefix, nsys, total_tiles, smem, st);
  } else if constexpr (f32) {
    if (ndot != 0) return cudaErrorInvalidValue;
    if (mode == PM_FWD) return launch_batched_t<Tc, Tin, Tout, PM_FWD, 0>(sys, tile_prefix, nsys, total_tiles, smem, st);
    if (mode == PM_FUSED)
      return launch_batched_t<Tc, Tin, Tout, PM_FUSED, 0>(sys, tile_prefix, nsys, total_tiles, smem, st);
    return launch_batched_t<Tc, Tin, Tout, PM_BWD, 0>(sys, tile_prefix, nsys, total_tiles, smem, st);
  } else {
    if (mode == PM_FWD) return launch_batched_t<Tc, Tin, Tout, PM_FWD, 0>(sys, tile_prefix, nsys, total_tiles, smem, st);
    if (mode == PM_FUSED)
      return launch_batched_t<Tc, Tin, Tout, PM_FUSED, 0>(sys, tile_prefix, nsys, total_tiles, smem, st);
    if (ndot == 0) return launch_batched_t<Tc, Tin, Tout, PM_BWD, 0>(sys, tile_prefix, nsys, total_tiles, smem, st);
    if (ndot == 1) return launch_batched_t<Tc, Tin, Tout, PM_BWD, 1>(sys, tile_prefix, nsys, total_tiles, smem, st);
    return launch_batched_t<Tc, Tin, Tout, PM_BWD, 2>(sys, tile_prefix, nsys, total_tiles, smem, st);
  }
}

template <typename Tin, typename Tout>
cudaError_t launch_wpass_batched(const PassDesc<float, Tin, Tout>* sys, const long long* tile_prefix, int nsys,
                                 long long total_tiles, size_t smem, int N, int kind, int pair, int mode, int ndot,
                                 cudaStream_t st) {
  switch (N) {
    case 64:
      return launch_wpass_batched_n<64, Tin, Tout>(sys, tile_prefix, nsys, total_tiles, smem, kind, pair, mode, ndot,
                                                   st);
    case 128:
      return launch_wpass_batched_n<128, Tin, Tout>(sys, tile_prefix, nsys, total_tiles, smem, kind, pair, mode, ndot,
                                                    st);
    case 256:
      return launch_wpass_batched_n<256, Tin, Tout>(sys, tile_prefix, nsys, total_tiles, smem, kind, pair, mode, ndot,
                                                    st);
    case 512:
      return launch_wpass_batched_n<512, Tin, Tout>(sys, tile_prefix, nsys, total_tiles, smem, kind, pair, mode, ndot,
                                                    st);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_wpass_batched<double, float>(const PassDesc<float, double, float>*, const long long*, int,
                                                         long long, size_t, int, int, int, int, int, cudaStream_t);
template cudaError_t launch_wpass_batched<float, float>(const PassDesc<float, float, float>*, const long long*, int,
                                                        long long, size_t, int, int, int, int, int, cudaStream_t);
template cudaError_t launch_wpass_batched<float, double>(const PassDesc<float, float, double>*, const long long*, int,
                                                         long long, size_t, int, int, int, int, int, cudaStream_t);

#define IFFD_INST_BATCHED(Tc, Tin, Tout)                                                                      \
  template cudaError_t launch_pass_batched<Tc, Tin, Tout>(const PassDesc<Tc, Tin, Tout>*, const long long*, int, \
                                                          long long, size_t, int, int, cudaStream_t);
IFFD_INST_BATCHED(double, double, double)
IFFD_INST_BATCHED(float, double, float)
IFFD_INST_BATCHED(float, float, float)
IFFD_INST_BATCHED(float, float, double)

template cudaError_t launch_pass<double, double, double>(const PassLaunch<double>&, int, int, const double*,
                                                         double*, cudaStream_t);
template cudaError_t launch_pass<float, double, float>(const PassLaunch<float>&, int, int, const double*, float*,
                                                       cudaStream_t);
template cudaError_t launch_pass<float, float, float>(const PassLaunch<float>&, int, int, const float*, float*,
                                                      cudaStream_t);
template cudaError_t launch_pass<float, float, double>(const PassLaunch<float>&, int, int, const float*, double*,
                                                       cudaStream_t);

}  // namespace iffd
