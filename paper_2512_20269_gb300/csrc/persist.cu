// Persistent engine launch: one kernel runs every phase of `k` PCG
// iterations (Section 3, with the IFFD preconditioner of eq. "preconditioner"
// and the stiffness of eq. "system_matrix") of all active systems of the
// batched engine, walking a device work queue instead of one launch per phase.
//
// The queue is a list of item ranges (PRange): the tiles (or vector blocks,
// or the single reduction) of one system in one phase of one iteration,
// listed phase-major: iteration, then phase (stiffness sweeps, (p, A p),
// update, (r, r), transform passes, (r, z)), then system. A CTA takes the next
// ticket from a global counter, finds its range, waits until its system has
// completed every earlier item (a per-system counter), runs the item with the
// same device body, tile decomposition and reduction order as the per-phase
// kernels -- so every result is bitwise that of the stand-alone solve -- and
// then counts the item as complete.
//
// Progress: an item waits only on items of its own system with smaller
// tickets; those were taken earlier by CTAs that are running, so the oldest
// unfinished item never waits and the walk cannot deadlock. Every wait is
// still bounded: after `wait_limit` polls the CTA records IFFD_ERR_TIMEOUT in
// the queue's status word, skips the item's work (the counter still
// advances, so nothing else waits on it) and carries on; the host reads the
// status after the launch. Data written by other CTAs during the launch is
// read through the L2-coherent path (CG loads); completion is published with
// a memory fence before the counter increment.
#include <cuda_runtime.h>

#include "../../include/iffd.h"
#include "device_common.cuh"
#include "kernels.h"
#include "pcg_dev.cuh"
#include "precond_block.cuh"
#include "stiff_dev.cuh"

namespace iffd {

namespace {

constexpr int kDescBytes = 1024;  // the largest descriptor (PassDesc) fits (checked below)
static_assert(sizeof(PassDesc<double, double, double>) <= kDescBytes, "descriptor buffer too small");
static_assert(sizeof(PassDesc<float, double, float>) <= kDescBytes, "descriptor buffer too small");
static_assert(sizeof(StiffDesc) <= kDescBytes && sizeof(VecDesc) <= kDescBytes && sizeof(FinDesc) <= kDescBytes,
              "descriptor buffer too small");
static_assert(sizeof(PassDesc<double, double, double>) % 8 == 0 && sizeof(PassDesc<float, double, float>) % 8 == 0 &&
                  sizeof(PassDesc<float, float, float>) % 8 == 0 && sizeof(PassDesc<float, float, double>) % 8 == 0 &&
                  sizeof(StiffDesc) % 8 == 0 && sizeof(VecDesc) % 8 == 0 && sizeof(FinDesc) % 8 == 0,
              "descriptors are copied in 8-byte words");

template <int P>
__device__ __forceinline__ void run_stiff(int stage, const StiffDesc& sd, long long tile, unsigned char* smem) {
  if (stage == SS_FIRST)
    first_body<P, true>(sd.dims, sd.axis, sd.PP, sd.ldt, sd.bt, sd.u, sd.z, sd.p_io, sd.beta, sd.pmode, sd.T1,
                        sd.T2, tile, smem);
  else if (stage == SS_MID)
    mid_body<P, true>(sd.dims, sd.axis, sd.PP, sd.ldt, sd.bt, sd.T1, sd.T2, tile, smem);
  else
    last_body<P, true>(sd.dims, sd.axis, sd.PP, sd.ldt, sd.bt, sd.T1, sd.T2, sd.out, sd.dotv, sd.partial, tile,
                       (int)tile, smem);
}

template <typename Tc, typename Tin, typename Tout, int MODE, int NDOT>
__device__ __forceinline__ void run_pass(const void* desc, long long tile, int ntiles, unsigned char* smem) {
  const PassDesc<Tc, Tin, Tout>& d = *static_cast<const PassDesc<Tc, Tin, Tout>*>(desc);
  precond_body<Tc, Tin, Tout, MODE, NDOT, true>(d.in, d.out, d.dims, d.axis, d.PP, d.ldt, d.ax, d.lamA, d.lamB, d.dot0,
                                                d.dot1, d.partial, tile, (int)tile, ntiles, smem);
}

// The system's `done` flag (set by its reductions) makes its remaining items
// return at once, as the early-exit test of the per-phase kernels does.
__device__ __forceinline__ bool finished(const int* done) { return done != nullptr && ldd<true>(done) != 0; }

__device__ void run_item(const PRange& rg, const void* desc, long long tile, double tol2, int maxit,
                         unsigned char* smem) {
  switch (rg.kind) {
    case PK_STIFF: {
      const StiffDesc& sd = *static_cast<const StiffDesc*>(desc);
      if (finished(sd.done)) return;
      const int stage = rg.arg >> 5, p = rg.arg & 31;
      switch (p) {
        case 2: run_stiff<2>(stage, sd, tile, smem); break;
        case 3: run_stiff<3>(stage, sd, tile, smem); break;
        case 4: run_stiff<4>(stage, sd, tile, smem); break;
        case 5: run_stiff<5>(stage, sd, tile, smem); break;
        case 6: run_stiff<6>(stage, sd, tile, smem); break;
        case 7: run_stiff<7>(stage, sd, tile, smem); break;
        default: run_stiff<8>(stage, sd, tile, smem); break;
      }
      return;
    }
    case PK_FIN: {
      const FinDesc& fd = *static_cast<const FinDesc*>(desc);
      finalize_body<true>(fd.st, fd.partial, fd.nparts, rg.arg, tol2, maxit);
      return;
    }
    case PK_UPD: {
      const VecDesc& vd = *static_cast<const VecDesc*>(desc);
      if (ldd<true>(&vd.st->done)) return;
      update_body<true>(vd.x, vd.r, vd.p, vd.q, vd.st, vd.N, vd.part_rr, (int)tile, rg.ntiles);
      return;
    }
    case PK_PASS_D: {
      if (finished(static_cast<const PassDesc<double, double, double>*>(desc)->done)) return;
      switch (rg.arg) {
        case PM_FWD * 4: run_pass<double, double, double, PM_FWD, 0>(desc, tile, rg.ntiles, smem); break;
        case PM_FUSED * 4: run_pass<double, double, double, PM_FUSED, 0>(desc, tile, rg.ntiles, smem); break;
        case PM_BWD * 4: run_pass<double, double, double, PM_BWD, 0>(desc, tile, rg.ntiles, smem); break;
        case PM_BWD * 4 + 1: run_pass<double, double, double, PM_BWD, 1>(desc, tile, rg.ntiles, smem); break;
        default: run_pass<double, double, double, PM_BWD, 2>(desc, tile, rg.ntiles, smem); break;
      }
      return;
    }
    case PK_PASS_F_IN: {
      if (finished(static_cast<const PassDesc<float, double, float>*>(desc)->done)) return;
      run_pass<float, double, float, PM_FWD, 0>(desc, tile, rg.ntiles, smem);
      return;
    }
    case PK_PASS_F_MID: {
      if (finished(static_cast<const PassDesc<float, float, float>*>(desc)->done)) return;
      if (rg.arg == PM_FWD) run_pass<float, float, float, PM_FWD, 0>(desc, tile, rg.ntiles, smem);
      else if (rg.arg == PM_FUSED) run_pass<float, float, float, PM_FUSED, 0>(desc, tile, rg.ntiles, smem);
      else run_pass<float, float, float, PM_BWD, 0>(desc, tile, rg.ntiles, smem);
      return;
    }
    default: {  // PK_PASS_F_OUT
      if (finished(static_cast<const PassDesc<float, float, double>*>(desc)->done)) return;
      if (rg.arg == 0) run_pass<float, float, double, PM_BWD, 0>(desc, tile, rg.ntiles, smem);
      else if (rg.arg == 1) run_pass<float, float, double, PM_BWD, 1>(desc, tile, rg.ntiles, smem);
      else run_pass<float, float, double, PM_BWD, 2>(desc, tile, rg.ntiles, smem);
      return;
    }
  }
}

// Index of the range holding ticket t, searching forward from `cur` (a CTA's
// tickets only grow): exponential steps, then bisection.
__device__ __forceinline__ int find_range(const PRange* __restrict__ ranges, int n, long long t, int cur) {
  int lo = cur, step = 1;
  while (lo + step < n && ranges[lo + step].first <= t) {
    lo += step;
    step <<= 1;
  }
  int hi = min(n - 1, lo + step);
  while (lo < hi) {  // last range with first <= t
    const int mid = (lo + hi + 1) >> 1;
    if (ranges[mid].first <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// At most 64 registers a thread (four CTAs an SM); the compiler's own choice
// (~106) halves the resident CTAs for a few spilled bytes saved.
__global__ void __launch_bounds__(kThreads, 4)
engine_persistent(const PRange* __restrict__ ranges, int nranges, long long total, long long* done_cnt, PQueue* q,
                  long long wait_limit, double tol2, int maxit) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) unsigned char s_desc[kDescBytes];
  __shared__ int s_r, s_skip;
  __shared__ long long s_tile;
  int cur = 0;  // thread 0's current range
  for (;;) {
    if (threadIdx.x == 0) {
      const long long t = (long long)atomicAdd(&q->head, 1ULL);
      int r = -1, skip = 0;
      if (t < total) {
        r = find_range(ranges, nranges, t, cur);
        cur = r;
        const PRange& rg = ranges[r];
        s_tile = t - rg.first;
        long long polls = 0;
        while (*((volatile long long*)(done_cnt + rg.sys)) < rg.need) {
          if (++polls > wait_limit) {
            atomicExch(&q->status, (int)IFFD_ERR_TIMEOUT);
            skip = 1;
            break;
          }
          __nanosleep(64);
        }
        __threadfence();
      }
      s_r = r;
      s_skip = skip;
    }
    __syncthreads();
    const int r = s_r;
    if (r < 0) break;
    const PRange rg = ranges[r];
    if (!s_skip) {
      // the system's descriptor, copied by the whole CTA
      const unsigned long long* src = static_cast<const unsigned long long*>(rg.desc);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(s_desc);
      for (int w = threadIdx.x; w < rg.desc_bytes / 8; w += blockDim.x) dst[w] = __ldg(src + w);
      __syncthreads();
      run_item(rg, s_desc, s_tile, tol2, maxit, smem);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long*>(done_cnt + rg.sys), 1ULL);
  }
}

}  // namespace

cudaError_t launch_persistent(const PRange* ranges, int nranges, long long total, long long* done_cnt, PQueue* q,
                              long long wait_limit, double tol2, int maxit, size_t smem, int grid, cudaStream_t st) {
  static size_t smem_set = 0;  // raised only when needed
  if (smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(engine_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    smem_set = smem;
  }
  if (total <= 0 || grid <= 0) return cudaSuccess;
  engine_persistent<<<grid, kThreads, smem, st>>>(ranges, nranges, total, done_cnt, q, wait_limit, tol2, maxit);
  return cudaGetLastError();
}

int persistent_grid(size_t smem) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(engine_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, engine_persistent, kThreads, smem) != cudaSuccess)
    return 0;
  return per_sm * sms;
}

}  // namespace iffd
