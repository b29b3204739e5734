// Arithmetic-pipe calibration: iffd_measure_peak.
//
// The roofline of the FP64-bound kernels (transform passes in FP64, stiffness
// sweeps) needs the rate at which this GPU retires FP64 fused multiply-adds,
// and the double-float transform passes need the FP32 rate. Neither figure is
// printed for GB300 with any certainty, so the library measures them: every
// thread of a grid that fills all SMs runs eight independent FMA chains
// x <- x * a + b (no memory traffic inside the loop), and the rate is the
// counted flops (2 per FMA) over the kernel's CUDA-event time. The chains are
// independent so that the FMA latency is covered by the other chains and by
// the other resident warps. A third kind times packed FP32 pairs
// (fma.rn.f32x2, two FMAs per instruction), which the double-float arithmetic
// can use for the real and imaginary parts of a complex value.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <type_traits>

#include "../../include/iffd.h"

namespace iffd {
int record_error(int code, const std::string& msg);
}

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kBlocksPerSm = 4;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_chains(T* out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // the chains converge to b / (1 - a) > 0, so this store never happens; it
  // keeps the compiler from removing the loop
  if (s < T(-1)) out[blockIdx.x] = s;
}

// Packed pairs of FP32 values: one fma.rn.f32x2 instruction carries two FMAs.
__device__ __forceinline__ float2 fma_x2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(d)
      : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)),
        "l"(*reinterpret_cast<unsigned long long*>(&c)));
  return *reinterpret_cast<float2*>(&d);
}

__global__ void __launch_bounds__(kPeakThreads) fma_chains_x2(float2* out, int iters, float2 a, float2 b) {
  float2 x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = make_float2((threadIdx.x + c) * 1e-3f, (threadIdx.x + 2 * c) * 1e-3f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma_x2(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
  if (s < -1.f) out[blockIdx.x] = make_float2(s, s);
}

template <typename T>
void launch_chains(T* sink, int grid, int iters, cudaStream_t st) {
  fma_chains<T><<<grid, kPeakThreads, 0, st>>>(sink, iters, T(0.9999), T(1e-4));
}
template <>
void launch_chains<float2>(float2* sink, int grid, int iters, cudaStream_t st) {
  fma_chains_x2<<<grid, kPeakThreads, 0, st>>>(sink, iters, make_float2(0.9999f, 0.9999f), make_float2(1e-4f, 1e-4f));
}

template <typename T>
int run_peak(cudaStream_t st, int sms, double* tflops) {
  const int grid = sms * kBlocksPerSm;
  T* sink = nullptr;  // one slot per block; never written in practice (see fma_chains)
  cudaError_t e = cudaMalloc(&sink, sizeof(T) * grid);
  if (e != cudaSuccess) return iffd::record_error(IFFD_ERR_CUDA, cudaGetErrorString(e));
  // flops per loop trip: 2 per FMA, two FMAs per packed instruction
  const double fl_per_iter = 2.0 * kChains * (double)grid * kPeakThreads * (std::is_same<T, float2>::value ? 2 : 1);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaFree(sink);
    return iffd::record_error(IFFD_ERR_CUDA, cudaGetErrorString(e));
  }
  int iters = 256;
  double best = 0.0;
  int rc = IFFD_OK;
  // a short launch sizes the loop for ~40 ms per timed launch; then the best
  // of three timed launches
  for (int rep = 0; rep < 4 && rc == IFFD_OK; ++rep) {
    cudaEventRecord(e0, st);
    launch_chains<T>(sink, grid, iters, st);
    cudaEventRecord(e1, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      rc = iffd::record_error(IFFD_ERR_CUDA, std::string("iffd_measure_peak: ") + cudaGetErrorString(e));
      break;
    }
    if (rep == 0) {
      const double per_iter_ms = std::max(1e-6, (double)ms / iters);
      iters = (int)std::min(1.0e8, std::max(256.0, 40.0 / per_iter_ms));
    } else {
      best = std::max(best, fl_per_iter * iters / (ms * 1e-3) / 1e12);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (rc == IFFD_OK) *tflops = best;
  return rc;
}

}  // namespace

extern "C" int iffd_measure_peak(int kind, void* stream, int* sm_count, double* tflops) {
  if (!tflops || kind < 0 || kind > 2)
    return iffd::record_error(IFFD_ERR_INVALID_ARG, "iffd_measure_peak: kind must be 0, 1 or 2, tflops non-NULL");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || sms < 1)
    return iffd::record_error(IFFD_ERR_CUDA, std::string("iffd_measure_peak: ") + cudaGetErrorString(e));
  if (sm_count) *sm_count = sms;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (kind == 2) return run_peak<float2>(st, sms, tflops);
  return kind == 0 ? run_peak<double>(st, sms, tflops) : run_peak<float>(st, sms, tflops);
}
