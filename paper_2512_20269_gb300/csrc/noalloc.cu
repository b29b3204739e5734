// Allocation-free stiffness apply: iffd_apply_stiffness_noalloc.
//
// iffd_apply_stiffness needs two N-vector temporaries, which it takes from the
// caller's workspace. Some callers cannot provide that buffer when they need
// A^ u: code running while its stream is being captured into a CUDA graph
// (cudaMalloc is not allowed there), latency-critical loops that must not hit
// cudaMalloc's implicit device synchronisation, hosts whose framework allocator
// owns all device memory and forbids side allocations, and embedded callers
// with a fixed device-memory budget fixed at start-up. For them this entry
// point keeps the temporaries in a file-scope device array of fixed size
// (2 x IFFD_NOALLOC_MAX_DOFS doubles = 16 MiB), which every GPU that loads this
// module holds until the process exits. The entry point itself calls no
// cudaMalloc, cudaFree or other allocating routine.
//
// Host code cannot use the array's name as a device address, so the first
// call on each device (with that device current) resolves the address once
// with cudaGetSymbolAddress and caches it; later calls reuse it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/iffd.h"
#include "device_common.cuh"
#include "kernels.h"

namespace iffd {

// Defined in capi.cu: runs the three stiffness sweeps of plan h with the given
// temporaries (no profiler events), and records error messages.
int plan_stiffness_with_scratch(iffd_handle h, const double* u, double* Au, double* T1, double* T2,
                                cudaStream_t st);
long long plan_num_dofs(iffd_handle h);
int record_error(int code, const std::string& msg);

// The two temporaries of the stiffness sweeps: [T1 | T2], each
// IFFD_NOALLOC_MAX_DOFS doubles.
static __device__ __align__(256) double g_stiffness_scratch[2 * (size_t)IFFD_NOALLOC_MAX_DOFS];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Address of g_stiffness_scratch on the current device (resolved once per device).
int scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return record_error(IFFD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return record_error(IFFD_ERR_UNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_stiffness_scratch);
    if (e != cudaSuccess || p == nullptr)
      return record_error(IFFD_ERR_CUDA, std::string("cudaGetSymbolAddress(stiffness scratch): ") +
                                             cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return IFFD_OK;
}
}  // namespace

}  // namespace iffd

extern "C" int iffd_apply_stiffness_noalloc(iffd_handle h, const double* u, double* Au, void* stream) {
  using namespace iffd;
  if (!h || !u || !Au) return record_error(IFFD_ERR_INVALID_ARG, "NULL argument");
  if (u == Au) return record_error(IFFD_ERR_INVALID_ARG, "u and Au must not alias");
  const long long N = plan_num_dofs(h);
  if (N > (long long)IFFD_NOALLOC_MAX_DOFS)
    return record_error(IFFD_ERR_UNSUPPORTED,
                        "iffd_apply_stiffness_noalloc: problem has " + std::to_string(N) +
                            " DoFs, above the static scratch limit IFFD_NOALLOC_MAX_DOFS = " +
                            std::to_string((long long)IFFD_NOALLOC_MAX_DOFS) +
                            "; use iffd_apply_stiffness with a workspace");
  double* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != IFFD_OK) return rc;
  // Nothing in the scratch needs to start at zero: the first sweep writes both
  // temporaries completely before the later sweeps read them.
  return plan_stiffness_with_scratch(h, u, Au, scratch, scratch + IFFD_NOALLOC_MAX_DOFS,
                                     static_cast<cudaStream_t>(stream));
}
