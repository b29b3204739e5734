// Allocation-free stiffness apply: iffd_apply_stiffness_noalloc.
//
// iffd_apply_stiffness needs two N-vector temporaries, which it takes from the
// caller's workspace. Some callers cannot provide that buffer when they need
// A^ u: a host framework whose caching allocator owns all device memory and
// forbids side allocations, an embedded solver whose device-memory budget is
// fixed at start-up, or a latency-critical loop that must not pay cudaMalloc's
// implicit device synchronisation. For them this entry point keeps the
// temporaries in a file-scope device array of fixed size
// (2 x IFFD_NOALLOC_MAX_DOFS doubles = 16 MiB), which every GPU that loads this
// module holds until the process exits. The entry point itself calls no
// cudaMalloc, cudaFree or other allocating routine.
//
// Host code cannot use the array's name as a device address, so the first
// call on each device (with that device current) resolves the address with
// cudaGetSymbolAddress and caches it together with the CUDA context it belongs
// to; a later call that finds another context current on that device (after a
// cudaDeviceReset, say) resolves the address again instead of reusing a stale
// one.
#include <cuda.h>
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
// Defined in capi.cu: the checks of iffd_apply_stiffness that come before any
// work (plan device current, constant coefficient).
int plan_check_noalloc(iffd_handle h);
long long plan_num_dofs(iffd_handle h);
int record_error(int code, const std::string& msg);

// The two temporaries of the stiffness sweeps: [T1 | T2], each
// IFFD_NOALLOC_MAX_DOFS doubles.
static __device__ __align__(256) double g_stiffness_scratch[2 * (size_t)IFFD_NOALLOC_MAX_DOFS];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchAddr {
  CUcontext ctx = nullptr;  // context the address was resolved in
  double* addr = nullptr;
};
ScratchAddr g_scratch[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

// The driver's cuCtxGetCurrent, reached through the runtime (no link-time
// dependency on the driver library).
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(f);
  }();
  return fn;
}

// Current context of this thread, or null (none current yet, or the driver
// entry point is unavailable).
CUcontext current_ctx() {
  CUcontext ctx = nullptr;
  CtxGetCurrentFn get = ctx_get_current();
  if (get == nullptr || get(&ctx) != CUDA_SUCCESS) return nullptr;
  return ctx;
}

// Address of g_stiffness_scratch on the current device, resolved on the first
// call on the device and again whenever the current context differs from the
// one it was resolved in (or cannot be identified).
int scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return record_error(IFFD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return record_error(IFFD_ERR_UNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lock(g_mu);
  ScratchAddr& s = g_scratch[dev];
  const CUcontext ctx = current_ctx();
  if (s.addr == nullptr || ctx == nullptr || s.ctx != ctx) {
    void* p = nullptr;
    // also makes the device's runtime context current on this thread
    e = cudaGetSymbolAddress(&p, g_stiffness_scratch);
    if (e != cudaSuccess || p == nullptr)
      return record_error(IFFD_ERR_CUDA, std::string("cudaGetSymbolAddress(stiffness scratch): ") +
                                             cudaGetErrorString(e));
    s.addr = static_cast<double*>(p);
    s.ctx = current_ctx();
  }
  *out = s.addr;
  return IFFD_OK;
}
}  // namespace

}  // namespace iffd

extern "C" int iffd_apply_stiffness_noalloc(iffd_handle h, const double* u, double* Au, void* stream) {
  using namespace iffd;
  if (!h || !u || !Au) return record_error(IFFD_ERR_INVALID_ARG, "NULL argument");
  if (u == Au) return record_error(IFFD_ERR_INVALID_ARG, "u and Au must not alias");
  int rc = plan_check_noalloc(h);  // same checks, same order, as iffd_apply_stiffness
  if (rc != IFFD_OK) return rc;
  const long long N = plan_num_dofs(h);
  if (N > (long long)IFFD_NOALLOC_MAX_DOFS)
    return record_error(IFFD_ERR_UNSUPPORTED,
                        "iffd_apply_stiffness_noalloc: problem has " + std::to_string(N) +
                            " DoFs, above the static scratch limit IFFD_NOALLOC_MAX_DOFS = " +
                            std::to_string((long long)IFFD_NOALLOC_MAX_DOFS) +
                            "; use iffd_apply_stiffness with a workspace");
  double* scratch = nullptr;
  rc = scratch_address(&scratch);
  if (rc != IFFD_OK) return rc;
  // Nothing in the scratch needs to start at zero: the first sweep writes both
  // temporaries completely before the later sweeps read them.
  return plan_stiffness_with_scratch(h, u, Au, scratch, scratch + IFFD_NOALLOC_MAX_DOFS,
                                     static_cast<cudaStream_t>(stream));
}
