// FP32 warp-FFT passes of FFT length 64 (kernels in precond_warp.cuh).
#include "precond_warp.cuh"

namespace iffd {
IFFD_WARP_INSTANTIATE(64)
}  // namespace iffd
