// FP32 and FP64 warp-FFT passes of FFT length 64 (kernels in precond_warp.cuh).
#include "precond_warp.cuh"

namespace iffd {
IFFD_WARP_INSTANTIATE(64)
IFFD_WARP_INSTANTIATE_F64(64)
}  // namespace iffd
