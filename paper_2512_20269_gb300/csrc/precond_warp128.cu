// FP32 and FP64 warp-FFT passes of FFT length 128 (kernels in precond_warp.cuh).
#include "precond_warp.cuh"

namespace iffd {
IFFD_WARP_INSTANTIATE(128)
IFFD_WARP_INSTANTIATE_F64(128)
}  // namespace iffd
