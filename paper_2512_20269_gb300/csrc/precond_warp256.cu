// FP32 and FP64 warp-FFT passes of FFT length 256 (kernels in precond_warp.cuh).
#include "precond_warp.cuh"

namespace iffd {
IFFD_WARP_INSTANTIATE(256)
IFFD_WARP_INSTANTIATE_F64(256)
}  // namespace iffd
