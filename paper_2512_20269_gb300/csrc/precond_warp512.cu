// FP32 warp-FFT passes of FFT length 512 (kernels in precond_warp.cuh).
#include "precond_warp.cuh"

namespace iffd {
IFFD_WARP_INSTANTIATE(512)
}  // namespace iffd
