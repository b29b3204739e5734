// Double-float warp-FFT passes of FFT length 256 (kernels in precond_warp.cuh):
// the FP64 preconditioner's transforms on the FP32 pipe.
#include "precond_warp.cuh"

namespace iffd {
IFFD_WARP_INSTANTIATE_DF(256)
}  // namespace iffd
