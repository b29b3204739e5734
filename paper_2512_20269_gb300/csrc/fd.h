// Launch interface of the exact Fast Diagonalization comparator passes.
#pragma once

#include <cuda_runtime.h>

#include "device_common.cuh"

namespace iffd {

size_t fd_smem(int m);
int fd_tiles(const Dims& dims, int axis);
cudaError_t launch_fd_pass(int mode, const double* in, double* out, const Dims& dims, int axis,
                           const double* QT, const double* Q, const double* lam, const double* lamA,
                           const double* lamB, const int* done, cudaStream_t st);

}  // namespace iffd
