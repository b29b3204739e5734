// Building blocks of the slab-decomposed solve of one problem on several GPUs
// (one process per GPU; the Python layer slab.py moves the data between ranks
// with all-to-all exchanges and reduces the inner products):
//
//  - iffd_apply_pass: one transform pass of the preconditioner (eq.
//    "preconditioner": Q~^T, Q~, or Q~^T, the eigenvalue scaling and Q~ along
//    one direction) on a box of the grid that holds whole pencils along that
//    direction. The box's offset in the global grid places it among the
//    eigenvalues of the other directions for the scaling.
//  - iffd_slab_stiffness: A^ u (eq. "system_matrix") on the rows [z0, z0 + nz)
//    of the slowest direction, from u on those rows plus up to p rows on each
//    side (the halo the neighbouring ranks send): the banded sweep along the
//    slowest direction takes the global band rows of M and K; the sweeps along
//    the other directions are the library's ordinary sweeps on the slab.
//  - iffd_copy_box: a 3D box copy between two arrays (packing and unpacking
//    the blocks of the all-to-all exchanges).
//  - iffd_vec_dot / iffd_vec_axpby: the PCG inner products (deterministic
//    reduction order) and vector updates on a rank's part of the vectors.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/iffd.h"
#include "device_common.cuh"
#include "kernels.h"
#include "plan.h"
#include "precond_dev.cuh"

namespace iffd {

namespace {

// T1 = M_L u, T2 = K_L u along the slowest direction L for the rows
// z0 .. z0 + nz - 1 (global numbering), u given on rows e0 .. e1 - 1.
__global__ void slab_first_sweep(const double* __restrict__ u_ext, double* __restrict__ T1, double* __restrict__ T2,
                                 long long plane, int nz, int z0, int e0, int e1, int p,
                                 const double* __restrict__ Mb, const double* __restrict__ Kb) {
  const long long total = plane * nz;
  const int bw = 2 * p + 1;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long k = idx / plane, xy = idx - k * plane;
    const int g = z0 + (int)k;
    const int jlo = max(g - p, e0), jhi = min(g + p, e1 - 1);
    double a = 0.0, b = 0.0;
    for (int j = jlo; j <= jhi; ++j) {
      const double v = u_ext[(long long)(j - e0) * plane + xy];
      a = fma(__ldg(Mb + (long long)g * bw + (j - g + p)), v, a);
      b = fma(__ldg(Kb + (long long)g * bw + (j - g + p)), v, b);
    }
    T1[idx] = a;
    T2[idx] = b;
  }
}

__global__ void copy_box_kernel(const double* __restrict__ src, long long sx, long long sy, long long s0,
                                double* __restrict__ dst, long long dx, long long dy, long long d0, int ex, int ey,
                                int ez) {
  const long long total = (long long)ex * ey * ez;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long i = idx % ex, rest = idx / ex;
    const long long j = rest % ey, k = rest / ey;
    dst[d0 + i + dx * j + dx * dy * k] = src[s0 + i + sx * j + sx * sy * k];
  }
}

// Fixed-order dot product: per-block partial sums (block b handles the
// grid-stride elements b, b + G, ... with G = 256 * kDotBlocks threads), then
// one block adds the partials in block order.
constexpr int kDotBlocks = 1024;

__global__ void dot_partials(const double* __restrict__ a, const double* __restrict__ b, long long n,
                             double* __restrict__ part) {
  __shared__ double red[kThreads / 32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

__global__ void dot_final(const double* __restrict__ part, int nparts, double* __restrict__ out) {
  __shared__ double red[kThreads / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    *out = t;
  }
}

__global__ void axpby_kernel(long long n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], b * y[i]);
}

int grid_for(long long n) {
  return (int)std::max<long long>(1, std::min<long long>((n + kThreads - 1) / kThreads, 8 * 152));
}

}  // namespace

int check_plan_device(const Plan* P) {
  int dev = -1;
  IFFD_CUDA(cudaGetDevice(&dev));
  if (dev != P->device) return fail(IFFD_ERR_INVALID_ARG, "plan was created on another CUDA device");
  return IFFD_OK;
}

}  // namespace iffd

using namespace iffd;

extern "C" {

int iffd_apply_pass(iffd_handle h, int axis, int mode, const int* box, const int* offset, const double* in,
                    double* out, void* stream) {
  g_err.clear();
  if (!h || !box || !offset || !in || !out) return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  const Plan* P = &h->P;
  int rc = check_plan_device(P);
  if (rc) return rc;
  const int d = P->d;
  if (axis < 0 || axis >= d || mode < PM_FWD || mode > PM_FUSED)
    return fail(IFFD_ERR_INVALID_ARG, "bad axis or mode");
  if (P->opt.precision != IFFD_PREC_FP64 || P->opt.precond != IFFD_PRECOND_IFFD)
    return fail(IFFD_ERR_UNSUPPORTED, "iffd_apply_pass: FP64 IFFD plans only");
  Dims dims{};
  dims.d = d;
  dims.N = 1;
  for (int k = 0; k < 3; ++k) dims.m[k] = 1;
  for (int k = 0; k < d; ++k) {
    if (box[k] < 1 || offset[k] < 0 || offset[k] + box[k] > P->dims.m[k])
      return fail(IFFD_ERR_INVALID_ARG, "box outside the grid");
    dims.m[k] = box[k];
    dims.N *= box[k];
  }
  if (box[axis] != P->dims.m[axis] || offset[axis] != 0)
    return fail(IFFD_ERR_INVALID_ARG, "the box must hold whole pencils along the pass direction");
  if (mode == PM_FUSED && axis != d - 1) return fail(IFFD_ERR_INVALID_ARG, "the fused pass runs along the last direction");
  PassLaunch<double> L{};
  L.dims = dims;
  L.axis = axis;
  L.PP = P->PPd[axis];
  L.ldt = P->ldtd[axis];
  L.ax = P->axd[axis];
  L.ax.rden = nullptr;  // the scaling divides by the eigenvalue sums of the box
  L.lamA = P->axd[0].lam + offset[0];
  L.lamB = (d == 3) ? P->axd[1].lam + offset[1] : P->axd[0].lam;
  L.pipe = 0;
  L.wN = 0;
  const int kind = mode == PM_FWD ? IFFD_K_PRECOND_FWD : (mode == PM_BWD ? IFFD_K_PRECOND_BWD : IFFD_K_PRECOND_FUSED);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  IFFD_LAUNCH(P, kind, st, (launch_pass<double, double, double>(L, mode, 0, in, out, st)));
  return IFFD_OK;
}

int iffd_slab_stiffness(iffd_handle h, int z0, int nz, const double* u_ext, double* Au, void* ws, void* stream) {
  g_err.clear();
  if (!h || !u_ext || !Au) return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  if (u_ext == Au) return fail(IFFD_ERR_INVALID_ARG, "u_ext and Au must not alias");
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(IFFD_ERR_WORKSPACE, "ws NULL or misaligned");
  const Plan* P = &h->P;
  int rc = check_plan_device(P);
  if (rc) return rc;
  if (P->opt.coef != IFFD_COEF_CONST) return fail(IFFD_ERR_UNSUPPORTED, "iffd_slab_stiffness: IFFD_COEF_CONST plans only");
  const int d = P->d, L = d - 1, m = P->dims.m[L], p = P->p;
  if (nz < 1 || z0 < 0 || z0 + nz > m) return fail(IFFD_ERR_INVALID_ARG, "slab rows outside the grid");
  const int e0 = std::max(0, z0 - p), e1 = std::min(m, z0 + nz + p);
  long long plane = 1;
  for (int k = 0; k < L; ++k) plane *= P->dims.m[k];
  const long long n = plane * nz;
  double* T1 = static_cast<double*>(ws);
  double* T2 = T1 + ((n + 31) / 32) * 32;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const BandTab& b = P->bt[L];
  P->prof.begin(IFFD_K_STIFF_FIRST, st);
  slab_first_sweep<<<grid_for(n), kThreads, 0, st>>>(u_ext, T1, T2, plane, nz, z0, e0, e1, p, b.Mb, b.Kb);
  IFFD_CUDA(cudaGetLastError());
  P->prof.end(st);
  StiffLaunch S{};
  S.dims = P->dims;
  S.dims.m[L] = nz;
  S.dims.N = n;
  if (d == 3) {
    S.axis = 1;
    S.PP = P->PPs[1];
    S.ldt = P->ldts[1];
    S.bt = P->bt[1];
    IFFD_LAUNCH(P, IFFD_K_STIFF_MID, st, launch_stiff_mid(S, T1, T2, nullptr, st));
  }
  S.axis = 0;
  S.PP = P->PPs[0];
  S.ldt = P->ldts[0];
  S.bt = P->bt[0];
  IFFD_LAUNCH(P, IFFD_K_STIFF_LAST, st, launch_stiff_last(S, T1, T2, Au, nullptr, nullptr, nullptr, st));
  return IFFD_OK;
}

int iffd_slab_workspace_bytes(iffd_handle h, int nz, size_t* bytes) {
  if (!h || !bytes || nz < 1) return fail(IFFD_ERR_INVALID_ARG, "bad argument");
  const Plan* P = &h->P;
  long long plane = 1;
  for (int k = 0; k < P->d - 1; ++k) plane *= P->dims.m[k];
  *bytes = (size_t)2 * (((plane * nz + 31) / 32) * 32) * sizeof(double);
  return IFFD_OK;
}

int iffd_copy_box(const double* src, const int* src_dims, const int* src_off, double* dst, const int* dst_dims,
                  const int* dst_off, const int* ext, void* stream) {
  g_err.clear();
  if (!src || !src_dims || !src_off || !dst || !dst_dims || !dst_off || !ext)
    return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  for (int k = 0; k < 3; ++k) {
    if (ext[k] < 0 || src_off[k] < 0 || dst_off[k] < 0 || src_off[k] + ext[k] > src_dims[k] ||
        dst_off[k] + ext[k] > dst_dims[k])
      return fail(IFFD_ERR_INVALID_ARG, "box outside an array");
  }
  const long long total = (long long)ext[0] * ext[1] * ext[2];
  if (total == 0) return IFFD_OK;
  const long long s0 = src_off[0] + (long long)src_dims[0] * (src_off[1] + (long long)src_dims[1] * src_off[2]);
  const long long d0 = dst_off[0] + (long long)dst_dims[0] * (dst_off[1] + (long long)dst_dims[1] * dst_off[2]);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  copy_box_kernel<<<grid_for(total), kThreads, 0, st>>>(src, src_dims[0], src_dims[1], s0, dst, dst_dims[0],
                                                        dst_dims[1], d0, ext[0], ext[1], ext[2]);
  IFFD_CUDA(cudaGetLastError());
  return IFFD_OK;
}

int iffd_vec_dot_workspace_bytes(size_t* bytes) {
  if (!bytes) return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  *bytes = (size_t)kDotBlocks * sizeof(double);
  return IFFD_OK;
}

int iffd_vec_dot(const double* a, const double* b, long long n, double* result, void* ws, void* stream) {
  g_err.clear();
  if (!a || !b || !result || !ws || n < 0) return fail(IFFD_ERR_INVALID_ARG, "bad argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* part = static_cast<double*>(ws);
  const int g = (int)std::max<long long>(1, std::min<long long>((n + kThreads - 1) / kThreads, kDotBlocks));
  dot_partials<<<g, kThreads, 0, st>>>(a, b, n, part);
  IFFD_CUDA(cudaGetLastError());
  dot_final<<<1, kThreads, 0, st>>>(part, g, result);
  IFFD_CUDA(cudaGetLastError());
  return IFFD_OK;
}

int iffd_vec_axpby(long long n, double a, const double* x, double b, double* y, void* stream) {
  g_err.clear();
  if (!x || !y || n < 0) return fail(IFFD_ERR_INVALID_ARG, "bad argument");
  if (n == 0) return IFFD_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  axpby_kernel<<<grid_for(n), kThreads, 0, st>>>(n, a, x, b, y);
  IFFD_CUDA(cudaGetLastError());
  return IFFD_OK;
}

}  // extern "C"
