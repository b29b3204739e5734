// Kronecker stiffness apply (eq. "system_matrix", written for d directions):
//   A^ u = sum_k (M x .. x K_k x .. x M) u,
// factorised into one banded (2p+1) sweep per direction (3D):
//   slowest direction z:  T1 = M_z u,           T2 = K_z u
//   direction y:          T1 <- M_y T1,        T2 <- K_y T1 + M_y T2
//   direction x:          A^ u = K_x T1 + M_x T2
// (2D: the first stage runs on y and the last on x.) Seven banded products in
// 3D, four in 2D. Interior rows of M and K are symmetric Toeplitz (uniform
// knots), so one set of pair sums u_{i-k} + u_{i+k} feeds both M and K; the
// first and last 2p-1 rows use the stored band.
#include "device_common.cuh"
#include "kernels.h"

namespace iffd {

// The degree P is a template parameter so that every banded loop is unrolled
// exactly: a runtime bound with a guarded unrolled loop would be if-converted
// into predicated FP64 instructions that still occupy the FP64 pipe.
template <int P>
struct Coefs {
  double m[P + 1];
  double k[P + 1];
};

template <int P>
__device__ __forceinline__ void load_coefs(const BandTab& bt, Coefs<P>& c) {
#pragma unroll
  for (int j = 0; j <= P; ++j) {
    c.m[j] = __ldg(bt.Mt + j);
    c.k[j] = __ldg(bt.Kt + j);
  }
}

// General band row (boundary rows): sum_j A[i][j] x[j].
template <int P>
__device__ __forceinline__ double band_row(const double* __restrict__ band, const double* row, int i, int m) {
  double s = 0.0;
  const double* b = band + (size_t)i * (2 * P + 1);
  const int j0 = max(0, i - P), j1 = min(m - 1, i + P);
  for (int j = j0; j <= j1; ++j) s = fma(__ldg(b + (j - i + P)), row[j], s);
  return s;
}

// Interior rows: (M x)_i and (K x)_i from shared pair sums.
template <int P>
__device__ __forceinline__ void toeplitz_mk(const Coefs<P>& c, const double* row, int i, double& mx, double& kx) {
  const double x0 = row[i];
  double am = c.m[0] * x0, ak = c.k[0] * x0;
#pragma unroll
  for (int k = 1; k <= P; ++k) {
    const double s = row[i - k] + row[i + k];
    am = fma(c.m[k], s, am);
    ak = fma(c.k[k], s, ak);
  }
  mx = am;
  kx = ak;
}

template <int P>
__device__ __forceinline__ double toeplitz_m(const Coefs<P>& c, const double* row, int i) {
  double a = c.m[0] * row[i];
#pragma unroll
  for (int k = 1; k <= P; ++k) a = fma(c.m[k], row[i - k] + row[i + k], a);
  return a;
}

template <int P>
__device__ __forceinline__ double toeplitz_k(const Coefs<P>& c, const double* row, int i) {
  double a = c.k[0] * row[i];
#pragma unroll
  for (int k = 1; k <= P; ++k) a = fma(c.k[k], row[i - k] + row[i + k], a);
  return a;
}

struct STile {
  long long base, S, pstr;
  int nvalid;
};

__device__ __forceinline__ STile stile(const Dims& dims, int axis, int PP, int tile) {
  STile g;
  const int m0 = dims.m[0], m1 = dims.m[1];
  if (axis == 0) {
    const long long rows = dims.N / m0;
    const long long r0 = (long long)tile * PP;
    g.base = r0 * m0;
    g.S = 1;
    g.pstr = m0;
    g.nvalid = (int)min((long long)PP, rows - r0);
  } else {
    const int ntx = (m0 + PP - 1) / PP;
    const int rest = tile / ntx;
    const int x0 = (tile - rest * ntx) * PP;
    g.S = (axis == 1) ? (long long)m0 : (long long)m0 * m1;
    g.base = x0 + ((axis == 1) ? (long long)rest * m0 * m1 : (long long)rest * m0);
    g.pstr = 1;
    g.nvalid = min(PP, m0 - x0);
  }
  return g;
}

__device__ __forceinline__ void tile_index(int axis, int e, int PP, int m, int& pc, int& i) {
  if (axis == 0) { pc = e / m; i = e - pc * m; }
  else { i = e / PP; pc = e - i * PP; }
}

int stiff_tiles(const Dims& dims, int axis, int PP) {
  if (axis == 0) return (int)((dims.N / dims.m[0] + PP - 1) / PP);
  const int ntx = (dims.m[0] + PP - 1) / PP;
  const long long rest = dims.N / ((long long)dims.m[0] * dims.m[axis]);
  return (int)(ntx * rest);
}

// pmode: 0 -> u = u; 1 -> u = z, p <- z; 2 -> u = z + beta p, p <- u
template <int P>
__global__ void __launch_bounds__(kThreads)
stiff_first(Dims dims, int axis, int PP, int ldt, BandTab bt, const double* __restrict__ u,
            const double* __restrict__ z, double* __restrict__ p_io, const double* __restrict__ betap, int pmode,
            double* __restrict__ T1, double* __restrict__ T2, const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  double* tile = reinterpret_cast<double*>(smem);
  const STile g = stile(dims, axis, PP, blockIdx.x);
  const int m = bt.m;
  const double beta = (pmode == 2) ? *betap : 0.0;
  for (int e = threadIdx.x; e < PP * m; e += blockDim.x) {
    int pc, i;
    tile_index(axis, e, PP, m, pc, i);
    double v = 0.0;
    if (pc < g.nvalid) {
      const long long off = g.base + pc * g.pstr + i * g.S;
      if (pmode == 0) {
        v = u[off];
      } else if (pmode == 1) {
        v = z[off];
        p_io[off] = v;
      } else {
        v = fma(beta, p_io[off], z[off]);
        p_io[off] = v;
      }
    }
    tile[pc * ldt + i] = v;
  }
  __syncthreads();
  Coefs<P> c;
  load_coefs<P>(bt, c);
  for (int e = threadIdx.x; e < PP * m; e += blockDim.x) {
    int pc, i;
    tile_index(axis, e, PP, m, pc, i);
    if (pc >= g.nvalid) continue;
    const double* row = tile + pc * ldt;
    double mx, kx;
    if (i >= bt.ilo && i < bt.ihi) {
      toeplitz_mk<P>(c, row, i, mx, kx);
    } else {
      mx = band_row<P>(bt.Mb, row, i, m);
      kx = band_row<P>(bt.Kb, row, i, m);
    }
    const long long off = g.base + pc * g.pstr + i * g.S;
    T1[off] = mx;
    T2[off] = kx;
  }
}

template <int P>
__global__ void __launch_bounds__(kThreads)
stiff_mid(Dims dims, int axis, int PP, int ldt, BandTab bt, double* __restrict__ T1, double* __restrict__ T2,
          const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  double* t1 = reinterpret_cast<double*>(smem);
  double* t2 = t1 + (size_t)PP * ldt;
  const STile g = stile(dims, axis, PP, blockIdx.x);
  const int m = bt.m;
  for (int e = threadIdx.x; e < PP * m; e += blockDim.x) {
    int pc, i;
    tile_index(axis, e, PP, m, pc, i);
    double a = 0.0, b = 0.0;
    if (pc < g.nvalid) {
      const long long off = g.base + pc * g.pstr + i * g.S;
      a = T1[off];
      b = T2[off];
    }
    t1[pc * ldt + i] = a;
    t2[pc * ldt + i] = b;
  }
  __syncthreads();
  Coefs<P> c;
  load_coefs<P>(bt, c);
  for (int e = threadIdx.x; e < PP * m; e += blockDim.x) {
    int pc, i;
    tile_index(axis, e, PP, m, pc, i);
    if (pc >= g.nvalid) continue;
    const double* r1 = t1 + pc * ldt;
    const double* r2 = t2 + pc * ldt;
    double mx, kx, m2;
    if (i >= bt.ilo && i < bt.ihi) {
      toeplitz_mk<P>(c, r1, i, mx, kx);
      m2 = toeplitz_m<P>(c, r2, i);
    } else {
      mx = band_row<P>(bt.Mb, r1, i, m);
      kx = band_row<P>(bt.Kb, r1, i, m);
      m2 = band_row<P>(bt.Mb, r2, i, m);
    }
    const long long off = g.base + pc * g.pstr + i * g.S;
    T1[off] = mx;
    T2[off] = kx + m2;
  }
}

template <int P>
__global__ void __launch_bounds__(kThreads)
stiff_last(Dims dims, int axis, int PP, int ldt, BandTab bt, const double* __restrict__ T1,
           const double* __restrict__ T2, double* __restrict__ out, const double* __restrict__ dotv,
           double* __restrict__ partial, const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  double* t1 = reinterpret_cast<double*>(smem);
  double* t2 = t1 + (size_t)PP * ldt;
  const STile g = stile(dims, axis, PP, blockIdx.x);
  const int m = bt.m;
  for (int e = threadIdx.x; e < PP * m; e += blockDim.x) {
    int pc, i;
    tile_index(axis, e, PP, m, pc, i);
    double a = 0.0, b = 0.0;
    if (pc < g.nvalid) {
      const long long off = g.base + pc * g.pstr + i * g.S;
      a = T1[off];
      b = T2[off];
    }
    t1[pc * ldt + i] = a;
    t2[pc * ldt + i] = b;
  }
  __syncthreads();
  Coefs<P> c;
  load_coefs<P>(bt, c);
  double dsum = 0.0;
  for (int e = threadIdx.x; e < PP * m; e += blockDim.x) {
    int pc, i;
    tile_index(axis, e, PP, m, pc, i);
    if (pc >= g.nvalid) continue;
    const double* r1 = t1 + pc * ldt;
    const double* r2 = t2 + pc * ldt;
    double v;
    if (i >= bt.ilo && i < bt.ihi) {
      v = toeplitz_k<P>(c, r1, i) + toeplitz_m<P>(c, r2, i);
    } else {
      v = band_row<P>(bt.Kb, r1, i, m) + band_row<P>(bt.Mb, r2, i, m);
    }
    const long long off = g.base + pc * g.pstr + i * g.S;
    out[off] = v;
    if (dotv != nullptr) dsum = fma(dotv[off], v, dsum);
  }
  if (dotv != nullptr) {
    __shared__ double red[kThreads / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
      partial[blockIdx.x] = s;
    }
  }
}

static size_t stiff_smem(const StiffLaunch& S, int arrays) { return (size_t)arrays * S.PP * S.ldt * sizeof(double); }

template <int P>
static cudaError_t first_p(const StiffLaunch& S, const double* u, const double* z, double* p_io, const double* beta,
                           int pmode, double* T1, double* T2, const int* done, cudaStream_t st) {
  const size_t sm = stiff_smem(S, 1);
  cudaError_t e = cudaFuncSetAttribute(stiff_first<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  stiff_first<P><<<stiff_tiles(S.dims, S.axis, S.PP), kThreads, sm, st>>>(S.dims, S.axis, S.PP, S.ldt, S.bt, u, z,
                                                                          p_io, beta, pmode, T1, T2, done);
  return cudaGetLastError();
}

template <int P>
static cudaError_t mid_p(const StiffLaunch& S, double* T1, double* T2, const int* done, cudaStream_t st) {
  const size_t sm = stiff_smem(S, 2);
  cudaError_t e = cudaFuncSetAttribute(stiff_mid<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  stiff_mid<P><<<stiff_tiles(S.dims, S.axis, S.PP), kThreads, sm, st>>>(S.dims, S.axis, S.PP, S.ldt, S.bt, T1, T2,
                                                                        done);
  return cudaGetLastError();
}

template <int P>
static cudaError_t last_p(const StiffLaunch& S, const double* T1, const double* T2, double* out, const double* dotv,
                          double* partial, const int* done, cudaStream_t st) {
  const size_t sm = stiff_smem(S, 2);
  cudaError_t e = cudaFuncSetAttribute(stiff_last<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  stiff_last<P><<<stiff_tiles(S.dims, S.axis, S.PP), kThreads, sm, st>>>(S.dims, S.axis, S.PP, S.ldt, S.bt, T1, T2,
                                                                         out, dotv, partial, done);
  return cudaGetLastError();
}

#define IFFD_DISPATCH_P(p, CALL)                                   \
  switch (p) {                                                     \
    case 1: return CALL(1); case 2: return CALL(2);                \
    case 3: return CALL(3); case 4: return CALL(4);                \
    case 5: return CALL(5); case 6: return CALL(6);                \
    case 7: return CALL(7); case 8: return CALL(8);                \
    case 9: return CALL(9); case 10: return CALL(10);              \
    case 11: return CALL(11); case 12: return CALL(12);            \
    case 13: return CALL(13); case 14: return CALL(14);            \
    case 15: return CALL(15); case 16: return CALL(16);            \
    default: return cudaErrorInvalidValue;                         \
  }

cudaError_t launch_stiff_first(const StiffLaunch& S, const double* u, const double* z, double* p_io,
                               const double* beta, int pmode, double* T1, double* T2, const int* done,
                               cudaStream_t st) {
#define CALL_FIRST(P) first_p<P>(S, u, z, p_io, beta, pmode, T1, T2, done, st)
  IFFD_DISPATCH_P(S.bt.p, CALL_FIRST)
#undef CALL_FIRST
}

cudaError_t launch_stiff_mid(const StiffLaunch& S, double* T1, double* T2, const int* done, cudaStream_t st) {
#define CALL_MID(P) mid_p<P>(S, T1, T2, done, st)
  IFFD_DISPATCH_P(S.bt.p, CALL_MID)
#undef CALL_MID
}

cudaError_t launch_stiff_last(const StiffLaunch& S, const double* T1, const double* T2, double* out,
                              const double* dotv, double* partial, const int* done, cudaStream_t st) {
#define CALL_LAST(P) last_p<P>(S, T1, T2, out, dotv, partial, done, st)
  IFFD_DISPATCH_P(S.bt.p, CALL_LAST)
#undef CALL_LAST
}

}  // namespace iffd
