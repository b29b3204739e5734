// Variable-coefficient stiffness for -div(a grad u) with the separable
// coefficient a = 1 + c s(x_1) s(x_2) s(x_3), s(x) = sin(2 pi x).
//
// With the tensor (p+1)-point Gauss rule the element integrals factorise, so
// the matrix-free sum-factorised operator equals exactly (up to rounding)
//   A_a = A^ + c sum_k (M^s x .. x K^s_k x .. x M^s),
// where M^s, K^s are the 1D mass / stiffness matrices with s under the
// integral (computed with the same Gauss rule). It is applied by the same
// three-sweep factorisation as A^, carrying four temporaries:
//   z:  T1 = M u, T2 = K u, T3 = M^s u, T4 = K^s u
//   y:  T1 <- M T1, T2 <- K T1 + M T2, T3 <- M^s T3, T4 <- K^s T3 + M^s T4
//   x:  A_a u = K T1 + M T2 + c (K^s T3 + M^s T4)
// The constant part uses the symmetric Toeplitz interior of M and K; M^s, K^s
// vary along the direction and use their stored bands.
#include "device_common.cuh"
#include "kernels.h"

namespace iffd {

namespace {

template <int P>
struct VCoefs {
  double m[P + 1];
  double k[P + 1];
};

template <int P>
__device__ __forceinline__ void vload(const BandTab& bt, VCoefs<P>& c) {
#pragma unroll
  for (int j = 0; j <= P; ++j) {
    c.m[j] = __ldg(bt.Mt + j);
    c.k[j] = __ldg(bt.Kt + j);
  }
}

// Toeplitz interior rows of M and K from shared pair sums.
template <int P>
__device__ __forceinline__ void t_mk(const VCoefs<P>& c, const double* row, int i, double& mx, double& kx) {
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

// acc + (M x)_i, the product chain continuing from acc (no separate add)
template <int P>
__device__ __forceinline__ double t_m_acc(const VCoefs<P>& c, const double* row, int i, double acc) {
  double a = fma(c.m[0], row[i], acc);
#pragma unroll
  for (int k = 1; k <= P; ++k) a = fma(c.m[k], row[i - k] + row[i + k], a);
  return a;
}

template <int P>
__device__ __forceinline__ double t_k(const VCoefs<P>& c, const double* row, int i) {
  double a = c.k[0] * row[i];
#pragma unroll
  for (int k = 1; k <= P; ++k) a = fma(c.k[k], row[i - k] + row[i + k], a);
  return a;
}

// Full band window (row i has all 2P+1 neighbours): (A x)_i and (B x)_i.
template <int P>
__device__ __forceinline__ void w_ab(const double* __restrict__ Ab, const double* __restrict__ Bb, const double* row,
                                     int i, double& ax, double& bx) {
  const double* a = Ab + (size_t)i * (2 * P + 1);
  const double* b = Bb + (size_t)i * (2 * P + 1);
  double sa = 0.0, sb = 0.0;
#pragma unroll
  for (int d = 0; d <= 2 * P; ++d) {
    const double x = row[i - P + d];
    sa = fma(__ldg(a + d), x, sa);
    sb = fma(__ldg(b + d), x, sb);
  }
  ax = sa;
  bx = sb;
}

// acc + (A x)_i over the full band window
template <int P>
__device__ __forceinline__ double w_a(const double* __restrict__ Ab, const double* row, int i, double acc = 0.0) {
  const double* a = Ab + (size_t)i * (2 * P + 1);
  double s = acc;
#pragma unroll
  for (int d = 0; d <= 2 * P; ++d) s = fma(__ldg(a + d), row[i - P + d], s);
  return s;
}

// Any row (clipped window).
template <int P>
__device__ __forceinline__ double g_a(const double* __restrict__ Ab, const double* row, int i, int m) {
  const double* a = Ab + (size_t)i * (2 * P + 1);
  double s = 0.0;
  const int j0 = max(0, i - P), j1 = min(m - 1, i + P);
  for (int j = j0; j <= j1; ++j) s = fma(__ldg(a + (j - i + P)), row[j], s);
  return s;
}

__device__ __forceinline__ void vcoords(int axis, int e, int PP, int n, int& pc, int& r) {
  if (axis == 0) { pc = e / n; r = e - pc * n; }
  else { r = e / PP; pc = e - r * PP; }
}

}  // namespace

template <int P>
__global__ void __launch_bounds__(kThreads)
vstiff_first(Dims dims, int axis, int PP, int ldt, BandTab bt, WBandTab wb, const double* __restrict__ u,
             const double* __restrict__ z, double* __restrict__ p_io, const double* __restrict__ betap, int pmode,
             double* __restrict__ T1, double* __restrict__ T2, double* __restrict__ T3, double* __restrict__ T4,
             const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  double* tile = reinterpret_cast<double*>(smem);
  __shared__ long long pbase[64];
  const TileInfo g = tile_setup(dims, axis, PP, blockIdx.x, pbase, nullptr, nullptr);
  __syncthreads();
  const int m = bt.m;
  const double beta = (pmode == 2) ? *betap : 0.0;
  for (int e = threadIdx.x; e < PP * m; e += blockDim.x) {
    int pc, i;
    vcoords(axis, e, PP, m, pc, i);
    double v = 0.0;
    if (pc < g.nvalid) {
      const long long off = pbase[pc] + i * g.S;
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
  VCoefs<P> c;
  vload<P>(bt, c);
  const int nint = bt.ihi - bt.ilo, nbd = m - nint;
  for (int e = threadIdx.x; e < PP * nint; e += blockDim.x) {
    int pc, r;
    vcoords(axis, e, PP, nint, pc, r);
    if (pc >= g.nvalid) continue;
    const int i = bt.ilo + r;
    const double* row = tile + pc * ldt;
    double mx, kx, msx, ksx;
    t_mk<P>(c, row, i, mx, kx);
    w_ab<P>(wb.Msb, wb.Ksb, row, i, msx, ksx);
    const long long off = pbase[pc] + i * g.S;
    T1[off] = mx;
    T2[off] = kx;
    T3[off] = msx;
    T4[off] = ksx;
  }
  for (int e = threadIdx.x; e < PP * nbd; e += blockDim.x) {
    int pc, r;
    vcoords(axis, e, PP, nbd, pc, r);
    if (pc >= g.nvalid) continue;
    const int i = (r < bt.ilo) ? r : bt.ihi + (r - bt.ilo);
    const double* row = tile + pc * ldt;
    const long long off = pbase[pc] + i * g.S;
    T1[off] = g_a<P>(bt.Mb, row, i, m);
    T2[off] = g_a<P>(bt.Kb, row, i, m);
    T3[off] = g_a<P>(wb.Msb, row, i, m);
    T4[off] = g_a<P>(wb.Ksb, row, i, m);
  }
}

template <int P>
__global__ void __launch_bounds__(kThreads)
vstiff_mid(Dims dims, int axis, int PP, int ldt, BandTab bt, WBandTab wb, double* __restrict__ T1,
           double* __restrict__ T2, double* __restrict__ T3, double* __restrict__ T4, const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  double* t1 = reinterpret_cast<double*>(smem);
  double* t2 = t1 + (size_t)PP * ldt;
  double* t3 = t2 + (size_t)PP * ldt;
  double* t4 = t3 + (size_t)PP * ldt;
  __shared__ long long pbase[64];
  const TileInfo g = tile_setup(dims, axis, PP, blockIdx.x, pbase, nullptr, nullptr);
  __syncthreads();
  const int m = bt.m;
  for (int e = threadIdx.x; e < PP * m; e += blockDim.x) {
    int pc, i;
    vcoords(axis, e, PP, m, pc, i);
    const long long off = pbase[pc] + i * g.S;
    t1[pc * ldt + i] = T1[off];
    t2[pc * ldt + i] = T2[off];
    t3[pc * ldt + i] = T3[off];
    t4[pc * ldt + i] = T4[off];
  }
  __syncthreads();
  VCoefs<P> c;
  vload<P>(bt, c);
  const int nint = bt.ihi - bt.ilo, nbd = m - nint;
  for (int e = threadIdx.x; e < PP * nint; e += blockDim.x) {
    int pc, r;
    vcoords(axis, e, PP, nint, pc, r);
    if (pc >= g.nvalid) continue;
    const int i = bt.ilo + r;
    double mx, kx, ms3, ks3;
    t_mk<P>(c, t1 + pc * ldt, i, mx, kx);
    w_ab<P>(wb.Msb, wb.Ksb, t3 + pc * ldt, i, ms3, ks3);
    const long long off = pbase[pc] + i * g.S;
    T1[off] = mx;
    T2[off] = t_m_acc<P>(c, t2 + pc * ldt, i, kx);            // K T1 + M T2
    T3[off] = ms3;
    T4[off] = w_a<P>(wb.Msb, t4 + pc * ldt, i, ks3);           // K^s T3 + M^s T4
  }
  for (int e = threadIdx.x; e < PP * nbd; e += blockDim.x) {
    int pc, r;
    vcoords(axis, e, PP, nbd, pc, r);
    if (pc >= g.nvalid) continue;
    const int i = (r < bt.ilo) ? r : bt.ihi + (r - bt.ilo);
    const long long off = pbase[pc] + i * g.S;
    const double* r1 = t1 + pc * ldt;
    const double* r2 = t2 + pc * ldt;
    const double* r3 = t3 + pc * ldt;
    const double* r4 = t4 + pc * ldt;
    T1[off] = g_a<P>(bt.Mb, r1, i, m);
    T2[off] = g_a<P>(bt.Kb, r1, i, m) + g_a<P>(bt.Mb, r2, i, m);
    T3[off] = g_a<P>(wb.Msb, r3, i, m);
    T4[off] = g_a<P>(wb.Ksb, r3, i, m) + g_a<P>(wb.Msb, r4, i, m);
  }
}

template <int P>
__global__ void __launch_bounds__(kThreads)
vstiff_last(Dims dims, int axis, int PP, int ldt, BandTab bt, WBandTab wb, const double* __restrict__ T1,
            const double* __restrict__ T2, const double* __restrict__ T3, const double* __restrict__ T4,
            double* __restrict__ out, const double* __restrict__ dotv, double* __restrict__ partial,
            const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  double* t1 = reinterpret_cast<double*>(smem);
  double* t2 = t1 + (size_t)PP * ldt;
  double* t3 = t2 + (size_t)PP * ldt;
  double* t4 = t3 + (size_t)PP * ldt;
  __shared__ long long pbase[64];
  const TileInfo g = tile_setup(dims, axis, PP, blockIdx.x, pbase, nullptr, nullptr);
  __syncthreads();
  const int m = bt.m;
  for (int e = threadIdx.x; e < PP * m; e += blockDim.x) {
    int pc, i;
    vcoords(axis, e, PP, m, pc, i);
    const long long off = pbase[pc] + i * g.S;
    t1[pc * ldt + i] = T1[off];
    t2[pc * ldt + i] = T2[off];
    t3[pc * ldt + i] = T3[off];
    t4[pc * ldt + i] = T4[off];
  }
  __syncthreads();
  VCoefs<P> c;
  vload<P>(bt, c);
  const double cc = wb.c;
  double dsum = 0.0;
  const int nint = bt.ihi - bt.ilo, nbd = m - nint;
  for (int e = threadIdx.x; e < PP * nint; e += blockDim.x) {
    int pc, r;
    vcoords(axis, e, PP, nint, pc, r);
    if (pc >= g.nvalid) continue;
    const int i = bt.ilo + r;
    const double cpart = t_m_acc<P>(c, t2 + pc * ldt, i, t_k<P>(c, t1 + pc * ldt, i));
    const double wpart = w_a<P>(wb.Msb, t4 + pc * ldt, i, w_a<P>(wb.Ksb, t3 + pc * ldt, i));
    const double v = fma(cc, wpart, cpart);
    const long long off = pbase[pc] + i * g.S;
    out[off] = v;
    if (dotv != nullptr) dsum = fma(dotv[off], v, dsum);
  }
  for (int e = threadIdx.x; e < PP * nbd; e += blockDim.x) {
    int pc, r;
    vcoords(axis, e, PP, nbd, pc, r);
    if (pc >= g.nvalid) continue;
    const int i = (r < bt.ilo) ? r : bt.ihi + (r - bt.ilo);
    const double cpart = g_a<P>(bt.Kb, t1 + pc * ldt, i, m) + g_a<P>(bt.Mb, t2 + pc * ldt, i, m);
    const double wpart = g_a<P>(wb.Ksb, t3 + pc * ldt, i, m) + g_a<P>(wb.Msb, t4 + pc * ldt, i, m);
    const double v = fma(cc, wpart, cpart);
    const long long off = pbase[pc] + i * g.S;
    out[off] = v;
    if (dotv != nullptr) dsum = fma(dotv[off], v, dsum);
  }
  if (dotv != nullptr) {
    __shared__ double red[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
      partial[blockIdx.x] = s;
    }
  }
}

namespace {

size_t vsmem(const StiffLaunch& S, int arrays) { return (size_t)arrays * S.PP * S.ldt * sizeof(double); }

template <int P>
cudaError_t vfirst_p(const StiffLaunch& S, const WBandTab& wb, const double* u, const double* z, double* p_io,
                     const double* beta, int pmode, double* T1, double* T2, double* T3, double* T4,
                     const int* done, cudaStream_t st) {
  const size_t sm = vsmem(S, 1);
  cudaError_t e = cudaFuncSetAttribute(vstiff_first<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  vstiff_first<P><<<stiff_tiles(S.dims, S.axis, S.PP), kThreads, sm, st>>>(
      S.dims, S.axis, S.PP, S.ldt, S.bt, wb, u, z, p_io, beta, pmode, T1, T2, T3, T4, done);
  return cudaGetLastError();
}

template <int P>
cudaError_t vmid_p(const StiffLaunch& S, const WBandTab& wb, double* T1, double* T2, double* T3, double* T4,
                   const int* done, cudaStream_t st) {
  const size_t sm = vsmem(S, 4);
  cudaError_t e = cudaFuncSetAttribute(vstiff_mid<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  vstiff_mid<P><<<stiff_tiles(S.dims, S.axis, S.PP), kThreads, sm, st>>>(S.dims, S.axis, S.PP, S.ldt, S.bt, wb,
                                                                         T1, T2, T3, T4, done);
  return cudaGetLastError();
}

template <int P>
cudaError_t vlast_p(const StiffLaunch& S, const WBandTab& wb, const double* T1, const double* T2, const double* T3,
                    const double* T4, double* out, const double* dotv, double* partial, const int* done,
                    cudaStream_t st) {
  const size_t sm = vsmem(S, 4);
  cudaError_t e = cudaFuncSetAttribute(vstiff_last<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  vstiff_last<P><<<stiff_tiles(S.dims, S.axis, S.PP), kThreads, sm, st>>>(
      S.dims, S.axis, S.PP, S.ldt, S.bt, wb, T1, T2, T3, T4, out, dotv, partial, done);
  return cudaGetLastError();
}

}  // namespace

#define IFFD_VDISPATCH(p, CALL)                                    \
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

cudaError_t launch_vstiff_first(const StiffLaunch& S, const WBandTab& wb, const double* u, const double* z,
                                double* p_io, const double* beta, int pmode, double* T1, double* T2, double* T3,
                                double* T4, const int* done, cudaStream_t st) {
#define VF(P) vfirst_p<P>(S, wb, u, z, p_io, beta, pmode, T1, T2, T3, T4, done, st)
  IFFD_VDISPATCH(S.bt.p, VF)
#undef VF
}

cudaError_t launch_vstiff_mid(const StiffLaunch& S, const WBandTab& wb, double* T1, double* T2, double* T3,
                              double* T4, const int* done, cudaStream_t st) {
#define VM(P) vmid_p<P>(S, wb, T1, T2, T3, T4, done, st)
  IFFD_VDISPATCH(S.bt.p, VM)
#undef VM
}

cudaError_t launch_vstiff_last(const StiffLaunch& S, const WBandTab& wb, const double* T1, const double* T2,
                               const double* T3, const double* T4, double* out, const double* dotv,
                               double* partial, const int* done, cudaStream_t st) {
#define VL(P) vlast_p<P>(S, wb, T1, T2, T3, T4, out, dotv, partial, done, st)
  IFFD_VDISPATCH(S.bt.p, VL)
#undef VL
}

}  // namespace iffd
