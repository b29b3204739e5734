// Device bodies of the Kronecker stiffness sweeps (eq. "system_matrix"),
// shared by the sweep kernels (stiffness.cu) and the persistent engine
// launch (persist.cu). CG selects L2-coherent loads of the solver data (see
// ldd in device_common.cuh).
#pragma once

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
__device__ __forceinline__ double toeplitz_k(const Coefs<P>& c, const double* row, int i) {
  double a = c.k[0] * row[i];
#pragma unroll
  for (int k = 1; k <= P; ++k) a = fma(c.k[k], row[i - k] + row[i + k], a);
  return a;
}

// acc + (M x)_i: the product chain continues from acc, so the sum of two
// banded products costs no separate multiply and add (2P + 1 FP64
// instructions for this product, against 2P + 2 for a product and a sum).
template <int P>
__device__ __forceinline__ double toeplitz_m_acc(const Coefs<P>& c, const double* row, int i, double acc) {
  double a = fma(c.m[0], row[i], acc);
#pragma unroll
  for (int k = 1; k <= P; ++k) a = fma(c.m[k], row[i - k] + row[i + k], a);
  return a;
}


// Loads one array's tile: element (pc, i) of pencil pc (x fastest among
// pencils for axis > 0, so a warp reads consecutive addresses).
__device__ __forceinline__ void tile_coords(int axis, int e, int PP, int m, int& pc, int& i) {
  if (axis == 0) { pc = e / m; i = e - pc * m; }
  else { i = e / PP; pc = e - i * PP; }
}

// Work split of the compute loops: first every interior (Toeplitz) row of
// every pencil, then the boundary rows, so that no warp mixes the two
// code paths. Item e of a region of nr rows starting at row r0:
__device__ __forceinline__ void region_coords(int axis, int e, int PP, int nr, int& pc, int& r) {
  if (axis == 0) { pc = e / nr; r = e - pc * nr; }
  else { r = e / PP; pc = e - r * PP; }
}

// pmode: 0 -> u = u; 1 -> u = z, p <- z; 2 -> u = z + beta p, p <- u
template <int P, bool CG = false>
__device__ __forceinline__ void first_body(const Dims& dims, int axis, int PP, int ldt, const BandTab& bt,
                                           const double* __restrict__ u, const double* __restrict__ z,
                                           double* __restrict__ p_io, const double* __restrict__ betap, int pmode,
                                           double* __restrict__ T1, double* __restrict__ T2, long long tile_id,
                                           unsigned char* smem) {
  double* tile = reinterpret_cast<double*>(smem);
  __shared__ long long pbase[64];
  const TileInfo g = tile_setup(dims, axis, PP, tile_id, pbase, nullptr, nullptr);
  __syncthreads();
  const int m = bt.m;
  const double beta = (pmode == 2) ? ldd<CG>(betap) : 0.0;
  for (int e = threadIdx.x; e < PP * m; e += blockDim.x) {
    int pc, i;
    tile_coords(axis, e, PP, m, pc, i);
    double v = 0.0;
    if (pc < g.nvalid) {
      const long long off = pbase[pc] + i * g.S;
      if (pmode == 0) {
        v = ldd<CG>(u + off);
      } else if (pmode == 1) {
        v = ldd<CG>(z + off);
        p_io[off] = v;
      } else {
        v = fma(beta, ldd<CG>(p_io + off), ldd<CG>(z + off));
        p_io[off] = v;
      }
    }
    tile[pc * ldt + i] = v;
  }
  __syncthreads();
  Coefs<P> c;
  load_coefs<P>(bt, c);
  const int nint = bt.ihi - bt.ilo, nbd = m - nint;
  for (int e = threadIdx.x; e < PP * nint; e += blockDim.x) {
    int pc, r;
    region_coords(axis, e, PP, nint, pc, r);
    if (pc >= g.nvalid) continue;
    const int i = bt.ilo + r;
    double mx, kx;
    toeplitz_mk<P>(c, tile + pc * ldt, i, mx, kx);
    const long long off = pbase[pc] + i * g.S;
    T1[off] = mx;
    T2[off] = kx;
  }
  for (int e = threadIdx.x; e < PP * nbd; e += blockDim.x) {
    int pc, r;
    region_coords(axis, e, PP, nbd, pc, r);
    if (pc >= g.nvalid) continue;
    const int i = (r < bt.ilo) ? r : bt.ihi + (r - bt.ilo);
    const double* row = tile + pc * ldt;
    const long long off = pbase[pc] + i * g.S;
    T1[off] = band_row<P>(bt.Mb, row, i, m);
    T2[off] = band_row<P>(bt.Kb, row, i, m);
  }
}

template <int P, bool CG = false>
__device__ __forceinline__ void mid_body(const Dims& dims, int axis, int PP, int ldt, const BandTab& bt,
                                         double* __restrict__ T1, double* __restrict__ T2, long long tile_id,
                                         unsigned char* smem) {
  double* t1 = reinterpret_cast<double*>(smem);
  double* t2 = t1 + (size_t)PP * ldt;
  __shared__ long long pbase[64];
  const TileInfo g = tile_setup(dims, axis, PP, tile_id, pbase, nullptr, nullptr);
  __syncthreads();
  const int m = bt.m;
  for (int e = threadIdx.x; e < PP * m; e += blockDim.x) {
    int pc, i;
    tile_coords(axis, e, PP, m, pc, i);
    const long long off = pbase[pc] + i * g.S;
    t1[pc * ldt + i] = ldd<CG>(T1 + off);
    t2[pc * ldt + i] = ldd<CG>(T2 + off);
  }
  __syncthreads();
  Coefs<P> c;
  load_coefs<P>(bt, c);
  const int nint = bt.ihi - bt.ilo, nbd = m - nint;
  for (int e = threadIdx.x; e < PP * nint; e += blockDim.x) {
    int pc, r;
    region_coords(axis, e, PP, nint, pc, r);
    if (pc >= g.nvalid) continue;
    const int i = bt.ilo + r;
    double mx, kx;
    toeplitz_mk<P>(c, t1 + pc * ldt, i, mx, kx);
    const long long off = pbase[pc] + i * g.S;
    T1[off] = mx;
    T2[off] = toeplitz_m_acc<P>(c, t2 + pc * ldt, i, kx);  // K T1 + M T2
  }
  for (int e = threadIdx.x; e < PP * nbd; e += blockDim.x) {
    int pc, r;
    region_coords(axis, e, PP, nbd, pc, r);
    if (pc >= g.nvalid) continue;
    const int i = (r < bt.ilo) ? r : bt.ihi + (r - bt.ilo);
    const double* r1 = t1 + pc * ldt;
    const double* r2 = t2 + pc * ldt;
    const long long off = pbase[pc] + i * g.S;
    T1[off] = band_row<P>(bt.Mb, r1, i, m);
    T2[off] = band_row<P>(bt.Kb, r1, i, m) + band_row<P>(bt.Mb, r2, i, m);
  }
}

template <int P, bool CG = false>
__device__ __forceinline__ void last_body(const Dims& dims, int axis, int PP, int ldt, const BandTab& bt,
                                          const double* __restrict__ T1, const double* __restrict__ T2,
                                          double* __restrict__ out, const double* __restrict__ dotv,
                                          double* __restrict__ partial, long long tile_id, int ptile,
                                          unsigned char* smem) {
  double* t1 = reinterpret_cast<double*>(smem);
  double* t2 = t1 + (size_t)PP * ldt;
  __shared__ long long pbase[64];
  const TileInfo g = tile_setup(dims, axis, PP, tile_id, pbase, nullptr, nullptr);
  __syncthreads();
  const int m = bt.m;
  for (int e = threadIdx.x; e < PP * m; e += blockDim.x) {
    int pc, i;
    tile_coords(axis, e, PP, m, pc, i);
    const long long off = pbase[pc] + i * g.S;
    t1[pc * ldt + i] = ldd<CG>(T1 + off);
    t2[pc * ldt + i] = ldd<CG>(T2 + off);
  }
  __syncthreads();
  Coefs<P> c;
  load_coefs<P>(bt, c);
  double dsum = 0.0;
  const int nint = bt.ihi - bt.ilo, nbd = m - nint;
  for (int e = threadIdx.x; e < PP * nint; e += blockDim.x) {
    int pc, r;
    region_coords(axis, e, PP, nint, pc, r);
    if (pc >= g.nvalid) continue;
    const int i = bt.ilo + r;
    const double v = toeplitz_m_acc<P>(c, t2 + pc * ldt, i, toeplitz_k<P>(c, t1 + pc * ldt, i));  // K T1 + M T2
    const long long off = pbase[pc] + i * g.S;
    out[off] = v;
    if (dotv != nullptr) dsum = fma(ldd<CG>(dotv + off), v, dsum);
  }
  for (int e = threadIdx.x; e < PP * nbd; e += blockDim.x) {
    int pc, r;
    region_coords(axis, e, PP, nbd, pc, r);
    if (pc >= g.nvalid) continue;
    const int i = (r < bt.ilo) ? r : bt.ihi + (r - bt.ilo);
    const double v = band_row<P>(bt.Kb, t1 + pc * ldt, i, m) + band_row<P>(bt.Mb, t2 + pc * ldt, i, m);
    const long long off = pbase[pc] + i * g.S;
    out[off] = v;
    if (dotv != nullptr) dsum = fma(ldd<CG>(dotv + off), v, dsum);
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
      partial[ptile] = s;
    }
  }
}


}  // namespace iffd
