// Stiffness with a general symmetric coefficient C(x) sampled at the tensor
// Gauss points: A u = sum_{k,l} G_k^T diag(w C_kl) G_l u, where G_k is the
// k-th partial derivative of the kept B-splines at the Gauss points (the
// Galerkin form of Section 2 with the coefficient under the integral; a
// geometry map of Section 7 pulled back to the parameter domain has this
// form). Applied by sum factorisation on the grid of Gauss points: one
// sparse 1D matrix (B, D or their transposes: at most p+1 entries per point,
// (p+1)^2 per basis function) per sweep, each sweep along one direction of a
// d-dimensional array with x fastest.
//
// 3D forward: U_B = B_x u, U_D = D_x u; V_BB = B_y U_B, V_BD = D_y U_B,
// V_DB = B_y U_D; then along z, in one pass element by element, g = (B_z V_DB,
// B_z V_BD, D_z V_BB), h = w C g and the transposed z products, so that the
// Gauss-grid values never reach memory. Backward along y and x with the
// transposes, the two contributions of each sweep summed in one pass.
#include <algorithm>
#include <cstring>
#include <vector>

#include "device_common.cuh"
#include "kernels.h"
#include "plan.h"

namespace iffd {

namespace {

// GS_ONE: out = A in; GS_TWO_OUT: out = A in, out2 = A2 in (same pattern);
// GS_TWO_IN: out = A in + A2 in2.
enum GenSweep : int { GS_ONE = 0, GS_TWO_OUT = 1, GS_TWO_IN = 2 };

// Launch shape of the sweeps and the pointwise step: threads along x (the
// fastest index, coalesced), one (y, z) row of the output per block row, so
// that the row's offsets are computed once per block and not per element.
template <int MODE>
__global__ void __launch_bounds__(kThreads)
gen_sweep(const double* __restrict__ in, const double* __restrict__ in2, double* __restrict__ out,
          double* __restrict__ out2, int o0, int o1, int o2, int in_len, int axis, const int* __restrict__ rp,
          const int* __restrict__ col, const double* __restrict__ val, const double* __restrict__ val2,
          const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  const long long n0 = axis == 0 ? in_len : o0, n1 = axis == 1 ? in_len : o1;
  const long long s_ax = axis == 0 ? 1 : (axis == 1 ? n0 : n0 * n1);
  const int rows = o1 * o2;
  for (int rr = blockIdx.y; rr < rows; rr += gridDim.y) {
    const int i1 = rr % o1, i2 = rr / o1;
    const long long rbase = (axis == 1 ? 0 : (long long)i1 * n0) + (axis == 2 ? 0 : (long long)i2 * n0 * n1);
    double* orow = out + (long long)rr * o0;
    double* orow2 = (MODE == GS_TWO_OUT) ? out2 + (long long)rr * o0 : nullptr;
    for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < o0; i0 += gridDim.x * blockDim.x) {
      const long long base = rbase + (axis == 0 ? 0 : i0);
      const int row = axis == 0 ? i0 : (axis == 1 ? i1 : i2);
      double s = 0.0, s2 = 0.0;
      const int k1 = __ldg(rp + row + 1);
      int k = __ldg(rp + row);
      // four entries per step: their loads are issued before the first FMA
      // waits, so a row costs about one memory latency per four entries
      for (; k + 4 <= k1; k += 4) {
        double v[4], v2[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const long long at = base + (long long)__ldg(col + k + e) * s_ax;
          v[e] = in[at];
          if (MODE == GS_TWO_IN) v2[e] = in2[at];
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          s = fma(__ldg(val + k + e), v[e], s);
          if (MODE == GS_TWO_OUT) s2 = fma(__ldg(val2 + k + e), v[e], s2);
          if (MODE == GS_TWO_IN) s = fma(__ldg(val2 + k + e), v2[e], s);
        }
      }
      for (; k < k1; ++k) {
        const long long at = base + (long long)__ldg(col + k) * s_ax;
        const double v = in[at];
        s = fma(__ldg(val + k), v, s);
        if (MODE == GS_TWO_OUT) s2 = fma(__ldg(val2 + k), v, s2);
        if (MODE == GS_TWO_IN) s = fma(__ldg(val2 + k), in2[at], s);
      }
      orow[i0] = s;
      if (MODE == GS_TWO_OUT) orow2[i0] = s2;
    }
  }
}

// h = w C g at Gauss point t (C: ncomp components of `total` points each).
template <int D>
__device__ __forceinline__ void coef_apply(double* g, const double* __restrict__ C, int ncomp, long long total,
                                           long long t, double w) {
  if (ncomp == 1) {
    const double wc = w * __ldg(C + t);
#pragma unroll
    for (int k = 0; k < D; ++k) g[k] = wc * g[k];
    return;
  }
  if (D == 2) {
    const double c11 = __ldg(C + t), c12 = __ldg(C + total + t), c22 = __ldg(C + 2 * total + t);
    const double h0 = fma(c12, g[1], c11 * g[0]), h1 = fma(c22, g[1], c12 * g[0]);
    g[0] = w * h0;
    g[1] = w * h1;
  } else {
    const double c11 = __ldg(C + t), c12 = __ldg(C + total + t), c13 = __ldg(C + 2 * total + t);
    const double c22 = __ldg(C + 3 * total + t), c23 = __ldg(C + 4 * total + t), c33 = __ldg(C + 5 * total + t);
    const double h0 = fma(c13, g[2], fma(c12, g[1], c11 * g[0]));
    const double h1 = fma(c23, g[2], fma(c22, g[1], c12 * g[0]));
    const double h2 = fma(c33, g[2], fma(c23, g[1], c13 * g[0]));
    g[0] = w * h0;
    g[1] = w * h1;
    g[2] = w * h2;
  }
}

// The last direction (D-1) in one pass: forward sweep, Gauss-point step and
// transposed sweep. A thread owns one column of the Gauss grid along that
// direction (a fixed (x, y) Gauss point in 3D, a fixed x Gauss point in 2D)
// and walks its elements in order. The p+1 Gauss points of element e share the
// element's basis functions (cnt <= p+1 columns of the sparse 1D matrices):
// at each point the thread forms g (3D: B_z in0, B_z in1, D_z in2; 2D: B_y in0,
// D_y in1), h = w C g, and accumulates the transposed products for those
// functions in registers; the element's sums are then added to the thread's
// own entries of out0..out2 (no other thread writes them). 3D: out = W_DB,
// W_BD, W_BB; 2D: out = X_D, X_B. Inputs and outputs have the shape
// (q0[, q1], m_last), x fastest; w = w_z (w_y w_x).
// P1: p + 1 (compile time, so that the per-thread arrays stay in registers).
constexpr int kFusedThreads = 128;

template <int D, int P1>
__global__ void __launch_bounds__(kFusedThreads)
gen_last_fused(const double* __restrict__ in0, const double* __restrict__ in1, const double* __restrict__ in2,
               double* __restrict__ out0, double* __restrict__ out1, double* __restrict__ out2, int q0, int q1,
               int nel, int m_last, const int* __restrict__ rp, const int* __restrict__ col,
               const double* __restrict__ bv, const double* __restrict__ dv, const double* __restrict__ C, int ncomp,
               const double* __restrict__ w0, const double* __restrict__ w1, const double* __restrict__ wl,
               const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  const long long ncol = (D == 3) ? (long long)q0 * q1 : q0;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= ncol) return;
  const int i0 = (int)(c % q0);
  const double wxy = (D == 3) ? __ldg(w1 + c / q0) * __ldg(w0 + i0) : __ldg(w0 + i0);
  const long long s = ncol;                       // stride of the last direction
  const long long total = ncol * (long long)nel * P1;  // Gauss points (one coefficient component)
  for (int j = 0; j < m_last; ++j) {
    out0[c + j * s] = 0.0;
    out1[c + j * s] = 0.0;
    if (D == 3) out2[c + j * s] = 0.0;
  }
  for (int e = 0; e < nel; ++e) {
    const int qa = e * P1;
    const int k0 = __ldg(rp + qa), cnt = __ldg(rp + qa + 1) - k0;
    long long at[P1];
    double a0[P1], a1[P1], a2[P1];
    double acc0[P1], acc1[P1], acc2[P1];
#pragma unroll
    for (int t = 0; t < P1; ++t) {
      acc0[t] = acc1[t] = acc2[t] = 0.0;
      if (t < cnt) {
        at[t] = c + (long long)__ldg(col + k0 + t) * s;
        a0[t] = in0[at[t]];
        a1[t] = in1[at[t]];
        if (D == 3) a2[t] = in2[at[t]];
      }
    }
    for (int qq = 0; qq < P1; ++qq) {
      const int q = qa + qq, kq = k0 + qq * cnt;  // every point of the element has the same cnt columns
      double g[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int t = 0; t < P1; ++t)
        if (t < cnt) {
          const double b = __ldg(bv + kq + t), dd = __ldg(dv + kq + t);
          g[0] = fma(b, a0[t], g[0]);
          if (D == 3) {
            g[1] = fma(b, a1[t], g[1]);
            g[2] = fma(dd, a2[t], g[2]);
          } else {
            g[1] = fma(dd, a1[t], g[1]);
          }
        }
      coef_apply<D>(g, C, ncomp, total, c + (long long)q * s, __ldg(wl + q) * wxy);
#pragma unroll
      for (int t = 0; t < P1; ++t)
        if (t < cnt) {
          const double b = __ldg(bv + kq + t), dd = __ldg(dv + kq + t);
          acc0[t] = fma(b, g[0], acc0[t]);
          if (D == 3) {
            acc1[t] = fma(b, g[1], acc1[t]);
            acc2[t] = fma(dd, g[2], acc2[t]);
          } else {
            acc1[t] = fma(dd, g[1], acc1[t]);
          }
        }
    }
#pragma unroll
    for (int t = 0; t < P1; ++t)
      if (t < cnt) {
        out0[at[t]] += acc0[t];
        out1[at[t]] += acc1[t];
        if (D == 3) out2[at[t]] += acc2[t];
      }
  }
}

template <int D, int P1>
cudaError_t launch_fused_p(const double* in0, const double* in1, const double* in2, double* out0, double* out1,
                           double* out2, int q0, int q1, int nel, int m_last, const GenAxis& L, const double* C,
                           int ncomp, const double* w0, const double* w1, const int* done, cudaStream_t st) {
  const long long ncol = (D == 3) ? (long long)q0 * q1 : q0;
  const int blocks = (int)((ncol + kFusedThreads - 1) / kFusedThreads);
  gen_last_fused<D, P1><<<blocks, kFusedThreads, 0, st>>>(in0, in1, in2, out0, out1, out2, q0, q1, nel, m_last, L.rp,
                                                          L.col, L.bv, L.dv, C, ncomp, w0, w1, L.w, done);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_fused(int p1, const double* in0, const double* in1, const double* in2, double* out0,
                         double* out1, double* out2, int q0, int q1, int nel, int m_last, const GenAxis& L,
                         const double* C, int ncomp, const double* w0, const double* w1, const int* done,
                         cudaStream_t st) {
#define IFFD_FUSED(PP)                                                                                          \
  case PP:                                                                                                     \
    return launch_fused_p<D, PP>(in0, in1, in2, out0, out1, out2, q0, q1, nel, m_last, L, C, ncomp, w0, w1, done, \
                                 st);
  switch (p1) {
    IFFD_FUSED(2) IFFD_FUSED(3) IFFD_FUSED(4) IFFD_FUSED(5) IFFD_FUSED(6) IFFD_FUSED(7)
    IFFD_FUSED(8) IFFD_FUSED(9) IFFD_FUSED(10) IFFD_FUSED(11) IFFD_FUSED(12)
    default: return cudaErrorInvalidValue;
  }
#undef IFFD_FUSED
}

// p = z (mode 1) or p = z + beta p (mode 2), beta read on the device.
__global__ void __launch_bounds__(kThreads)
gen_pupdate(const double* __restrict__ z, double* __restrict__ p, const SolveState* __restrict__ S, int mode,
            long long N, const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  const double beta = (mode == 2) ? S->beta : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    p[i] = (mode == 2) ? fma(beta, p[i], z[i]) : z[i];
}

// Block of up to 256 threads along x (128 for short rows) and a grid of
// (x blocks, rows), the rows capped at the grid's y limit (grid-stride loop).
struct Shape2 {
  dim3 grid, block;
};
Shape2 shape_for(long long o0, long long rows) {
  const int tb = o0 > 128 ? kThreads : 128;
  const unsigned gx = (unsigned)((o0 + tb - 1) / tb);
  const unsigned gy = (unsigned)std::min<long long>(rows, 65535);
  return {dim3(gx, gy), dim3(tb)};
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// Device tables of every direction in one allocation.
int build_general_tables(Plan* P, cudaStream_t st) {
  std::vector<char> bytes;
  size_t off[3][10];
  auto add = [&](const void* src, size_t n) {
    const size_t o = al256(bytes.size());
    bytes.resize(o + std::max(n, (size_t)8), 0);
    if (n) std::memcpy(bytes.data() + o, src, n);
    return o;
  };
  QuadAxis Q[3];
  for (int a = 0; a < P->d; ++a) {
    build_quad_axis(P->host[a], &Q[a]);
    off[a][0] = add(Q[a].rp.data(), Q[a].rp.size() * sizeof(int));
    off[a][1] = add(Q[a].col.data(), Q[a].col.size() * sizeof(int));
    off[a][2] = add(Q[a].bv.data(), Q[a].bv.size() * sizeof(double));
    off[a][3] = add(Q[a].dv.data(), Q[a].dv.size() * sizeof(double));
    off[a][4] = add(Q[a].trp.data(), Q[a].trp.size() * sizeof(int));
    off[a][5] = add(Q[a].tcol.data(), Q[a].tcol.size() * sizeof(int));
    off[a][6] = add(Q[a].tbv.data(), Q[a].tbv.size() * sizeof(double));
    off[a][7] = add(Q[a].tdv.data(), Q[a].tdv.size() * sizeof(double));
    off[a][8] = add(Q[a].w.data(), Q[a].w.size() * sizeof(double));
  }
  char* dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, bytes.size());
  if (e == cudaSuccess) e = cudaMemcpyAsync(dev, bytes.data(), bytes.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    if (dev) cudaFree(dev);
    return cuda_fail(e, "general-coefficient tables");
  }
  P->gen_mem = dev;
  for (int a = 0; a < P->d; ++a) {
    GenAxis& g = P->gen[a];
    g.nq = Q[a].nq;
    g.m = Q[a].m;
    g.rp = reinterpret_cast<const int*>(dev + off[a][0]);
    g.col = reinterpret_cast<const int*>(dev + off[a][1]);
    g.bv = reinterpret_cast<const double*>(dev + off[a][2]);
    g.dv = reinterpret_cast<const double*>(dev + off[a][3]);
    g.trp = reinterpret_cast<const int*>(dev + off[a][4]);
    g.tcol = reinterpret_cast<const int*>(dev + off[a][5]);
    g.tbv = reinterpret_cast<const double*>(dev + off[a][6]);
    g.tdv = reinterpret_cast<const double*>(dev + off[a][7]);
    g.w = reinterpret_cast<const double*>(dev + off[a][8]);
  }
  return IFFD_OK;
}

// Scratch of one application: 3D, two arrays with direction 0 at the Gauss
// points and six with directions 0 and 1; 2D, four with direction 0 at the
// Gauss points. No array spans the whole Gauss grid.
size_t general_ws_bytes(const Plan* P) {
  const long long q0 = P->gen[0].nq, q1 = P->gen[1].nq, m1 = P->gen[1].m;
  if (P->d == 2) return 4 * al256(q0 * m1 * 8);
  const long long m2 = P->gen[2].m;
  return 2 * al256(q0 * m1 * m2 * 8) + 6 * al256(q0 * q1 * m2 * 8);
}

int run_general(Plan* P, const double* C, int ncomp, const double* u, double* Au, void* gws, cudaStream_t st,
                const int* done) {
  const GenAxis* G = P->gen;
  const int d = P->d;
  char* b = static_cast<char*>(gws);
  const long long m0 = G[0].m, m1 = G[1].m, q0 = G[0].nq, q1 = G[1].nq;
  const long long m2 = d == 3 ? G[2].m : 1, q2 = d == 3 ? G[2].nq : 1;
  auto take = [&](size_t n) {
    double* p = reinterpret_cast<double*>(b);
    b += al256(n * 8);
    return p;
  };
  double* U[2] = {take(q0 * m1 * m2), take(q0 * m1 * m2)};
  double* V[3] = {nullptr, nullptr, nullptr};
  if (d == 3) {
    V[0] = take(q0 * q1 * m2);
    V[1] = take(q0 * q1 * m2);
    V[2] = take(q0 * q1 * m2);
  }
  // outputs of the fused last direction: 3D W_DB, W_BD, W_BB (as V); 2D X_D, X_B (as U)
  double* T[3] = {nullptr, nullptr, nullptr};
  if (d == 3) {
    T[0] = take(q0 * q1 * m2);
    T[1] = take(q0 * q1 * m2);
    T[2] = take(q0 * q1 * m2);
  } else {
    T[0] = take(q0 * m1);
    T[1] = take(q0 * m1);
  }
  const int p1 = P->p + 1;
  auto sweep = [&](int mode, const double* in, const double* in2, double* out, double* out2, long long o0,
                   long long o1, long long o2, int in_len, int axis, const int* rp, const int* col, const double* v,
                   const double* v2) -> cudaError_t {
    const Shape2 sh = shape_for(o0, o1 * o2);
    const int a0 = (int)o0, a1 = (int)o1, a2 = (int)o2;
    if (mode == GS_ONE)
      gen_sweep<GS_ONE><<<sh.grid, sh.block, 0, st>>>(in, in2, out, out2, a0, a1, a2, in_len, axis, rp, col, v, v2,
                                                      done);
    else if (mode == GS_TWO_OUT)
      gen_sweep<GS_TWO_OUT><<<sh.grid, sh.block, 0, st>>>(in, in2, out, out2, a0, a1, a2, in_len, axis, rp, col, v,
                                                          v2, done);
    else
      gen_sweep<GS_TWO_IN><<<sh.grid, sh.block, 0, st>>>(in, in2, out, out2, a0, a1, a2, in_len, axis, rp, col, v,
                                                         v2, done);
    return cudaGetLastError();
  };
  const GenAxis &X = G[0], &Y = G[1];
  // forward: U_B = B_x u, U_D = D_x u
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_TWO_OUT, u, nullptr, U[0], U[1], q0, m1, m2, (int)m0, 0, X.rp, X.col,
                                           X.bv, X.dv));
  if (d == 2) {
    // X_D = B_y^T h_x, X_B = D_y^T h_y with h = w C (B_y U_D, D_y U_B), fused
    IFFD_LAUNCH(P, IFFD_K_GENERAL, st, launch_fused<2>(p1, U[1], U[0], nullptr, T[1], T[0], nullptr, (int)q0, 1,
                                                       (int)(q1 / p1), (int)m1, Y, C, ncomp, X.w, nullptr, done,
                                                       st));
    // Au = D_x^T X_D + B_x^T X_B
    IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_TWO_IN, T[1], T[0], Au, nullptr, m0, m1, 1, (int)q0, 0, X.trp,
                                             X.tcol, X.tdv, X.tbv));
    return IFFD_OK;
  }
  const GenAxis& Z = G[2];
  // V_BB = B_y U_B, V_BD = D_y U_B, V_DB = B_y U_D
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_TWO_OUT, U[0], nullptr, V[0], V[1], q0, q1, m2, (int)m1, 1, Y.rp,
                                           Y.col, Y.bv, Y.dv));
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_ONE, U[1], nullptr, V[2], nullptr, q0, q1, m2, (int)m1, 1, Y.rp,
                                           Y.col, Y.bv, nullptr));
  // W_DB = B_z^T h_x, W_BD = B_z^T h_y, W_BB = D_z^T h_z with
  // h = w C (B_z V_DB, B_z V_BD, D_z V_BB), fused along z
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, launch_fused<3>(p1, V[2], V[1], V[0], T[2], T[1], T[0], (int)q0, (int)q1,
                                                     (int)(q2 / p1), (int)m2, Z, C, ncomp, X.w, Y.w, done, st));
  // X_D = B_y^T W_DB -> U[1]; X_B = D_y^T W_BD + B_y^T W_BB -> U[0]
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_ONE, T[2], nullptr, U[1], nullptr, q0, m1, m2, (int)q1, 1, Y.trp,
                                           Y.tcol, Y.tbv, nullptr));
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_TWO_IN, T[1], T[0], U[0], nullptr, q0, m1, m2, (int)q1, 1, Y.trp,
                                           Y.tcol, Y.tdv, Y.tbv));
  // Au = D_x^T X_D + B_x^T X_B
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_TWO_IN, U[1], U[0], Au, nullptr, m0, m1, m2, (int)q0, 0, X.trp, X.tcol,
                                           X.tdv, X.tbv));
  return IFFD_OK;
}

cudaError_t launch_gen_pupdate(const double* z, double* p, const SolveState* S, int mode, long long N,
                               const int* done, cudaStream_t st) {
  gen_pupdate<<<vec_grid(N), kThreads, 0, st>>>(z, p, S, mode, N, done);
  return cudaGetLastError();
}

}  // namespace iffd
