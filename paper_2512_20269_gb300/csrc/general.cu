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
// V_DB = B_y U_D; g_x = B_z V_DB, g_y = B_z V_BD, g_z = D_z V_BB. Pointwise
// h = w C g. Backward with the transposes in the reverse order, the two
// contributions of each sweep summed in one pass.
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

template <int MODE>
__global__ void __launch_bounds__(kThreads)
gen_sweep(const double* __restrict__ in, const double* __restrict__ in2, double* __restrict__ out,
          double* __restrict__ out2, long long o0, long long o1, long long o2, int in_len, int axis,
          const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
          const double* __restrict__ val2, const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  const long long total = o0 * o1 * o2;
  const long long n0 = axis == 0 ? in_len : o0, n1 = axis == 1 ? in_len : o1;
  const long long s_ax = axis == 0 ? 1 : (axis == 1 ? n0 : n0 * n1);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long i0 = t % o0, r = t / o0;
    const long long i1 = r % o1, i2 = r / o1;
    const long long base = (axis == 0 ? 0 : i0) + (axis == 1 ? 0 : i1 * n0) + (axis == 2 ? 0 : i2 * n0 * n1);
    const int row = (int)(axis == 0 ? i0 : (axis == 1 ? i1 : i2));
    double s = 0.0, s2 = 0.0;
    const int k1 = __ldg(rp + row + 1);
    for (int k = __ldg(rp + row); k < k1; ++k) {
      const long long at = base + (long long)__ldg(col + k) * s_ax;
      const double v = in[at];
      s = fma(__ldg(val + k), v, s);
      if (MODE == GS_TWO_OUT) s2 = fma(__ldg(val2 + k), v, s2);
      if (MODE == GS_TWO_IN) s = fma(__ldg(val2 + k), in2[at], s);
    }
    out[t] = s;
    if (MODE == GS_TWO_OUT) out2[t] = s2;
  }
}

// h_k = w sum_l C_kl g_l at every Gauss point (in place); w = w_z (w_y w_x).
__global__ void __launch_bounds__(kThreads)
gen_pointwise(double* __restrict__ g0, double* __restrict__ g1, double* __restrict__ g2,
              const double* __restrict__ C, int ncomp, int d, long long q0, long long q1, long long q2,
              const double* __restrict__ w0, const double* __restrict__ w1, const double* __restrict__ w2,
              const int* __restrict__ done) {
  if (done != nullptr && *((volatile const int*)done)) return;
  const long long total = q0 * q1 * q2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long i0 = t % q0, r = t / q0;
    const long long i1 = r % q1, i2 = r / q1;
    double w = __ldg(w1 + i1) * __ldg(w0 + i0);
    if (d == 3) w = __ldg(w2 + i2) * w;
    const double a0 = g0[t], a1 = g1[t];
    if (d == 2) {
      double h0, h1;
      if (ncomp == 1) {
        const double c = __ldg(C + t);
        h0 = c * a0;
        h1 = c * a1;
      } else {
        const double c11 = __ldg(C + t), c12 = __ldg(C + total + t), c22 = __ldg(C + 2 * total + t);
        h0 = fma(c12, a1, c11 * a0);
        h1 = fma(c22, a1, c12 * a0);
      }
      g0[t] = w * h0;
      g1[t] = w * h1;
    } else {
      const double a2 = g2[t];
      double h0, h1, h2;
      if (ncomp == 1) {
        const double c = __ldg(C + t);
        h0 = c * a0;
        h1 = c * a1;
        h2 = c * a2;
      } else {
        const double c11 = __ldg(C + t), c12 = __ldg(C + total + t), c13 = __ldg(C + 2 * total + t);
        const double c22 = __ldg(C + 3 * total + t), c23 = __ldg(C + 4 * total + t);
        const double c33 = __ldg(C + 5 * total + t);
        h0 = fma(c13, a2, fma(c12, a1, c11 * a0));
        h1 = fma(c23, a2, fma(c22, a1, c12 * a0));
        h2 = fma(c33, a2, fma(c23, a1, c13 * a0));
      }
      g0[t] = w * h0;
      g1[t] = w * h1;
      g2[t] = w * h2;
    }
  }
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

int grid_for(long long total) {
  const long long g = (total + kThreads - 1) / kThreads;
  return (int)std::max(1LL, std::min(g, 152LL * 16));
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

// Scratch of one application: two arrays with direction 0 at the Gauss
// points, three with directions 0 and 1 (3D), d with all of them.
size_t general_ws_bytes(const Plan* P) {
  const long long q0 = P->gen[0].nq, q1 = P->gen[1].nq, m1 = P->gen[1].m;
  if (P->d == 2) return 2 * al256(q0 * m1 * 8) + 2 * al256(q0 * q1 * 8);
  const long long q2 = P->gen[2].nq, m2 = P->gen[2].m;
  return 2 * al256(q0 * m1 * m2 * 8) + 3 * al256(q0 * q1 * m2 * 8) + 3 * al256(q0 * q1 * q2 * 8);
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
  double* H[3] = {take(q0 * q1 * q2), take(q0 * q1 * q2), d == 3 ? take(q0 * q1 * q2) : nullptr};
  auto sweep = [&](int mode, const double* in, const double* in2, double* out, double* out2, long long o0,
                   long long o1, long long o2, int in_len, int axis, const int* rp, const int* col, const double* v,
                   const double* v2) -> cudaError_t {
    const int g = grid_for(o0 * o1 * o2);
    if (mode == GS_ONE)
      gen_sweep<GS_ONE><<<g, kThreads, 0, st>>>(in, in2, out, out2, o0, o1, o2, in_len, axis, rp, col, v, v2, done);
    else if (mode == GS_TWO_OUT)
      gen_sweep<GS_TWO_OUT><<<g, kThreads, 0, st>>>(in, in2, out, out2, o0, o1, o2, in_len, axis, rp, col, v, v2,
                                                     done);
    else
      gen_sweep<GS_TWO_IN><<<g, kThreads, 0, st>>>(in, in2, out, out2, o0, o1, o2, in_len, axis, rp, col, v, v2,
                                                    done);
    return cudaGetLastError();
  };
  const GenAxis &X = G[0], &Y = G[1];
  // forward: U_B = B_x u, U_D = D_x u
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_TWO_OUT, u, nullptr, U[0], U[1], q0, m1, m2, (int)m0, 0, X.rp, X.col,
                                           X.bv, X.dv));
  if (d == 2) {
    // g_x = B_y U_D, g_y = D_y U_B
    IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_ONE, U[1], nullptr, H[0], nullptr, q0, q1, 1, (int)m1, 1, Y.rp,
                                             Y.col, Y.bv, nullptr));
    IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_ONE, U[0], nullptr, H[1], nullptr, q0, q1, 1, (int)m1, 1, Y.rp,
                                             Y.col, Y.dv, nullptr));
    auto pointwise2 = [&] {
      gen_pointwise<<<grid_for(q0 * q1), kThreads, 0, st>>>(H[0], H[1], nullptr, C, ncomp, 2, q0, q1, 1, X.w, Y.w,
                                                            nullptr, done);
      return cudaGetLastError();
    };
    IFFD_LAUNCH(P, IFFD_K_GENERAL, st, pointwise2());
    // X_D = B_y^T h_x, X_B = D_y^T h_y; Au = D_x^T X_D + B_x^T X_B
    IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_ONE, H[0], nullptr, U[1], nullptr, q0, m1, 1, (int)q1, 1, Y.trp,
                                             Y.tcol, Y.tbv, nullptr));
    IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_ONE, H[1], nullptr, U[0], nullptr, q0, m1, 1, (int)q1, 1, Y.trp,
                                             Y.tcol, Y.tdv, nullptr));
    IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_TWO_IN, U[1], U[0], Au, nullptr, m0, m1, 1, (int)q0, 0, X.trp,
                                             X.tcol, X.tdv, X.tbv));
    return IFFD_OK;
  }
  const GenAxis& Z = G[2];
  // V_BB = B_y U_B, V_BD = D_y U_B, V_DB = B_y U_D
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_TWO_OUT, U[0], nullptr, V[0], V[1], q0, q1, m2, (int)m1, 1, Y.rp,
                                           Y.col, Y.bv, Y.dv));
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_ONE, U[1], nullptr, V[2], nullptr, q0, q1, m2, (int)m1, 1, Y.rp,
                                           Y.col, Y.bv, nullptr));
  // g_x = B_z V_DB, g_y = B_z V_BD, g_z = D_z V_BB
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_ONE, V[2], nullptr, H[0], nullptr, q0, q1, q2, (int)m2, 2, Z.rp, Z.col,
                                           Z.bv, nullptr));
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_ONE, V[1], nullptr, H[1], nullptr, q0, q1, q2, (int)m2, 2, Z.rp, Z.col,
                                           Z.bv, nullptr));
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_ONE, V[0], nullptr, H[2], nullptr, q0, q1, q2, (int)m2, 2, Z.rp, Z.col,
                                           Z.dv, nullptr));
  auto pointwise3 = [&] {
    gen_pointwise<<<grid_for(q0 * q1 * q2), kThreads, 0, st>>>(H[0], H[1], H[2], C, ncomp, 3, q0, q1, q2, X.w, Y.w,
                                                               Z.w, done);
    return cudaGetLastError();
  };
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, pointwise3());
  // W_DB = B_z^T h_x -> V[2], W_BD = B_z^T h_y -> V[1], W_BB = D_z^T h_z -> V[0]
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_ONE, H[0], nullptr, V[2], nullptr, q0, q1, m2, (int)q2, 2, Z.trp,
                                           Z.tcol, Z.tbv, nullptr));
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_ONE, H[1], nullptr, V[1], nullptr, q0, q1, m2, (int)q2, 2, Z.trp,
                                           Z.tcol, Z.tbv, nullptr));
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_ONE, H[2], nullptr, V[0], nullptr, q0, q1, m2, (int)q2, 2, Z.trp,
                                           Z.tcol, Z.tdv, nullptr));
  // X_D = B_y^T W_DB -> U[1]; X_B = D_y^T W_BD + B_y^T W_BB -> U[0]
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_ONE, V[2], nullptr, U[1], nullptr, q0, m1, m2, (int)q1, 1, Y.trp,
                                           Y.tcol, Y.tbv, nullptr));
  IFFD_LAUNCH(P, IFFD_K_GENERAL, st, sweep(GS_TWO_IN, V[1], V[0], U[0], nullptr, q0, m1, m2, (int)q1, 1, Y.trp,
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
