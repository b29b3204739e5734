// Internal plan structure shared by the C ABI (capi.cu) and the batched /
// serving engine (engine.cu). Not part of the public interface.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/iffd.h"
#include "device_common.cuh"
#include "host_setup.h"
#include "kernels.h"

namespace iffd {

extern thread_local std::string g_err;
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* where);

#define IFFD_CUDA(call)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return ::iffd::cuda_fail(e_, #call); \
  } while (0)

// Launch `call` as one kernel of kind `kind`, with optional event timing.
#define IFFD_LAUNCH(P, kind, st, call)  \
  do {                                  \
    (P)->prof.begin((kind), (st));      \
    IFFD_CUDA(call);                    \
    (P)->prof.end(st);                  \
  } while (0)

// CUDA-event timing of every launch (optional) and a launch counter.
struct Profiler {
  bool on = false;
  long long launches = 0;
  struct Pending {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> pool;
  std::vector<Pending> pending;
  long long cnt[IFFD_K_KINDS] = {};
  double ms[IFFD_K_KINDS] = {};
  cudaEvent_t take() {
    cudaEvent_t e = nullptr;
    if (!pool.empty()) {
      e = pool.back();
      pool.pop_back();
    } else {
      cudaEventCreate(&e);
    }
    return e;
  }
  void begin(int kind, cudaStream_t st) {
    ++launches;
    if (!on) return;
    Pending p{kind, take(), nullptr};
    cudaEventRecord(p.a, st);
    pending.push_back(p);
  }
  void end(cudaStream_t st) {
    if (!on || pending.empty() || pending.back().b != nullptr) return;
    pending.back().b = take();
    cudaEventRecord(pending.back().b, st);
  }
  cudaError_t collect() {
    for (auto& p : pending) {
      if (p.b == nullptr) continue;
      cudaError_t e = cudaEventSynchronize(p.b);
      if (e != cudaSuccess) return e;
      float t = 0.f;
      e = cudaEventElapsedTime(&t, p.a, p.b);
      if (e != cudaSuccess) return e;
      cnt[p.kind] += 1;
      ms[p.kind] += t;
    }
    for (auto& p : pending) {
      pool.push_back(p.a);
      if (p.b) pool.push_back(p.b);
    }
    pending.clear();
    return cudaSuccess;
  }
  void release() {
    for (auto& p : pending) {
      cudaEventDestroy(p.a);
      if (p.b) cudaEventDestroy(p.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
    pending.clear();
    pool.clear();
  }
};

// Smallest pencils-per-tile the tuner tries (sizes the partial-sum buffer).
constexpr int kMinTunePP = 2;

// One radix sequence of the FFT of one direction, with its device twiddles.
struct FftVar {
  int len, nst;
  int radix[kMaxStages], twoff[kMaxStages];
  const double* twd;
  const float* twf;
  const df* twq;  // double-float copy (the double-float block passes)
};

// Plan of one problem: host 1D data, device tables, launch geometry.
// One direction of the general-coefficient stiffness: its Gauss-point
// tables (QuadAxis) on the device.
struct GenAxis {
  int nq = 0, m = 0;
  const int *rp = nullptr, *col = nullptr, *trp = nullptr, *tcol = nullptr;
  const double *bv = nullptr, *dv = nullptr, *tbv = nullptr, *tdv = nullptr, *w = nullptr;
};

struct Plan {
  mutable Profiler prof;
  int d = 0, p = 0;
  int n[3] = {0, 0, 0};
  int device = 0;
  iffd_options opt{};
  Dims dims{};
  Axis1D host[3];
  void* dev = nullptr;  // single allocation for all device tables
  double* rden = nullptr;  // FP64 IFFD plans: N reciprocals of the summed eigenvalues
  AxisTab<double> axd[3];
  AxisTab<float> axf[3];
  BandTab bt[3];
  WBandTab wb[3];  // variable-coefficient bands (IFFD_COEF_SEPARABLE_SIN)
  int PPd[3], ldtd[3], PPf[3], ldtf[3], PPs[3], ldts[3], PPv[3];
  // FFT radix sequences of each direction (lengths L, and F for Bluestein) and
  // the one selected per precision (index into fvar[a])
  std::vector<FftVar> fvar[3];
  int vsel_d[3] = {0, 0, 0}, vsel_f[3] = {0, 0, 0};
  // 1: the direction's transform passes run as the persistent pipelined kernel
  // (where input and arithmetic types agree); chosen by the tuner
  int pipe_d[3] = {0, 0, 0}, pipe_f[3] = {0, 0, 0};
  // FP32 transforms: 1 where the direction runs the warp-FFT pass (only if
  // wpass_len(axf[a]) > 0; on by default, off once a tile size is set by
  // hand or the tuner finds the block kernel faster), and its twiddle table
  int warp_f[3] = {0, 0, 0};
  // 1 where that warp-FFT pass runs paired (two sequences per lane group, FFT
  // length <= 256; the default for the last direction, whose pass is fused)
  int pair_f[3] = {0, 0, 0};
  const float2* wtab[3] = {nullptr, nullptr, nullptr};
  // FP64 transforms: the same for the FP64 warp-FFT pass (wpass_len(axd[a]) > 0;
  // off by default, chosen by hand or by the tuner) and its FP64 twiddles
  int warp_d[3] = {0, 0, 0};
  const double2* wtab_d[3] = {nullptr, nullptr, nullptr};
  // FP64 IFFD plans whose directions all have a warp-FFT pass of length 64,
  // 128 or 256 (D = {0,1}): dfq = 1 runs every transform pass in double-float
  // arithmetic on the FP32 pipe (the default for such plans; a transform
  // geometry set by hand turns it off), with these tables and twiddles
  int dfq = 0;
  AxisTab<df> axq[3];
  const df2* wtab_q[3] = {nullptr, nullptr, nullptr};
  // General-coefficient stiffness: per direction the Gauss-point tables (one
  // device allocation, gen_mem)
  GenAxis gen[3];
  char* gen_mem = nullptr;
  bool tuned = false;
  // exact FD tables
  const double* QT[3] = {nullptr, nullptr, nullptr};
  const double* Q[3] = {nullptr, nullptr, nullptr};
  const double* lamQ[3] = {nullptr, nullptr, nullptr};
  // workspace layout (bytes)
  size_t off_r, off_z, off_p, off_q, off_t1, off_t2, off_t3, off_t4, off_tf, off_part, off_state, ws_bytes;
  int max_parts = 0;
  SolveState* host_state = nullptr;  // pinned
  // Captured CUDA graphs of the PCG solve's chunks (iffd_pcg_solve): the
  // start and first iterations, and a chunk of later iterations, for one
  // (f, u, workspace) each; two such sets (double-buffered callers), dropped
  // when the launch geometry changes.
  struct SolveGraph {
    const double* f = nullptr;
    double* u = nullptr;
    void* ws = nullptr;
    cudaGraphExec_t first = nullptr, next = nullptr;
    int nfirst = 0;                   // iterations in `first`
    long long kfirst = 0, knext = 0;  // kernels per replay
    unsigned long long used = 0;      // last use (replacement order)
    long long replays = 0;            // launches after the capture
  };
  struct SolveGraphs {
    cudaStream_t cap = nullptr;  // private capture stream
    SolveGraph g[2];
    bool failed = false;  // capture not possible here: launch directly
    // the (f, u, workspace) of the last two solves: graphs are captured when
    // a solve repeats one, so one-off solves pay no capture
    const double* seen_f[2] = {nullptr, nullptr};
    double* seen_u[2] = {nullptr, nullptr};
    void* seen_ws[2] = {nullptr, nullptr};
    unsigned long long tick = 0;
  };
  mutable SolveGraphs graphs;
  // iterations of the last converged solve: the length of the first chunk
  // of iterations enqueued before the solve state is read (0: none yet)
  mutable int last_iters = 0;
};


}  // namespace iffd

struct iffd_plan {
  iffd::Plan P;
};

namespace iffd {

// Builds a plan (host 1D setup + device tables) on the current device.
// nrep[k] repeated knots for direction k, listed as (knot, extra) pairs in
// reps, direction by direction; both may be NULL (no repeated knots).
int plan_create(int d, const int* n_elems, int p, const int* dirichlet, const iffd_options* opt, cudaStream_t stream,
                iffd_plan** out, const int* nrep = nullptr, const int* reps = nullptr);
void plan_release(iffd_plan* h);
// Drops the captured solve graphs (after a change of launch geometry).
void plan_drop_graphs(Plan* P);
// Launch geometry of the FP32 transform passes of direction a: pencils per
// tile, tile row length, warp-FFT length (0: block kernel) and its twiddles,
// shared memory of one (non-pipelined) CTA.
struct F32Geom {
  int PP, ldt, wN;
  const float2* wt;
  size_t smem;
  int pair;  // the paired warp-FFT pass
};
// Partial sums of the last FP32 backward pass (two per tile when paired).
int f32_last_parts(const Plan& P);
F32Geom f32_geom(const Plan& P, int a);
// General-coefficient stiffness (general.cu): device tables (at plan
// creation), scratch bytes of one application, the application Au = A_C u
// (C: ncomp arrays at the Gauss points), and the p-update of its PCG.
constexpr int kGenMaxDegree = 11;  // the fused last-direction pass holds p + 1 entries per thread
int build_general_tables(Plan* P, cudaStream_t st);
size_t general_ws_bytes(const Plan* P);
int run_general(Plan* P, const double* C, int ncomp, const double* u, double* Au, void* gws, cudaStream_t st,
                const int* done);
cudaError_t launch_gen_pupdate(const double* z, double* p, const SolveState* S, int mode, long long N,
                               const int* done, cudaStream_t st);
// FFT length of direction a's FP64 warp-FFT pass (0: the block kernel runs).
int f64_warp_len(const Plan& P, int a);
// 1 if every direction of an FP64 IFFD plan can run the double-float warp pass.
int dfq_eligible(const Plan& P);
StiffLaunch plan_stiff_launch(const Plan* P, int axis);
template <typename T>
void set_fft(AxisTab<T>* t, const FftVar& v);
// Tunes the tiles and radix sequences of a plan on workspace ws (iffd_autotune).
int plan_autotune(Plan* P, void* ws, cudaStream_t st);

}  // namespace iffd
