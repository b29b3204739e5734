// Autotuner of the pass geometry (iffd_autotune): pencils per tile of every
// transform pass and stiffness sweep, and the radix sequence of every
// direction's FFT.
//
// Each candidate runs the real kernel of the plan on the caller's workspace
// (one warm-up launch, then the best of three CUDA-event timings). Choices are
// cached per size class in a process-wide table, so every plan of the same
// class (a stand-alone plan, or the engine's plan of the same (d, n, p)) gets
// the same geometry, and with it bitwise the same results.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <vector>

#include "../../include/iffd.h"
#include "device_common.cuh"
#include "kernels.h"
#include "plan.h"

namespace iffd {

template <typename Tc>
PassLaunch<Tc> make_pass(const Plan* P, int axis, const AxisTab<Tc>* tabs, const int* PPs, const int* ldts,
                         const int* done);
StiffLaunch make_stiff(const Plan* P, int axis);

namespace {

// Size class of one tuned pass.
struct Key {
  int kind;  // 0: transform pass, 1: stiffness sweep, 2: variable-coefficient sweep
  int prec;  // transform arithmetic (iffd_precision); 0 for sweeps
  int d, axis, m, len, p, qlog;
  bool operator<(const Key& o) const {
    return std::tie(kind, prec, d, axis, m, len, p, qlog) <
           std::tie(o.kind, o.prec, o.d, o.axis, o.m, o.len, o.p, o.qlog);
  }
};
struct Choice {
  int pp;
  std::vector<int> radix;  // transform passes only
  int pipe = 0;            // transform passes only: pipelined persistent kernel
  int warp = 0;            // FP32 transform passes only: warp-FFT pass
};

std::mutex g_mu;
std::map<Key, Choice> g_cache;

constexpr int kCandPP[] = {2, 4, 8, 16, 32};
constexpr size_t kMaxTuneSmem = 200 * 1024;
// A pass is tuned only if one launch of it has at least this many CTAs (four
// waves of 152 SMs) with its default tile: a smaller launch cannot fill the GPU
// alone, so its stand-alone timing says little about its cost next to others.
constexpr long long kMinTuneTiles = 4 * 152;

int ilog2ll(long long x) {
  int r = 0;
  while (x > 1) {
    x >>= 1;
    ++r;
  }
  return r;
}

struct Timer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~Timer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

// Best of three timed launches after one warm-up launch (milliseconds).
template <typename F>
int time_best(F&& launch, cudaStream_t st, Timer& t, float* best) {
  IFFD_CUDA(launch());
  *best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    IFFD_CUDA(cudaEventRecord(t.e0, st));
    IFFD_CUDA(launch());
    IFFD_CUDA(cudaEventRecord(t.e1, st));
    IFFD_CUDA(cudaEventSynchronize(t.e1));
    float ms = 0.f;
    IFFD_CUDA(cudaEventElapsedTime(&ms, t.e0, t.e1));
    *best = std::min(*best, ms);
  }
  return IFFD_OK;
}

std::vector<int> var_radices(const FftVar& v) { return std::vector<int>(v.radix, v.radix + v.nst); }

// Transform pass along direction a for arithmetic Tc: FUSED on the last
// direction, FWD on the others (BWD shares the tile and radix sequence).
template <typename Tc>
int tune_transform(Plan* P, int a, char* ws, cudaStream_t st, Timer& tm) {
  constexpr bool f64 = std::is_same<Tc, double>::value;
  AxisTab<Tc>* tabs;
  if constexpr (f64) tabs = P->axd;
  else tabs = P->axf;
  int* PPs = f64 ? P->PPd : P->PPf;
  int* ldts = f64 ? P->ldtd : P->ldtf;
  int* vsel = f64 ? P->vsel_d : P->vsel_f;
  int* pipes = f64 ? P->pipe_d : P->pipe_f;
  // the timed pass reads Tc except FP32's first direction (FP64 input)
  const bool pipe_ok = f64 || a > 0;
  AxisTab<Tc>& ax = tabs[a];
  const int mode = (a == P->d - 1) ? PM_FUSED : PM_FWD;
  const Key key{0, f64 ? IFFD_PREC_FP64 : IFFD_PREC_FP32_TRANSFORM, P->d, a, ax.m, ax.F, P->p,
                ilog2ll(P->dims.N / ax.m)};
  std::vector<int> vars;
  for (size_t i = 0; i < P->fvar[a].size(); ++i)
    if (P->fvar[a][i].len == ax.F) vars.push_back((int)i);
  // warp: 0 block kernel, 1 warp-FFT pass, 2 paired warp-FFT pass (FP32)
  auto apply = [&](int vi, int pp, int pipe, int warp) {
    vsel[a] = vi;
    set_fft(&ax, P->fvar[a][vi]);
    PPs[a] = pp;
    pipes[a] = pipe;
    (f64 ? P->warp_d : P->warp_f)[a] = warp > 0 ? 1 : 0;
    if (!f64) P->pair_f[a] = warp == 2 ? 1 : 0;
  };
  if (precond_tiles(P->dims, a, PPs[a]) < kMinTuneTiles) return IFFD_OK;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      for (int vi : vars)
        if (var_radices(P->fvar[a][vi]) == it->second.radix) {
          apply(vi, it->second.pp, it->second.pipe, it->second.warp);
          return IFFD_OK;
        }
    }
  }
  double* r = reinterpret_cast<double*>(ws + P->off_r);
  double* z = reinterpret_cast<double*>(ws + P->off_z);
  float* tf = reinterpret_cast<float*>(ws + P->off_tf);
  float best = 1e30f;
  int best_v = vsel[a], best_pp = PPs[a], best_pipe = pipes[a], best_warp = 0;
  auto time_pass = [&](float* ms) -> int {
    const PassLaunch<Tc> L = make_pass<Tc>(P, a, tabs, PPs, ldts, nullptr);
    if constexpr (f64) {
      return time_best([&] { return launch_pass<double, double, double>(L, mode, 0, a == 0 ? r : z, z, st); }, st,
                       tm, ms);
    } else {
      if (a == 0)
        return time_best([&] { return launch_pass<float, double, float>(L, mode, 0, r, tf, st); }, st, tm, ms);
      return time_best([&] { return launch_pass<float, float, float>(L, mode, 0, tf, tf, st); }, st, tm, ms);
    }
  };
  if constexpr (!f64) {
    if (const int wN = wpass_len(ax)) {  // the warp-FFT pass (its tile is fixed), unpaired and paired
      for (int w = 1; w <= (wN <= 256 ? 2 : 1); ++w) {
        apply(vsel[a], PPs[a], 0, w);
        float ms = 0.f;
        if (int rc = time_pass(&ms)) return rc;
        if (ms < best) {
          best = ms;
          best_warp = w;
          best_pipe = 0;
        }
      }
    }
  }
  for (int vi : vars)
    for (int pp : kCandPP)
      for (int pipe = 0; pipe <= (pipe_ok ? 1 : 0); ++pipe) {
      const size_t need = pipe ? precond_smem_bytes_pipe(pp, ldts[a], ax.F, sizeof(Tc))
                               : precond_smem_bytes(pp, ldts[a], ax.F, sizeof(Tc));
      if (need > kMaxTuneSmem) continue;
      apply(vi, pp, pipe, 0);
      float ms = 0.f;
      if (int rc = time_pass(&ms)) return rc;
      if (ms < best) {
        best = ms;
        best_v = vi;
        best_pp = pp;
        best_pipe = pipe;
        best_warp = 0;
      }
    }
  apply(best_v, best_pp, best_pipe, best_warp);
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[key] = Choice{best_pp, var_radices(P->fvar[a][best_v]), best_pipe, best_warp};
  return IFFD_OK;
}

// Stiffness sweep along direction a: FIRST on the last direction, MID on the
// middle one (3D), LAST on direction 0.
int tune_stiffness(Plan* P, int a, char* ws, cudaStream_t st, Timer& tm) {
  const bool var = P->opt.coef == IFFD_COEF_SEPARABLE_SIN;
  int* PPx = var ? P->PPv : P->PPs;
  const int arrays = var ? 4 : 2;
  const Key key{var ? 2 : 1, 0, P->d, a, P->dims.m[a], 0, P->p, ilog2ll(P->dims.N / P->dims.m[a])};
  if (stiff_tiles(P->dims, a, PPx[a]) < kMinTuneTiles) return IFFD_OK;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      PPx[a] = it->second.pp;
      return IFFD_OK;
    }
  }
  double* r = reinterpret_cast<double*>(ws + P->off_r);
  double* q = reinterpret_cast<double*>(ws + P->off_q);
  double* T1 = reinterpret_cast<double*>(ws + P->off_t1);
  double* T2 = reinterpret_cast<double*>(ws + P->off_t2);
  double* T3 = reinterpret_cast<double*>(ws + P->off_t3);
  double* T4 = reinterpret_cast<double*>(ws + P->off_t4);
  const int stage = (a == P->d - 1) ? SS_FIRST : (a == 0 ? SS_LAST : SS_MID);
  float best = 1e30f;
  int best_pp = PPx[a];
  for (int pp : kCandPP) {
    if ((size_t)arrays * pp * P->ldts[a] * sizeof(double) > kMaxTuneSmem) continue;
    StiffLaunch S = make_stiff(P, a);
    S.PP = pp;
    auto launch = [&]() -> cudaError_t {
      if (!var) {
        if (stage == SS_FIRST) return launch_stiff_first(S, r, nullptr, nullptr, nullptr, 0, T1, T2, nullptr, st);
        if (stage == SS_MID) return launch_stiff_mid(S, T1, T2, nullptr, st);
        return launch_stiff_last(S, T1, T2, q, nullptr, nullptr, nullptr, st);
      }
      const WBandTab& wb = P->wb[a];
      if (stage == SS_FIRST)
        return launch_vstiff_first(S, wb, r, nullptr, nullptr, nullptr, 0, T1, T2, T3, T4, nullptr, st);
      if (stage == SS_MID) return launch_vstiff_mid(S, wb, T1, T2, T3, T4, nullptr, st);
      return launch_vstiff_last(S, wb, T1, T2, T3, T4, q, nullptr, nullptr, nullptr, st);
    };
    float ms = 0.f;
    const int rc = time_best(launch, st, tm, &ms);
    if (rc) return rc;
    if (ms < best) {
      best = ms;
      best_pp = pp;
    }
  }
  PPx[a] = best_pp;
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[key] = Choice{best_pp, {}};
  return IFFD_OK;
}

}  // namespace

int plan_autotune(Plan* P, void* ws, cudaStream_t st) {
  plan_drop_graphs(P);
  char* w = static_cast<char*>(ws);
  Timer tm;
  IFFD_CUDA(cudaEventCreate(&tm.e0));
  IFFD_CUDA(cudaEventCreate(&tm.e1));
  // defined inputs for the timing runs (the values do not matter)
  const size_t vec = (size_t)P->dims.N * sizeof(double);
  IFFD_CUDA(cudaMemsetAsync(w + P->off_r, 0, vec, st));
  IFFD_CUDA(cudaMemsetAsync(w + P->off_z, 0, vec, st));
  IFFD_CUDA(cudaMemsetAsync(w + P->off_t1, 0, vec, st));
  IFFD_CUDA(cudaMemsetAsync(w + P->off_t2, 0, vec, st));
  if (P->opt.coef == IFFD_COEF_SEPARABLE_SIN) {
    IFFD_CUDA(cudaMemsetAsync(w + P->off_t3, 0, vec, st));
    IFFD_CUDA(cudaMemsetAsync(w + P->off_t4, 0, vec, st));
  }
  if (P->opt.precision == IFFD_PREC_FP32_TRANSFORM)
    IFFD_CUDA(cudaMemsetAsync(w + P->off_tf, 0, (size_t)P->dims.N * sizeof(float), st));
  int rc;
  for (int a = 0; a < P->d; ++a) {
    // the double-float passes of an FP64 plan have a fixed geometry
    if (P->opt.precond == IFFD_PRECOND_IFFD && !(P->opt.precision == IFFD_PREC_FP64 && P->dfq)) {
      rc = (P->opt.precision == IFFD_PREC_FP64) ? tune_transform<double>(P, a, w, st, tm)
                                                : tune_transform<float>(P, a, w, st, tm);
      if (rc) return rc;
    }
    if ((rc = tune_stiffness(P, a, w, st, tm))) return rc;
  }
  IFFD_CUDA(cudaStreamSynchronize(st));
  P->tuned = true;
  return IFFD_OK;
}

}  // namespace iffd

using namespace iffd;

extern "C" {

int iffd_autotune(iffd_handle h, void* ws, void* stream) {
  g_err.clear();
  if (!h || !ws) return fail(!h ? IFFD_ERR_INVALID_ARG : IFFD_ERR_WORKSPACE, "NULL argument");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(IFFD_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->P.device) return fail(IFFD_ERR_INVALID_ARG, "plan was created on another device");
  return plan_autotune(&h->P, ws, static_cast<cudaStream_t>(stream));
}

int iffd_set_geometry(iffd_handle h, int axis, int pencils_transform, int pencils_stiffness, int pipelined) {
  g_err.clear();
  if (!h || axis < 0 || axis >= h->P.d) return fail(IFFD_ERR_INVALID_ARG, "bad handle or axis");
  Plan& P = h->P;
  plan_drop_graphs(&P);
  const bool f64 = P.opt.precision == IFFD_PREC_FP64;
  auto pow2 = [](int v) { return v >= kMinTunePP && v <= 32 && (v & (v - 1)) == 0; };
  if (pipelined == 3) {
    // double-float transforms for the whole plan (FP64 IFFD plans; every
    // direction by the warp-FFT pass or the block kernel without Bluestein)
    if (!f64 || !dfq_eligible(P))
      return fail(IFFD_ERR_UNSUPPORTED, "double-float transforms need an FP64 IFFD plan whose every direction runs "
                                        "its transform without Bluestein's convolution");
    if (pencils_transform > 0) return fail(IFFD_ERR_INVALID_ARG, "the double-float pass has a fixed tile");
    P.dfq = 1;
    pipelined = -1;
  } else if (f64 && (pencils_transform > 0 || (pipelined >= 0 && pipelined <= 2))) {
    P.dfq = 0;  // an FP64-pipe transform geometry set by hand
  }
  if (pipelined == 2 || pipelined == 4) {
    if (f64 ? wpass_len(P.axd[axis]) == 0 : wpass_len(P.axf[axis]) == 0)
      return fail(IFFD_ERR_UNSUPPORTED, "the warp-FFT pass needs a D = {0,1} direction of FFT length 64, 128, 256 "
                                        "or 512 (FP64: up to 256)");
    if (pipelined == 4 && (f64 || wpass_len(P.axf[axis]) > 256))
      return fail(IFFD_ERR_UNSUPPORTED, "the paired warp-FFT pass needs FP32 transforms and an FFT length of 64, "
                                        "128 or 256");
    if (pencils_transform > 0) return fail(IFFD_ERR_INVALID_ARG, "the warp-FFT pass has a fixed tile");
    (f64 ? P.warp_d : P.warp_f)[axis] = 1;
    (f64 ? P.pipe_d : P.pipe_f)[axis] = 0;
    if (!f64) P.pair_f[axis] = pipelined == 4 ? 1 : 0;
    pipelined = -1;
  } else if (pipelined > 2) {
    return fail(IFFD_ERR_INVALID_ARG, "pipelined must be 0, 1, 2, 3 or 4 (or < 0)");
  } else if (pencils_transform > 0 || pipelined >= 0) {
    (f64 ? P.warp_d : P.warp_f)[axis] = 0;  // a block-kernel geometry set by hand
  }
  if (pencils_transform > 0) {
    if (!pow2(pencils_transform)) return fail(IFFD_ERR_INVALID_ARG, "pencils per tile must be 2, 4, 8, 16 or 32");
    const int ldt = f64 ? P.ldtd[axis] : P.ldtf[axis];
    const int F = f64 ? P.axd[axis].F : P.axf[axis].F;
    const size_t elt = f64 ? sizeof(double) : sizeof(float);
    const int pipe = pipelined > 0 ? 1 : (pipelined == 0 ? 0 : (f64 ? P.pipe_d[axis] : P.pipe_f[axis]));
    const size_t need = pipe ? precond_smem_bytes_pipe(pencils_transform, ldt, F, elt)
                             : precond_smem_bytes(pencils_transform, ldt, F, elt);
    if (need > kMaxTuneSmem) return fail(IFFD_ERR_UNSUPPORTED, "tile does not fit in shared memory");
    (f64 ? P.PPd : P.PPf)[axis] = pencils_transform;
  }
  if (pipelined >= 0) {
    const int PP = f64 ? P.PPd[axis] : P.PPf[axis];
    const int ldt = f64 ? P.ldtd[axis] : P.ldtf[axis];
    const int F = f64 ? P.axd[axis].F : P.axf[axis].F;
    const size_t elt = f64 ? sizeof(double) : sizeof(float);
    if (pipelined && precond_smem_bytes_pipe(PP, ldt, F, elt) > kMaxTuneSmem)
      return fail(IFFD_ERR_UNSUPPORTED, "pipelined tile does not fit in shared memory");
    (f64 ? P.pipe_d : P.pipe_f)[axis] = pipelined ? 1 : 0;
  }
  if (pencils_stiffness > 0) {
    if (!pow2(pencils_stiffness)) return fail(IFFD_ERR_INVALID_ARG, "pencils per tile must be 2, 4, 8, 16 or 32");
    const bool var = P.opt.coef == IFFD_COEF_SEPARABLE_SIN;
    if ((size_t)(var ? 4 : 2) * pencils_stiffness * P.ldts[axis] * sizeof(double) > kMaxTuneSmem)
      return fail(IFFD_ERR_UNSUPPORTED, "stiffness tile does not fit in shared memory");
    (var ? P.PPv : P.PPs)[axis] = pencils_stiffness;
  }
  return IFFD_OK;
}

int iffd_get_tiles(iffd_handle h, int axis, int* pencils_transform, int* pencils_stiffness, int* radices,
                   int* nstages, int* pipelined) {
  if (!h || axis < 0 || axis >= h->P.d) return fail(IFFD_ERR_INVALID_ARG, "bad handle or axis");
  const Plan& P = h->P;
  const bool f64 = P.opt.precision == IFFD_PREC_FP64;
  if (f64 && P.dfq && wpass_len(P.axq[axis]) == 0) {  // double-float block pass: the FP64 tile and radices
    if (pencils_transform) *pencils_transform = P.PPd[axis];
    if (pencils_stiffness)
      *pencils_stiffness = (P.opt.coef == IFFD_COEF_SEPARABLE_SIN) ? P.PPv[axis] : P.PPs[axis];
    if (nstages) *nstages = P.axq[axis].nst;
    if (radices)
      for (int s = 0; s < P.axq[axis].nst; ++s) radices[s] = P.axq[axis].radix[s];
    if (pipelined) *pipelined = 5;
    return IFFD_OK;
  }
  if (f64 && P.dfq) {  // double-float warp pass: fixed tile and radices 8, 8, then 4 or 2
    const int N = wpass_len(P.axq[axis]);
    if (pencils_transform) *pencils_transform = wpass_pencils(N);
    if (pencils_stiffness)
      *pencils_stiffness = (P.opt.coef == IFFD_COEF_SEPARABLE_SIN) ? P.PPv[axis] : P.PPs[axis];
    const int rad[3] = {8, 8, N == 256 ? 4 : 2};
    const int ns = N == 64 ? 2 : 3;
    if (nstages) *nstages = ns;
    if (radices)
      for (int s = 0; s < ns; ++s) radices[s] = rad[s];
    if (pipelined) *pipelined = 3;
    return IFFD_OK;
  }
  const int wd = f64 ? f64_warp_len(P, axis) : 0;
  if (pencils_transform) *pencils_transform = f64 ? (wd ? wpass_pencils(wd) : P.PPd[axis]) : f32_geom(P, axis).PP;
  if (pencils_stiffness)
    *pencils_stiffness = (P.opt.coef == IFFD_COEF_SEPARABLE_SIN) ? P.PPv[axis] : P.PPs[axis];
  const int nst = f64 ? P.axd[axis].nst : P.axf[axis].nst;
  if (nstages) *nstages = nst;
  if (pipelined) {
    const F32Geom g = f32_geom(P, axis);
    *pipelined = f64 ? (wd ? 2 : P.pipe_d[axis]) : (g.wN ? (g.pair ? 4 : 2) : P.pipe_f[axis]);
  }
  if (radices)
    for (int s = 0; s < nst; ++s) radices[s] = f64 ? P.axd[axis].radix[s] : P.axf[axis].radix[s];
  return IFFD_OK;
}

}  // extern "C"
