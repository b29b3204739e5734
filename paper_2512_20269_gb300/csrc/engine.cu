// Batched solves with continuous batching (iffd_engine_*).
//
// Many independent IFFD-PCG solves advance together. The active systems are
// split into lanes by degree and by the shared memory of their transform
// passes; within a lane each phase of a PCG iteration (stiffness sweeps,
// reductions, vector update, transform passes) is one batched launch covering
// the tiles of every system of the lane, and the lanes run concurrently on
// separate streams. A system's kernels, tile decomposition and reduction order
// are exactly those of the single-system path, so its result does not depend
// on which other systems share the launches.
//
// Requests are admitted while their workspace fits the engine's device arena
// (the budget); an admitted request is initialised at the next step and then
// iterates with the others; finished systems are retired after each step and
// their workspace returns to the arena, so later requests can join while
// earlier ones are still iterating. The per-iteration launch sequence of all
// lanes (forked from and joined to the engine stream) is captured into one CUDA
// graph and replayed while the set of systems is unchanged.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/iffd.h"
#include "device_common.cuh"
#include "kernels.h"
#include "plan.h"

namespace iffd {

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr size_t kLaneStreams = 8;  // streams the lanes of one iteration graph run on

// First-fit sub-allocator over one device allocation.
struct Arena {
  char* base = nullptr;
  size_t bytes = 0;
  std::map<size_t, size_t> free_;  // offset -> size
  void init(char* b, size_t n) {
    base = b;
    bytes = n;
    free_.clear();
    free_[0] = n;
  }
  bool alloc(size_t n, size_t* off) {
    n = al256(n);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n;
        const size_t noff = it->first + n;
        free_.erase(it);
        if (rest) free_[noff] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = al256(n);
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t available() const {
    size_t s = 0;
    for (auto& kv : free_) s += kv.second;
    return s;
  }
};

struct Sys {
  long long id;
  iffd_plan* plan;
  const double* f;
  double* u;
  size_t off, bytes;
  char* ws;
  int phase;  // 0: admitted, not initialised; 1: iterating
  int slot;   // index among the active systems (persistent launch counters)
};

// Growable device buffer.
struct DevBuf {
  char* p = nullptr;
  size_t cap = 0;
  cudaError_t reserve(size_t n) {
    if (n <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, n);
    if (e == cudaSuccess) cap = n;
    return e;
  }
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

// Host staging of all descriptors of one launch sequence; uploaded in one copy.
struct Staging {
  std::vector<char> bytes;
  template <typename T>
  size_t put(const std::vector<T>& v) {
    const size_t off = al256(bytes.size());
    bytes.resize(off + std::max<size_t>(1, v.size()) * sizeof(T));
    if (!v.empty()) std::memcpy(bytes.data() + off, v.data(), v.size() * sizeof(T));
    return off;
  }
};

}  // namespace

struct Engine {
  iffd_options opt{};
  cudaStream_t st = nullptr;       // the engine's own stream (graph capture needs a non-default stream)
  cudaStream_t user_st = nullptr;  // the caller's stream: each step starts after its pending work
  cudaEvent_t ev = nullptr;
  int device = 0;
  char* arena_mem = nullptr;
  Arena arena;
  std::map<std::tuple<int, int, int, int>, iffd_plan*> plans;  // (d, n, p, Dirichlet flag bits)
  std::vector<Sys> active;
  std::vector<iffd_completion> done_list;
  long long next_id = 1;
  long long launches = 0;
  // descriptor buffers: init phase and iteration phase
  DevBuf dinit, diter, dstates;
  SolveState* hstates = nullptr;
  size_t hstates_cap = 0;
  // captured iteration graph, its kernel count and the membership it was built for
  cudaGraphExec_t graph = nullptr;
  long long graph_kernels = 0;
  int graph_lanes = 0;
  std::vector<long long> graph_ids;
  // persistent mode: one launch per step walks a device work queue
  // (persist.cu) instead of replaying the graph of batched launches
  bool persistent = false;
  long long wait_limit = 1LL << 26;  // polls of a bounded wait (64 ns sleeps)
  int inject_stall = 0;              // test hook: the first dependent range waits on a count never reached
  DevBuf dpers;                      // ranges, counters and the queue of the persistent launch
  std::vector<long long> pers_ids;   // membership the staged descriptors were built for
  std::vector<PRange> pers_ranges;   // host copy of the ranges of the current staging (one iteration)
  size_t pers_smem = 0;
  long long pers_items_per_iter = 0;
  PQueue* hqueue = nullptr;          // pinned copy of the queue after a launch
  // lane streams (forked from and joined to `st` inside the captured graph)
  std::vector<cudaStream_t> lane_st;
  std::vector<cudaEvent_t> lane_ev;
  cudaEvent_t fork_ev = nullptr;
  ~Engine() {
    if (st) cudaStreamSynchronize(st);
    if (graph) cudaGraphExecDestroy(graph);
    for (auto e : lane_ev) cudaEventDestroy(e);
    for (auto s : lane_st) cudaStreamDestroy(s);
    if (fork_ev) cudaEventDestroy(fork_ev);
    if (ev) cudaEventDestroy(ev);
    if (st) cudaStreamDestroy(st);
    for (auto& kv : plans) plan_release(kv.second);
    if (arena_mem) cudaFree(arena_mem);
    if (hstates) cudaFreeHost(hstates);
    if (hqueue) cudaFreeHost(hqueue);
  }
};

namespace {

template <typename T>
T* at(char* base, size_t off) {
  return reinterpret_cast<T*>(base + off);
}

double* vr(const Sys& s) { return reinterpret_cast<double*>(s.ws + s.plan->P.off_r); }
double* vz(const Sys& s) { return reinterpret_cast<double*>(s.ws + s.plan->P.off_z); }
double* vp(const Sys& s) { return reinterpret_cast<double*>(s.ws + s.plan->P.off_p); }
double* vq(const Sys& s) { return reinterpret_cast<double*>(s.ws + s.plan->P.off_q); }
double* vt1(const Sys& s) { return reinterpret_cast<double*>(s.ws + s.plan->P.off_t1); }
double* vt2(const Sys& s) { return reinterpret_cast<double*>(s.ws + s.plan->P.off_t2); }
float* vtf(const Sys& s) { return reinterpret_cast<float*>(s.ws + s.plan->P.off_tf); }
double* vpart(const Sys& s) { return reinterpret_cast<double*>(s.ws + s.plan->P.off_part); }
SolveState* vst(const Sys& s) { return reinterpret_cast<SolveState*>(s.ws + s.plan->P.off_state); }

// One batched transform launch: descriptors of the systems taking part.
template <typename Tc, typename Tin, typename Tout>
struct PassLaunchB {
  std::vector<PassDesc<Tc, Tin, Tout>> desc;
  std::vector<long long> prefix{0};
  size_t smem = 0;
  int mode = PM_FWD, ndot = 0;
  int wN = 0;     // > 0: every system runs the FP32 warp-FFT pass of this length
  int wkind = 0;  // and this transform kind (AxisTab::kind)
  int pair = 0;   // paired FP32 warp-FFT pass
  size_t off_desc = 0, off_prefix = 0;
  std::vector<int> sid;  // slot of the system of every descriptor
  void add(const PassDesc<Tc, Tin, Tout>& d, int tiles, size_t sm, int slot) {
    desc.push_back(d);
    sid.push_back(slot);
    prefix.push_back(prefix.back() + tiles);
    smem = std::max(smem, sm);
  }
};

struct StiffLaunchB {
  int p = 0, stage = 0;
  std::vector<StiffDesc> desc;
  std::vector<int> sid;
  std::vector<long long> prefix{0};
  size_t smem = 0;
  size_t off_desc = 0, off_prefix = 0;
};

struct VecLaunchB {
  std::vector<VecDesc> desc;
  std::vector<int> sid;
  std::vector<long long> prefix{0};
  size_t off_desc = 0, off_prefix = 0;
};

struct FinLaunchB {
  std::vector<FinDesc> desc;
  std::vector<int> sid;
  int phase = 0;
  size_t off = 0;
};

// The transform passes of one preconditioner apply for a set of systems, as
// batched launches. ndot: dot products fused into the last pass.
struct PrecondSeq {
  bool fp32 = false;
  // FP64 passes
  std::vector<PassLaunchB<double, double, double>> d64;
  // FP32 passes: first (r -> tf), middle (tf -> tf), last (tf -> z); one
  // launch per kernel: key 0 the block kernel, key N the warp-FFT pass of
  // length N (systems of one pass are independent, so splitting a pass into
  // launches does not change any result); key 2 N + (kind == 1) for the warp pass
  std::map<int, PassLaunchB<float, double, float>> f_first;
  std::vector<std::map<int, PassLaunchB<float, float, float>>> f_mid;
  std::map<int, PassLaunchB<float, float, double>> f_last;
};

template <typename L>
L& pass_slot(std::map<int, L>& m, int wN, int wkind, int pair, int mode, int ndot) {
  const int key = wN ? 4 * wN + 2 * (pair ? 1 : 0) + (wkind == 1 ? 1 : 0) : 0;
  auto it = m.find(key);
  if (it == m.end()) {
    L l;
    l.mode = mode;
    l.ndot = ndot;
    l.wN = wN;
    l.wkind = wkind;
    l.pair = pair;
    it = m.emplace(key, std::move(l)).first;
  }
  return it->second;
}

template <typename Tc>
PassDesc<Tc, Tc, Tc> pdesc_same(const Plan& P, int axis, const AxisTab<Tc>* tabs, const int* PPs, const int* ldts,
                                const int* done) {
  PassDesc<Tc, Tc, Tc> d{};
  d.dims = P.dims;
  d.axis = axis;
  d.PP = PPs[axis];
  d.ldt = ldts[axis];
  d.ax = tabs[axis];
  d.lamA = tabs[0].lam;
  d.lamB = (P.d == 3) ? tabs[1].lam : tabs[0].lam;
  d.done = done;
  d.wN = 0;
  d.wt = nullptr;
  d.pair = 0;
  if constexpr (std::is_same<Tc, float>::value) {
    const F32Geom g = f32_geom(P, axis);
    d.PP = g.PP;
    d.ldt = g.ldt;
    d.wN = g.wN;
    d.wt = g.wt;
    d.pair = g.pair;
  }
  return d;
}

// Builds the pass sequence; pass k of the sequence is: FWD axis 0, FWD axis 1
// (3D), FUSED last axis, BWD axis 1 (3D), BWD axis 0 (+dots).
void build_precond(const std::vector<const Sys*>& sys, int ndot, bool use_q, PrecondSeq* seq) {
  seq->fp32 = !sys.empty() && sys[0]->plan->P.opt.precision == IFFD_PREC_FP32_TRANSFORM;
  if (!seq->fp32) {
    seq->d64.assign(5, {});
    const int modes[5] = {PM_FWD, PM_FWD, PM_FUSED, PM_BWD, PM_BWD};
    for (int k = 0; k < 5; ++k) seq->d64[k].mode = modes[k];
    seq->d64[4].ndot = ndot;
    for (const Sys* s : sys) {
      const Plan& P = s->plan->P;
      const int* done = &vst(*s)->done;
      const int d = P.d;
      const int axes[5] = {0, 1, d - 1, 1, 0};
      for (int k = 0; k < 5; ++k) {
        if (d == 2 && (k == 1 || k == 3)) continue;
        const int a = axes[k];
        auto D = pdesc_same<double>(P, a, P.axd, P.PPd, P.ldtd, done);
        D.in = (k == 0) ? vr(*s) : vz(*s);
        D.out = vz(*s);
        if (k == 4) {
          D.dot0 = vr(*s);
          D.dot1 = use_q ? vq(*s) : nullptr;
          D.partial = vpart(*s);
        }
        seq->d64[k].add(D, precond_tiles(P.dims, a, P.PPd[a]),
                        precond_smem_bytes(P.PPd[a], P.ldtd[a], P.axd[a].F, sizeof(double)), s->slot);
      }
    }
    return;
  }
  seq->f_first.clear();
  seq->f_mid.assign(3, {});
  seq->f_last.clear();
  const int mid_modes[3] = {PM_FWD, PM_FUSED, PM_BWD};  // axis 1 (3D), last axis, axis 1 (3D)
  for (const Sys* s : sys) {
    const Plan& P = s->plan->P;
    const int* done = &vst(*s)->done;
    const int d = P.d;
    {
      PassDesc<float, double, float> D{};
      auto T = pdesc_same<float>(P, 0, P.axf, P.PPf, P.ldtf, done);
      D.dims = T.dims; D.axis = 0; D.PP = T.PP; D.ldt = T.ldt; D.ax = T.ax; D.lamA = T.lamA; D.lamB = T.lamB;
      D.wN = T.wN; D.wt = T.wt; D.pair = T.pair;
      D.done = done;
      D.in = vr(*s);
      D.out = vtf(*s);
      pass_slot(seq->f_first, D.wN, D.ax.kind, D.pair, PM_FWD, 0)
          .add(D, precond_tiles(P.dims, 0, D.PP), f32_geom(P, 0).smem, s->slot);
    }
    const int axes[3] = {1, d - 1, 1};
    for (int k = 0; k < 3; ++k) {
      if (d == 2 && k != 1) continue;
      const int a = axes[k];
      auto D = pdesc_same<float>(P, a, P.axf, P.PPf, P.ldtf, done);
      D.in = vtf(*s);
      D.out = vtf(*s);
      pass_slot(seq->f_mid[k], D.wN, D.ax.kind, D.pair, mid_modes[k], 0)
          .add(D, precond_tiles(P.dims, a, D.PP), f32_geom(P, a).smem, s->slot);
    }
    {
      PassDesc<float, float, double> D{};
      auto T = pdesc_same<float>(P, 0, P.axf, P.PPf, P.ldtf, done);
      D.dims = T.dims; D.axis = 0; D.PP = T.PP; D.ldt = T.ldt; D.ax = T.ax; D.lamA = T.lamA; D.lamB = T.lamB;
      D.wN = T.wN; D.wt = T.wt; D.pair = T.pair;
      D.done = done;
      D.in = vtf(*s);
      D.out = vz(*s);
      D.dot0 = vr(*s);
      D.dot1 = use_q ? vq(*s) : nullptr;
      D.partial = vpart(*s);
      pass_slot(seq->f_last, D.wN, D.ax.kind, D.pair, PM_BWD, ndot)
          .add(D, precond_tiles(P.dims, 0, D.PP), f32_geom(P, 0).smem, s->slot);
    }
  }
}

template <typename L>
void stage_pass(Staging& sg, L& l) {
  l.off_desc = sg.put(l.desc);
  l.off_prefix = sg.put(l.prefix);
}

void stage_precond(Staging& sg, PrecondSeq& q) {
  if (!q.fp32) {
    for (auto& l : q.d64) stage_pass(sg, l);
  } else {
    for (auto& kv : q.f_first) stage_pass(sg, kv.second);
    for (auto& m : q.f_mid)
      for (auto& kv : m) stage_pass(sg, kv.second);
    for (auto& kv : q.f_last) stage_pass(sg, kv.second);
  }
}

template <typename Tc, typename Tin, typename Tout>
int run_pass(Engine* E, char* base, PassLaunchB<Tc, Tin, Tout>& l, cudaStream_t st) {
  if (l.desc.empty()) return IFFD_OK;
  if constexpr (std::is_same<Tc, float>::value) {
    if (l.wN) {
      IFFD_CUDA((launch_wpass_batched<Tin, Tout>(at<PassDesc<Tc, Tin, Tout>>(base, l.off_desc),
                                                 at<long long>(base, l.off_prefix), (int)l.desc.size(),
                                                 l.prefix.back(), l.smem, l.wN, l.wkind, l.pair, l.mode,
                                                 l.ndot, st)));
      if (l.prefix.back() > 0) ++E->launches;
      return IFFD_OK;
    }
  }
  IFFD_CUDA((launch_pass_batched<Tc, Tin, Tout>(at<PassDesc<Tc, Tin, Tout>>(base, l.off_desc),
                                                at<long long>(base, l.off_prefix), (int)l.desc.size(),
                                                l.prefix.back(), l.smem, l.mode, l.ndot, st)));
  if (l.prefix.back() > 0) ++E->launches;
  return IFFD_OK;
}

int run_precond_seq(Engine* E, char* base, PrecondSeq& q, cudaStream_t st) {
  int rc;
  if (!q.fp32) {
    for (auto& l : q.d64)
      if ((rc = run_pass(E, base, l, st))) return rc;
    return IFFD_OK;
  }
  for (auto& kv : q.f_first)
    if ((rc = run_pass(E, base, kv.second, st))) return rc;
  for (auto& m : q.f_mid)
    for (auto& kv : m)
      if ((rc = run_pass(E, base, kv.second, st))) return rc;
  for (auto& kv : q.f_last)
    if ((rc = run_pass(E, base, kv.second, st))) return rc;
  return IFFD_OK;
}

int run_fin(Engine* E, char* base, FinLaunchB& f, cudaStream_t st) {
  if (f.desc.empty()) return IFFD_OK;
  IFFD_CUDA(launch_finalize_batched(at<FinDesc>(base, f.off), (int)f.desc.size(), f.phase,
                                    E->opt.rtol * E->opt.rtol, E->opt.maxit, st));
  ++E->launches;
  return IFFD_OK;
}

// ---- init phase of newly admitted systems
int run_init(Engine* E, const std::vector<const Sys*>& sys) {
  if (sys.empty()) return IFFD_OK;
  VecLaunchB vl;
  FinLaunchB fff, frz0;
  fff.phase = FP_FF;
  frz0.phase = FP_RZ0;
  for (const Sys* s : sys) {
    const Plan& P = s->plan->P;
    VecDesc v{};
    v.f = s->f;
    v.x = s->u;
    v.r = vr(*s);
    v.st = vst(*s);
    v.N = P.dims.N;
    v.part_rr = vpart(*s);
    v.p_zero = vp(*s);
    vl.desc.push_back(v);
    vl.prefix.push_back(vl.prefix.back() + vec_grid(P.dims.N));
    fff.desc.push_back({vst(*s), vpart(*s), vec_grid(P.dims.N)});
    frz0.desc.push_back({vst(*s), vpart(*s),
                         (P.opt.precision == IFFD_PREC_FP32_TRANSFORM) ? f32_last_parts(P)
                                                                        : precond_tiles(P.dims, 0, P.PPd[0])});
  }
  PrecondSeq pc;
  build_precond(sys, 1, false, &pc);
  Staging sg;
  stage_pass(sg, vl);
  fff.off = sg.put(fff.desc);
  frz0.off = sg.put(frz0.desc);
  stage_precond(sg, pc);
  IFFD_CUDA(E->dinit.reserve(sg.bytes.size()));
  char* base = E->dinit.p;
  IFFD_CUDA(cudaMemcpyAsync(base, sg.bytes.data(), sg.bytes.size(), cudaMemcpyHostToDevice, E->st));
  IFFD_CUDA(launch_pcg_init_batched(at<VecDesc>(base, vl.off_desc), at<long long>(base, vl.off_prefix),
                                    (int)vl.desc.size(), vl.prefix.back(), E->st));
  ++E->launches;
  int rc;
  if ((rc = run_fin(E, base, fff, E->st))) return rc;
  if ((rc = run_precond_seq(E, base, pc, E->st))) return rc;
  if ((rc = run_fin(E, base, frz0, E->st))) return rc;
  // the host copy of the staging must outlive the asynchronous upload
  IFFD_CUDA(cudaStreamSynchronize(E->st));
  return IFFD_OK;
}

// ---- one PCG iteration of all iterating systems, captured into a graph
struct IterSeq {
  std::vector<StiffLaunchB> stiff;  // grouped by (stage, p), in stage order
  FinLaunchB fpq, frr, frz;
  VecLaunchB upd;
  PrecondSeq pc;
};

int enqueue_iteration(Engine* E, char* base, IterSeq& it, cudaStream_t st) {
  int rc;
  for (auto& l : it.stiff) {
    if (l.desc.empty()) continue;
    IFFD_CUDA(launch_stiff_batched(l.p, l.stage, at<StiffDesc>(base, l.off_desc), at<long long>(base, l.off_prefix),
                                   (int)l.desc.size(), l.prefix.back(), l.smem, st));
    ++E->launches;
  }
  if ((rc = run_fin(E, base, it.fpq, st))) return rc;
  IFFD_CUDA(launch_pcg_update_batched(at<VecDesc>(base, it.upd.off_desc), at<long long>(base, it.upd.off_prefix),
                                      (int)it.upd.desc.size(), it.upd.prefix.back(), st));
  ++E->launches;
  if ((rc = run_fin(E, base, it.frr, st))) return rc;
  if ((rc = run_precond_seq(E, base, it.pc, st))) return rc;
  return run_fin(E, base, it.frz, st);
}

// The launch sequence of one iteration for the systems of one lane.
void build_lane(const Engine* E, const std::vector<const Sys*>& sys, IterSeq* out) {
  IterSeq& it = *out;
  std::map<std::pair<int, int>, size_t> group;  // (stage, p) -> index
  const bool flex = E->opt.flexible || E->opt.precision == IFFD_PREC_FP32_TRANSFORM;
  it.fpq.phase = FP_PQ;
  it.frr.phase = FP_RR;
  it.frz.phase = flex ? FP_RZ_FLEX : FP_RZ;
  for (const Sys* s : sys) {
    const Plan& P = s->plan->P;
    const int d = P.d;
    for (int stage = SS_FIRST; stage <= SS_LAST; ++stage) {
      if (d == 2 && stage == SS_MID) continue;
      const int axis = (stage == SS_FIRST) ? d - 1 : (stage == SS_MID ? 1 : 0);
      auto key = std::make_pair(stage, P.p);
      if (!group.count(key)) {
        group[key] = it.stiff.size();
        it.stiff.push_back({});
        it.stiff.back().p = P.p;
        it.stiff.back().stage = stage;
      }
      StiffLaunchB& l = it.stiff[group[key]];
      const StiffLaunch S = plan_stiff_launch(&P, axis);
      StiffDesc D{};
      D.dims = S.dims;
      D.axis = axis;
      D.PP = S.PP;
      D.ldt = S.ldt;
      D.bt = S.bt;
      D.z = vz(*s);
      D.p_io = vp(*s);
      D.beta = &vst(*s)->beta;
      D.pmode = 2;  // p = z + beta p, beta = 0 and p = 0 after the batched init
      D.T1 = vt1(*s);
      D.T2 = vt2(*s);
      D.out = vq(*s);
      D.dotv = vp(*s);
      D.partial = vpart(*s);
      D.done = &vst(*s)->done;
      l.desc.push_back(D);
      l.sid.push_back(s->slot);
      l.prefix.push_back(l.prefix.back() + stiff_tiles(P.dims, axis, S.PP));
      l.smem = std::max(l.smem, (size_t)(stage == SS_FIRST ? 1 : 2) * S.PP * S.ldt * sizeof(double));
    }
    it.fpq.desc.push_back({vst(*s), vpart(*s), stiff_tiles(P.dims, 0, P.PPs[0])});
    it.fpq.sid.push_back(s->slot);
    VecDesc v{};
    v.x = s->u;
    v.r = vr(*s);
    v.p = vp(*s);
    v.q = vq(*s);
    v.st = vst(*s);
    v.N = P.dims.N;
    v.part_rr = vpart(*s);
    it.upd.desc.push_back(v);
    it.upd.sid.push_back(s->slot);
    it.upd.prefix.push_back(it.upd.prefix.back() + vec_grid(P.dims.N));
    it.frr.desc.push_back({vst(*s), vpart(*s), vec_grid(P.dims.N)});
    it.frr.sid.push_back(s->slot);
    it.frz.desc.push_back({vst(*s), vpart(*s),
                           (P.opt.precision == IFFD_PREC_FP32_TRANSFORM) ? f32_last_parts(P)
                                                                          : precond_tiles(P.dims, 0, P.PPd[0])});
    it.frz.sid.push_back(s->slot);
  }
  // A system's three sweeps must run in stage order. Groups are created in the
  // order systems are met (a 2D system creates no MID group), so order them by
  // stage: every FIRST launch, then every MID, then every LAST.
  std::stable_sort(it.stiff.begin(), it.stiff.end(),
                   [](const StiffLaunchB& a, const StiffLaunchB& b) { return a.stage < b.stage; });
  build_precond(sys, flex ? 2 : 1, flex, &it.pc);
}

// Lane of a system: its degree and the occupancy class of its largest
// transform pass (CTAs of 227 KB / shared memory per SM, capped at 4), so that
// every batched launch of a lane sizes shared memory for systems alike.
std::pair<int, int> lane_key(const Sys& s) {
  const Plan& P = s.plan->P;
  const bool f32 = P.opt.precision == IFFD_PREC_FP32_TRANSFORM;
  size_t sm = 0;
  for (int a = 0; a < P.d; ++a)
    sm = std::max(sm, f32 ? f32_geom(P, a).smem
                          : precond_smem_bytes(P.PPd[a], P.ldtd[a], P.axd[a].F, sizeof(double)));
  const int occ = (int)std::min<size_t>(4, std::max<size_t>(1, (227 * 1024) / std::max<size_t>(sm, 1)));
  return {occ, P.p};
}

int build_iteration(Engine* E) {
  // partition the iterating systems into lanes; each lane runs its own launch
  // sequence on one of the engine's lane streams, concurrently with the others
  std::map<std::pair<int, int>, std::vector<const Sys*>> lanes;
  for (auto& s : E->active) lanes[lane_key(s)].push_back(&s);
  std::vector<IterSeq> seqs(lanes.size());
  {
    size_t k = 0;
    for (auto& kv : lanes) build_lane(E, kv.second, &seqs[k++]);
  }
  Staging sg;
  for (auto& it : seqs) {
    for (auto& l : it.stiff) stage_pass(sg, l);
    it.fpq.off = sg.put(it.fpq.desc);
    it.frr.off = sg.put(it.frr.desc);
    it.frz.off = sg.put(it.frz.desc);
    stage_pass(sg, it.upd);
    stage_precond(sg, it.pc);
  }
  IFFD_CUDA(E->diter.reserve(sg.bytes.size()));
  char* base = E->diter.p;
  IFFD_CUDA(cudaMemcpyAsync(base, sg.bytes.data(), sg.bytes.size(), cudaMemcpyHostToDevice, E->st));
  IFFD_CUDA(cudaStreamSynchronize(E->st));
  // raise the shared-memory attributes outside the capture (zero-tile launches)
  for (auto& it : seqs) {
    for (auto& l : it.stiff)
      IFFD_CUDA(launch_stiff_batched(l.p, l.stage, nullptr, nullptr, 0, 0, l.smem, E->st));
    IterSeq dry = it;
    for (auto& l : dry.pc.d64) l.prefix.assign(l.prefix.size(), 0);
    for (auto& kv : dry.pc.f_first) kv.second.prefix.assign(kv.second.prefix.size(), 0);
    for (auto& m : dry.pc.f_mid)
      for (auto& kv : m) kv.second.prefix.assign(kv.second.prefix.size(), 0);
    for (auto& kv : dry.pc.f_last) kv.second.prefix.assign(kv.second.prefix.size(), 0);
    const int rc = run_precond_seq(E, base, dry.pc, E->st);
    if (rc) return rc;
  }
  if (E->graph) {
    cudaGraphExecDestroy(E->graph);
    E->graph = nullptr;
  }
  const int nst = (int)std::min<size_t>(seqs.size(), kLaneStreams);
  for (int k = (int)E->lane_st.size(); k < nst; ++k) {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    IFFD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    E->lane_st.push_back(s);
    IFFD_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    E->lane_ev.push_back(ev);
  }
  // capture: fork every lane stream from the engine stream, enqueue each lane
  // on stream (lane mod nst), join them back
  cudaGraph_t g = nullptr;
  IFFD_CUDA(cudaStreamBeginCapture(E->st, cudaStreamCaptureModeThreadLocal));
  const long long before = E->launches;
  int rc = IFFD_OK;
  cudaError_t ce = cudaEventRecord(E->fork_ev, E->st);
  for (int k = 0; k < nst && ce == cudaSuccess; ++k) ce = cudaStreamWaitEvent(E->lane_st[k], E->fork_ev, 0);
  for (size_t k = 0; k < seqs.size() && ce == cudaSuccess && rc == IFFD_OK; ++k)
    rc = enqueue_iteration(E, base, seqs[k], E->lane_st[k % nst]);
  for (int k = 0; k < nst && ce == cudaSuccess; ++k) {
    ce = cudaEventRecord(E->lane_ev[k], E->lane_st[k]);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(E->st, E->lane_ev[k], 0);
  }
  const cudaError_t ce_end = cudaStreamEndCapture(E->st, &g);
  E->graph_kernels = E->launches - before;  // kernels per replay, counted when the graph is launched
  E->launches = before;
  if (rc || ce != cudaSuccess || ce_end != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (rc) return rc;
    return cuda_fail(ce != cudaSuccess ? ce : ce_end, "iteration graph capture");
  }
  ce = cudaGraphInstantiate(&E->graph, g, 0);
  cudaGraphDestroy(g);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
  E->graph_ids.clear();
  for (auto& s : E->active) E->graph_ids.push_back(s.id);
  E->pers_ids.clear();  // the persistent ranges' descriptors in diter were overwritten
  E->graph_lanes = (int)seqs.size();
  return IFFD_OK;
}

// ---- persistent launch: the item ranges of one iteration of every active
// system (all lanes), phase-major. Phase slots: the three stiffness stages,
// (p, A p), the update, (r, r), the five (3D) or three (2D) transform passes
// and (r, z); within a slot, the lanes' launches in lane order and their
// systems in launch order. `need` is filled per iteration by the caller.
template <typename L>
void add_ranges(std::vector<PRange>& out, char* base, L& l, size_t dsize, int kind, int arg) {
  for (size_t j = 0; j < l.desc.size(); ++j) {
    PRange r{};
    r.ntiles = (int)(l.prefix[j + 1] - l.prefix[j]);
    if (r.ntiles <= 0) continue;
    r.kind = kind;
    r.arg = arg;
    r.sys = l.sid[j];
    r.desc = base + l.off_desc + j * dsize;
    r.desc_bytes = (int)dsize;
    out.push_back(r);
  }
}

void add_fin_ranges(std::vector<PRange>& out, char* base, FinLaunchB& f) {
  for (size_t j = 0; j < f.desc.size(); ++j) {
    PRange r{};
    r.ntiles = 1;
    r.kind = PK_FIN;
    r.arg = f.phase;
    r.sys = f.sid[j];
    r.desc = base + f.off + j * sizeof(FinDesc);
    r.desc_bytes = (int)sizeof(FinDesc);
    out.push_back(r);
  }
}

int build_persistent(Engine* E) {
  std::map<std::pair<int, int>, std::vector<const Sys*>> lanes;
  for (auto& s : E->active) lanes[lane_key(s)].push_back(&s);
  std::vector<IterSeq> seqs(lanes.size());
  {
    size_t k = 0;
    for (auto& kv : lanes) build_lane(E, kv.second, &seqs[k++]);
  }
  Staging sg;
  for (auto& it : seqs) {
    for (auto& l : it.stiff) stage_pass(sg, l);
    it.fpq.off = sg.put(it.fpq.desc);
    it.frr.off = sg.put(it.frr.desc);
    it.frz.off = sg.put(it.frz.desc);
    stage_pass(sg, it.upd);
    stage_precond(sg, it.pc);
  }
  IFFD_CUDA(E->diter.reserve(sg.bytes.size()));
  char* base = E->diter.p;
  IFFD_CUDA(cudaMemcpyAsync(base, sg.bytes.data(), sg.bytes.size(), cudaMemcpyHostToDevice, E->st));
  std::vector<PRange>& R = E->pers_ranges;
  R.clear();
  size_t smem = 0;
  for (int stage = SS_FIRST; stage <= SS_LAST; ++stage)
    for (auto& it : seqs)
      for (auto& l : it.stiff)
        if (l.stage == stage) {
          add_ranges(R, base, l, sizeof(StiffDesc), PK_STIFF, stage * 32 + l.p);
          smem = std::max(smem, l.smem);
        }
  for (auto& it : seqs) add_fin_ranges(R, base, it.fpq);
  for (auto& it : seqs) add_ranges(R, base, it.upd, sizeof(VecDesc), PK_UPD, 0);
  for (auto& it : seqs) add_fin_ranges(R, base, it.frr);
  for (int k = 0; k < 5; ++k) {
    for (auto& it : seqs) {
      PrecondSeq& q = it.pc;
      if (!q.fp32) {
        auto& l = q.d64[k];
        add_ranges(R, base, l, sizeof(PassDesc<double, double, double>), PK_PASS_D, l.mode * 4 + l.ndot);
        smem = std::max(smem, l.smem);
      } else if (k == 0) {
        for (auto& kv : q.f_first) {
          if (kv.second.wN) return fail(IFFD_ERR_UNSUPPORTED, "persistent engine launch: warp-FFT passes");
          add_ranges(R, base, kv.second, sizeof(PassDesc<float, double, float>), PK_PASS_F_IN, 0);
          smem = std::max(smem, kv.second.smem);
        }
      } else if (k == 4) {
        for (auto& kv : q.f_last) {
          if (kv.second.wN) return fail(IFFD_ERR_UNSUPPORTED, "persistent engine launch: warp-FFT passes");
          add_ranges(R, base, kv.second, sizeof(PassDesc<float, float, double>), PK_PASS_F_OUT, kv.second.ndot);
          smem = std::max(smem, kv.second.smem);
        }
      } else {
        for (auto& kv : q.f_mid[k - 1]) {
          if (kv.second.wN) return fail(IFFD_ERR_UNSUPPORTED, "persistent engine launch: warp-FFT passes");
          add_ranges(R, base, kv.second, sizeof(PassDesc<float, float, float>), PK_PASS_F_MID, kv.second.mode);
          smem = std::max(smem, kv.second.smem);
        }
      }
    }
  }
  for (auto& it : seqs) add_fin_ranges(R, base, it.frz);
  long long items = 0;
  for (auto& r : R) items += r.ntiles;
  E->pers_items_per_iter = items;
  E->pers_smem = smem;
  E->pers_ids.clear();
  for (auto& s : E->active) E->pers_ids.push_back(s.id);
  E->graph_ids.clear();  // the graph's descriptors in diter were overwritten
  // the host staging must outlive the asynchronous upload
  IFFD_CUDA(cudaStreamSynchronize(E->st));
  return IFFD_OK;
}

// One persistent launch running `iterations` iterations of every active
// system; returns IFFD_ERR_TIMEOUT if a bounded wait ran out.
int run_persistent(Engine* E, int iterations) {
  const int nsys = (int)E->active.size();
  std::vector<PRange> all;
  all.reserve(E->pers_ranges.size() * iterations);
  std::vector<long long> cnt(nsys, 0);
  long long first = 0;
  for (int it = 0; it < iterations; ++it)
    for (const PRange& r0 : E->pers_ranges) {
      PRange r = r0;
      r.first = first;
      r.need = cnt[r.sys];
      cnt[r.sys] += r.ntiles;
      first += r.ntiles;
      all.push_back(r);
    }
  if (E->inject_stall) {
    // test hook: the first range that depends on earlier work waits on a
    // count nothing reaches, so its waits run out
    for (auto& r : all)
      if (r.need > 0) {
        r.need = 1LL << 62;
        break;
      }
  }
  const size_t off_cnt = al256(all.size() * sizeof(PRange));
  const size_t off_q = off_cnt + al256(nsys * sizeof(long long));
  const size_t bytes = off_q + al256(sizeof(PQueue));
  std::vector<char> host(bytes, 0);
  if (!all.empty()) std::memcpy(host.data(), all.data(), all.size() * sizeof(PRange));
  IFFD_CUDA(E->dpers.reserve(bytes));
  char* d = E->dpers.p;
  IFFD_CUDA(cudaMemcpyAsync(d, host.data(), bytes, cudaMemcpyHostToDevice, E->st));
  const int grid = std::min<long long>(persistent_grid(E->pers_smem), std::max<long long>(1, first));
  if (grid < 1) return fail(IFFD_ERR_UNSUPPORTED, "persistent engine launch does not fit on an SM");
  IFFD_CUDA(launch_persistent(reinterpret_cast<PRange*>(d), (int)all.size(), first,
                              reinterpret_cast<long long*>(d + off_cnt), reinterpret_cast<PQueue*>(d + off_q),
                              E->wait_limit, E->opt.rtol * E->opt.rtol, E->opt.maxit, E->pers_smem, grid, E->st));
  ++E->launches;
  if (!E->hqueue) IFFD_CUDA(cudaHostAlloc((void**)&E->hqueue, sizeof(PQueue), cudaHostAllocDefault));
  IFFD_CUDA(cudaMemcpyAsync(E->hqueue, d + off_q, sizeof(PQueue), cudaMemcpyDeviceToHost, E->st));
  // the host copy must outlive the upload; the status is read after the step's sync
  IFFD_CUDA(cudaStreamSynchronize(E->st));
  if (E->hqueue->status != 0)
    return fail(IFFD_ERR_TIMEOUT, "persistent engine launch: a bounded device wait ran out (results of this step "
                                  "are not valid)");
  return IFFD_OK;
}

}  // namespace

}  // namespace iffd

using namespace iffd;

struct iffd_engine {
  Engine E;
};

namespace iffd {
// One engine step (iffd_engine_step without the handle): initialise the
// admitted systems, run `iterations` PCG iterations of every active system,
// retire the finished ones.
int engine_step(Engine& E, int iterations, int* active);
}  // namespace iffd

extern "C" {

int iffd_engine_create(const iffd_options* opt, size_t budget_bytes, void* stream, iffd_engine_handle* out) {
  g_err.clear();
  if (!out) return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  iffd_options o;
  iffd_default_options(&o);
  if (opt) o = *opt;
  if (o.precond != IFFD_PRECOND_IFFD || o.coef != IFFD_COEF_CONST)
    return fail(IFFD_ERR_UNSUPPORTED, "the engine serves IFFD-preconditioned constant-coefficient solves");
  if (budget_bytes < 4096) return fail(IFFD_ERR_INVALID_ARG, "budget too small");
  iffd_engine* h = new iffd_engine();
  Engine& E = h->E;
  E.opt = o;
  E.user_st = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&E.device);
  cudaError_t e = cudaStreamCreateWithFlags(&E.st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&E.ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&E.fork_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "engine stream");
  }
  e = cudaMalloc(&E.arena_mem, budget_bytes);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "engine arena");
  }
  E.arena.init(E.arena_mem, budget_bytes);
  *out = h;
  return IFFD_OK;
}

// Plan of a request class; dirichlet: 2d flags (NULL: Dirichlet on every face).
static int engine_plan(iffd_engine* h, int d, int n, int p, const int* dirichlet, iffd_plan** out) {
  Engine& E = h->E;
  if (d != 2 && d != 3) return fail(IFFD_ERR_INVALID_ARG, "d must be 2 or 3");
  int dir[6] = {1, 1, 1, 1, 1, 1};
  int bits = 0;
  for (int k = 0; k < 2 * d; ++k) {
    if (dirichlet) dir[k] = dirichlet[k] != 0;
    bits |= dir[k] << k;
  }
  auto key = std::make_tuple(d, n, p, bits);
  auto it = E.plans.find(key);
  if (it != E.plans.end()) {
    *out = it->second;
    return IFFD_OK;
  }
  const int nn[3] = {n, n, n};
  iffd_options o = E.opt;
  o.true_residual = 0;
  iffd_plan* P = nullptr;
  const int rc = plan_create(d, nn, p, dir, &o, E.st, &P);
  if (rc) return rc;
  P->P.dfq = 0;  // the engine's batched FP64 passes are the block kernel
  if (E.persistent)
    for (int a = 0; a < d; ++a) P->P.warp_f[a] = 0;  // the persistent launch runs the block kernel
  E.plans[key] = P;
  *out = P;
  return IFFD_OK;
}

int iffd_engine_request_bytes(iffd_engine_handle h, int d, int n, int p, const int* dirichlet, size_t* bytes) {
  if (!h || !bytes) return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  iffd_plan* P = nullptr;
  const int rc = engine_plan(h, d, n, p, dirichlet, &P);
  if (rc) return rc;
  *bytes = al256(P->P.ws_bytes);
  return IFFD_OK;
}

int iffd_engine_submit(iffd_engine_handle h, int d, int n, int p, const int* dirichlet, const double* f, double* u,
                       long long* id) {
  if (!h || !f || !u || !id) return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  if (f == u) return fail(IFFD_ERR_INVALID_ARG, "f and u must not alias");
  Engine& E = h->E;
  if (E.persistent && (p < kPersistMinP || p > kPersistMaxP))
    return fail(IFFD_ERR_UNSUPPORTED, "the persistent engine launch serves degrees 2..8");
  iffd_plan* P = nullptr;
  int rc = engine_plan(h, d, n, p, dirichlet, &P);
  if (rc) return rc;
  const size_t need = al256(P->P.ws_bytes);
  if (need > E.arena.bytes) return fail(IFFD_ERR_UNSUPPORTED, "request needs more workspace than the whole budget");
  size_t off = 0;
  if (!E.arena.alloc(need, &off)) return fail(IFFD_ERR_WORKSPACE, "budget exhausted: resubmit after completions");
  if (E.opt.autotune && !P->P.tuned) {
    // first request of this (d, n, p): tune its plan on the request's own
    // workspace (no other system uses this plan yet)
    rc = plan_autotune(&P->P, E.arena_mem + off, E.st);
    if (rc) {
      E.arena.release(off, need);
      return rc;
    }
    if (E.persistent)
      for (int a = 0; a < d; ++a) P->P.warp_f[a] = 0;
  }
  Sys s{};
  s.id = E.next_id++;
  s.plan = P;
  s.f = f;
  s.u = u;
  s.off = off;
  s.bytes = need;
  s.ws = E.arena_mem + off;
  s.phase = 0;
  E.active.push_back(s);
  *id = s.id;
  return IFFD_OK;
}

int iffd_engine_step(iffd_engine_handle h, int iterations, int* active) {
  if (!h || iterations < 0) return fail(IFFD_ERR_INVALID_ARG, "bad argument");
  return engine_step(h->E, iterations, active);
}

}  // extern "C"

namespace iffd {

int engine_step(Engine& E, int iterations, int* active) {
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != E.device) return fail(IFFD_ERR_INVALID_ARG, "engine was created on another device");
  IFFD_CUDA(cudaEventRecord(E.ev, E.user_st));
  IFFD_CUDA(cudaStreamWaitEvent(E.st, E.ev, 0));
  for (size_t i = 0; i < E.active.size(); ++i) E.active[i].slot = (int)i;
  // 1. initialise newly admitted systems
  std::vector<const Sys*> fresh;
  for (auto& s : E.active)
    if (s.phase == 0) fresh.push_back(&s);
  int rc = run_init(&E, fresh);
  if (rc) return rc;
  for (auto& s : E.active) s.phase = 1;
  // 2. iterations of every active system: one persistent launch (descriptors
  // rebuilt when membership changed), or the captured graph of batched
  // launches (rebuilt when membership changed)
  if (E.persistent && !E.active.empty() && iterations > 0) {
    bool same = E.pers_ids.size() == E.active.size();
    for (size_t i = 0; same && i < E.active.size(); ++i) same = E.pers_ids[i] == E.active[i].id;
    if (!same) {
      rc = build_persistent(&E);
      if (rc) return rc;
    }
    rc = run_persistent(&E, iterations);
    if (rc) return rc;
  } else if (!E.active.empty() && iterations > 0) {
    bool same = E.graph && E.graph_ids.size() == E.active.size();
    for (size_t i = 0; same && i < E.active.size(); ++i) same = E.graph_ids[i] == E.active[i].id;
    if (!same) {
      rc = build_iteration(&E);
      if (rc) return rc;
    }
    for (int k = 0; k < iterations; ++k) {
      cudaError_t e = cudaGraphLaunch(E.graph, E.st);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
      E.launches += E.graph_kernels;
    }
  }
  // 3. read every state, retire finished systems
  const int n = (int)E.active.size();
  if (n > 0) {
    std::vector<SolveState*> ptrs(n);
    for (int i = 0; i < n; ++i) ptrs[i] = vst(E.active[i]);
    IFFD_CUDA(E.dstates.reserve(al256(n * sizeof(SolveState*)) + n * sizeof(SolveState)));
    SolveState** dptr = reinterpret_cast<SolveState**>(E.dstates.p);
    SolveState* dst = reinterpret_cast<SolveState*>(E.dstates.p + al256(n * sizeof(SolveState*)));
    IFFD_CUDA(cudaMemcpyAsync(dptr, ptrs.data(), n * sizeof(SolveState*), cudaMemcpyHostToDevice, E.st));
    IFFD_CUDA(launch_gather_states(dptr, dst, n, E.st));
    ++E.launches;
    if ((size_t)n > E.hstates_cap) {
      if (E.hstates) cudaFreeHost(E.hstates);
      E.hstates = nullptr;
      IFFD_CUDA(cudaHostAlloc((void**)&E.hstates, n * sizeof(SolveState), cudaHostAllocDefault));
      E.hstates_cap = n;
    }
    IFFD_CUDA(cudaMemcpyAsync(E.hstates, dst, n * sizeof(SolveState), cudaMemcpyDeviceToHost, E.st));
    IFFD_CUDA(cudaStreamSynchronize(E.st));
    std::vector<Sys> keep;
    for (int i = 0; i < n; ++i) {
      const SolveState& ss = E.hstates[i];
      if (ss.done) {
        iffd_completion c{};
        c.id = E.active[i].id;
        c.info.iters = ss.iters;
        c.info.rel_res = ss.ff > 0 ? std::sqrt(ss.rr / ss.ff) : 0.0;
        c.info.true_rel_res = -1.0;
        c.info.status = ss.status;
        E.done_list.push_back(c);
        E.arena.release(E.active[i].off, E.active[i].bytes);
      } else {
        keep.push_back(E.active[i]);
      }
    }
    E.active.swap(keep);
  }
  if (active) *active = (int)E.active.size();
  return IFFD_OK;
}

}  // namespace iffd

extern "C" {

int iffd_engine_poll(iffd_engine_handle h, iffd_completion* out, int capacity, int* count) {
  if (!h || !count || (capacity > 0 && !out)) return fail(IFFD_ERR_INVALID_ARG, "bad argument");
  Engine& E = h->E;
  const int n = std::min<int>(capacity, (int)E.done_list.size());
  for (int i = 0; i < n; ++i) out[i] = E.done_list[i];
  E.done_list.erase(E.done_list.begin(), E.done_list.begin() + n);
  *count = n;
  return IFFD_OK;
}

int iffd_engine_stats(iffd_engine_handle h, int* active, size_t* bytes_free, long long* kernel_launches) {
  if (!h) return fail(IFFD_ERR_INVALID_ARG, "NULL handle");
  if (active) *active = (int)h->E.active.size();
  if (bytes_free) *bytes_free = h->E.arena.available();
  if (kernel_launches) *kernel_launches = h->E.launches;
  return IFFD_OK;
}

int iffd_engine_set_persistent(iffd_engine_handle h, int on, long long wait_limit, int inject_stall) {
  g_err.clear();
  if (!h) return fail(IFFD_ERR_INVALID_ARG, "NULL handle");
  Engine& E = h->E;
  if (!E.active.empty()) return fail(IFFD_ERR_INVALID_ARG, "change the launch mode only while no request is active");
  E.persistent = on != 0;
  E.wait_limit = wait_limit > 0 ? wait_limit : (1LL << 26);
  E.inject_stall = inject_stall != 0;
  if (E.persistent)
    for (auto& kv : E.plans)
      for (int a = 0; a < kv.second->P.d; ++a) kv.second->P.warp_f[a] = 0;
  E.pers_ids.clear();
  return IFFD_OK;
}

int iffd_engine_destroy(iffd_engine_handle h) {
  if (!h) return IFFD_OK;
  cudaStreamSynchronize(h->E.st);
  delete h;
  return IFFD_OK;
}

}  // extern "C"

// ------------------------------------------------------------ batch solve
// iffd_batch_solve: the systems (plan i, right-hand side j < nrhs[i]) of one
// call run through the engine's batched launches, over the caller's plans and
// the caller's workspace. Systems whose plans the engine's kernels cannot run
// exactly as iffd_pcg_solve would (another preconditioner or coefficient, or
// an FP64 plan set to the FP64 warp-FFT pass) are solved one by one with
// iffd_pcg_solve on their slice of the same workspace. Every result is
// therefore that of iffd_pcg_solve on the same plan.

namespace iffd {

int plan_true_residual(iffd_handle h, const double* f, const double* u, void* ws, cudaStream_t st, double* out);

namespace {

bool engine_runs_exactly(const Plan& P) {
  if (P.opt.precond != IFFD_PRECOND_IFFD || P.opt.coef != IFFD_COEF_CONST) return false;
  if (P.opt.precision == IFFD_PREC_FP64 && P.dfq) return false;  // double-float passes: not batched
  if (P.opt.precision == IFFD_PREC_FP64)
    for (int a = 0; a < P.d; ++a)
      if (f64_warp_len(P, a)) return false;
  return true;
}

// Engine options of a plan's systems: the solve options that the engine
// applies to all systems of one engine.
std::tuple<int, int, double, int> engine_key(const Plan& P) {
  const int flex = (P.opt.flexible || P.opt.precision == IFFD_PREC_FP32_TRANSFORM) ? 1 : 0;
  return std::make_tuple(P.opt.precision, flex, P.opt.rtol, P.opt.maxit);
}

int batch_check(int count, const iffd_handle* plans, const int* nrhs) {
  if (count < 0 || (count > 0 && (!plans || !nrhs))) return fail(IFFD_ERR_INVALID_ARG, "bad count or NULL array");
  int dev = -1;
  IFFD_CUDA(cudaGetDevice(&dev));
  for (int i = 0; i < count; ++i) {
    if (!plans[i]) return fail(IFFD_ERR_INVALID_ARG, "NULL plan in the batch");
    if (nrhs[i] < 0) return fail(IFFD_ERR_INVALID_ARG, "negative right-hand-side count");
    if (plans[i]->P.device != dev) return fail(IFFD_ERR_INVALID_ARG, "a plan was created on another CUDA device");
  }
  return IFFD_OK;
}

}  // namespace
}  // namespace iffd

extern "C" {

int iffd_batch_workspace_bytes(int count, const iffd_handle* plans, const int* nrhs, size_t* bytes) {
  g_err.clear();
  if (!bytes) return fail(IFFD_ERR_INVALID_ARG, "NULL argument");
  int rc = batch_check(count, plans, nrhs);
  if (rc) return rc;
  size_t total = 0;
  for (int i = 0; i < count; ++i) total += (size_t)nrhs[i] * al256(plans[i]->P.ws_bytes);
  *bytes = total;
  return IFFD_OK;
}

int iffd_batch_solve(int count, const iffd_handle* plans, const double* const* f, double* const* u, const int* nrhs,
                     void* ws, void* stream, iffd_pcg_info* infos) {
  g_err.clear();
  int rc = batch_check(count, plans, nrhs);
  if (rc) return rc;
  long long nsys = 0;
  for (int i = 0; i < count; ++i) {
    if (nrhs[i] > 0 && (!f || !u || !f[i] || !u[i])) return fail(IFFD_ERR_INVALID_ARG, "NULL right-hand side or solution");
    if (nrhs[i] > 0 && f[i] == u[i]) return fail(IFFD_ERR_INVALID_ARG, "f[i] and u[i] must not alias");
    nsys += nrhs[i];
  }
  if (nsys == 0) return IFFD_OK;
  if (!infos) return fail(IFFD_ERR_INVALID_ARG, "NULL infos");
  if (!ws) return fail(IFFD_ERR_WORKSPACE, "workspace pointer is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(IFFD_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  size_t total = 0;
  iffd_batch_workspace_bytes(count, plans, nrhs, &total);

  // every system: its plan, right-hand side, solution and workspace slice
  struct Item {
    iffd_plan* plan;
    const double* f;
    double* u;
    char* ws;
    size_t off, bytes;
    long long slot;  // index into infos
  };
  std::vector<Item> items;
  {
    size_t off = 0;
    long long slot = 0;
    for (int i = 0; i < count; ++i) {
      const long long N = plans[i]->P.dims.N;
      const size_t b = al256(plans[i]->P.ws_bytes);
      for (int j = 0; j < nrhs[i]; ++j, ++slot) {
        items.push_back({plans[i], f[i] + (size_t)j * N, u[i] + (size_t)j * N, base + off, off, b, slot});
        off += b;
      }
    }
  }
  for (long long k = 0; k < nsys; ++k) infos[k] = iffd_pcg_info{0, 0.0, -1.0, IFFD_OK};

  // engine groups (one engine per set of solve options); the rest one by one
  std::map<std::tuple<int, int, double, int>, std::vector<const Item*>> groups;
  std::vector<const Item*> alone;
  for (const Item& it : items) {
    if (engine_runs_exactly(it.plan->P)) groups[engine_key(it.plan->P)].push_back(&it);
    else alone.push_back(&it);
  }
  for (auto& kv : groups) {
    Engine E;
    iffd_default_options(&E.opt);
    E.opt.precision = std::get<0>(kv.first);
    E.opt.flexible = std::get<1>(kv.first);
    E.opt.rtol = std::get<2>(kv.first);
    E.opt.maxit = std::get<3>(kv.first);
    E.user_st = st;
    IFFD_CUDA(cudaGetDevice(&E.device));
    IFFD_CUDA(cudaStreamCreateWithFlags(&E.st, cudaStreamNonBlocking));
    IFFD_CUDA(cudaEventCreateWithFlags(&E.ev, cudaEventDisableTiming));
    IFFD_CUDA(cudaEventCreateWithFlags(&E.fork_ev, cudaEventDisableTiming));
    // the arena bookkeeping spans the caller's workspace and hands every
    // system of the group its slice laid out above (E.arena_mem stays null:
    // the engine frees nothing of the caller's)
    E.arena.init(base, total);
    for (const Item& it : items) {
      size_t off = 0;
      if (!E.arena.alloc(it.bytes, &off) || off != it.off) return fail(IFFD_ERR_WORKSPACE, "batch workspace layout");
    }
    std::map<long long, const Item*> by_id;
    for (const Item* it : kv.second) {
      Sys s{};
      s.id = E.next_id++;
      s.plan = it->plan;
      s.f = it->f;
      s.u = it->u;
      s.off = it->off;
      s.bytes = it->bytes;
      s.ws = it->ws;
      s.phase = 0;
      E.active.push_back(s);
      by_id[s.id] = it;
    }
    int active = (int)E.active.size();
    while (active > 0) {
      rc = engine_step(E, 4, &active);
      if (rc) return rc;
    }
    for (const iffd_completion& c : E.done_list) infos[by_id[c.id]->slot] = c.info;
  }
  for (const Item* it : alone) {
    iffd_pcg_info info{};
    rc = iffd_pcg_solve(it->plan, it->f, it->u, it->ws, stream, &info);
    if (rc != IFFD_OK && rc != IFFD_ERR_NOT_CONVERGED && rc != IFFD_ERR_BREAKDOWN) return rc;
    infos[it->slot] = info;
  }
  // true residuals where the plan asks for them (as iffd_pcg_solve reports them)
  for (const Item& it : items) {
    if (!it.plan->P.opt.true_residual || !engine_runs_exactly(it.plan->P)) continue;
    double tr = -1.0;
    rc = plan_true_residual(it.plan, it.f, it.u, it.ws, st, &tr);
    if (rc) return rc;
    infos[it.slot].true_rel_res = tr;
  }
  g_err.clear();
  for (long long k = 0; k < nsys; ++k)
    if (infos[k].status != IFFD_OK)
      return fail(infos[k].status, "system " + std::to_string(k) + " of the batch: " +
                                       (infos[k].status == IFFD_ERR_NOT_CONVERGED ? "PCG did not reach rtol within maxit"
                                                                                  : "PCG breakdown"));
  return IFFD_OK;
}

}  // extern "C"
