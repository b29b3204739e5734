// Host-visible launch interfaces of the IFFD CUDA kernels.
#pragma once

#include <cuda_runtime.h>

#include "device_common.cuh"

namespace iffd {

enum PassMode : int { PM_FWD = 0, PM_BWD = 1, PM_FUSED = 2 };

template <typename Tc>
struct PassLaunch {
  Dims dims;
  int axis;
  int PP;   // pencils per CTA (even)
  int ldt;  // shared-memory row length of the pencil tile
  AxisTab<Tc> ax;
  const Tc* lamA;  // eigenvalues of direction 0 (FUSED)
  const Tc* lamB;  // eigenvalues of direction 1 (FUSED, d = 3)
  const double* dot0;  // optional: partial (dot0, out) per CTA
  const double* dot1;  // optional: partial (dot1, out) per CTA
  double* partial;
  const int* done;     // optional early-exit flag (PCG)
  int pipe;            // 1: persistent two-stage pipelined kernel (same input and arithmetic type only)
  int wN;              // > 0 runs the warp-FFT pass of length wN (PP, ldt as wpass_pencils)
  const vec2_t<Tc>* wt;  // its twiddles exp(-2 pi i e / wN), e < wN
  int pair;            // FP32 warp pass with two sequences per lane group (wN <= 256)
};

// Per-system descriptor of one batched transform pass.
template <typename Tc, typename Tin, typename Tout>
struct PassDesc {
  const Tin* in;
  Tout* out;
  Dims dims;
  int axis, PP, ldt;
  AxisTab<Tc> ax;
  const Tc* lamA;
  const Tc* lamB;
  const double* dot0;
  const double* dot1;
  double* partial;
  const int* done;
  int wN;            // as PassLaunch
  const vec2_t<Tc>* wt;
  int pair;          // as PassLaunch
};

template <typename Tc, typename Tin, typename Tout>
cudaError_t launch_pass_batched(const PassDesc<Tc, Tin, Tout>* sys, const long long* tile_prefix, int nsys,
                                long long total_tiles, size_t smem, int mode, int ndot, cudaStream_t st);

// Batched warp-FFT passes: every system of the launch has wN == N and
// transform kind `kind` (AxisTab::kind: 1 DST-II/III, 0 DST-I).
template <typename Tin, typename Tout>
cudaError_t launch_wpass_batched(const PassDesc<float, Tin, Tout>* sys, const long long* tile_prefix, int nsys,
                                 long long total_tiles, size_t smem, int N, int kind, int pair, int mode,
                                 int ndot, cudaStream_t st);

// Per FFT length N (one translation unit each): the warp-FFT pass of one
// direction, and its batched form (every system of the launch has wN == N and
// transform kind `kind`).
template <int N, typename Tc, typename Tin, typename Tout>
cudaError_t launch_wpass(const PassLaunch<Tc>& P, int mode, int ndot, const Tin* in, Tout* out, cudaStream_t st);
template <int N, typename Tin, typename Tout>
cudaError_t launch_wpass_batched_n(const PassDesc<float, Tin, Tout>* sys, const long long* tile_prefix, int nsys,
                                   long long total_tiles, size_t smem, int kind, int pair, int mode, int ndot,
                                   cudaStream_t st);

size_t precond_smem_bytes(int PP, int ldt, int F, size_t elt);       // F: FFT length (AxisTab::F)
size_t precond_smem_bytes_pipe(int PP, int ldt, int F, size_t elt);  // pipelined kernel: one more tile
// Fills AxisTab::rden of an FP64 plan (see device_common.cuh).
cudaError_t launch_rden_fill(double* rden, const Dims& dims, const double* lamF, const double* lam0,
                             const double* lam1, cudaStream_t st);  // F: FFT length (AxisTab::F)
int precond_tiles(const Dims& dims, int axis, int PP);
// Warp-FFT passes (D = {0,1} directions whose FFT length is 64, 128, 256 or
// 512 -- FP64: 64, 128 or 256: DST-II/III with n_reg of that length, DST-I
// with 2 (n_reg + 1)): the length the pass runs at for a direction with these
// tables (0: not eligible), its pencils per tile, and its shared memory for
// tile row length ldt and arithmetic of elt bytes.
int wpass_len(const AxisTab<float>& ax);
int wpass_len(const AxisTab<double>& ax);
int wpass_len(const AxisTab<df>& ax);
// Double-float transform pass (the warp-FFT pass of length P.wN with df
// arithmetic): FP64 in / df out (FWD), df in and out (any mode), df in / FP64
// out (BWD, 0..2 dot products).
template <typename Tin, typename Tout>
cudaError_t launch_pass_df(const PassLaunch<df>& P, int mode, int ndot, const Tin* in, Tout* out, cudaStream_t st);
// Pencils per CTA and shared memory of the warp-FFT pass of length N (pair:
// the paired FP32 pass, N <= 256; ldt: tile row length in pencil values).
int wpass_pencils(int N, bool pair = false);
// SMs of the current device (cached at the first call).
int device_sm_count();
size_t wpass_smem_bytes(int N, int ldt, size_t elt = sizeof(float), bool pair = false, bool alias = false);
// Tile row length of the warp-FFT pass of length N for m values per pencil
// (odd, for banks; with alias the rows of a pencil pair also hold its
// sequence buffer, see walias).
int wpass_ldt(int N, int m, bool alias);

template <typename Tc, typename Tin, typename Tout>
cudaError_t launch_pass(const PassLaunch<Tc>& P, int mode, int ndot, const Tin* in, Tout* out, cudaStream_t st);

// ---------------------------------------------------------------- stiffness
// Banded 1D operator data for one direction (device pointers).
struct BandTab {
  int m, p;
  const double* Mb;  // m * (2p+1) band rows of M
  const double* Kb;  // m * (2p+1) band rows of K
  const double* Mt;  // p+1 Toeplitz coefficients of interior rows of M
  const double* Kt;  // p+1 Toeplitz coefficients of interior rows of K
  int ilo, ihi;      // rows [ilo, ihi) are Toeplitz interior rows
};

enum StiffStage : int { SS_FIRST = 0, SS_MID = 1, SS_LAST = 2 };

struct StiffLaunch {
  Dims dims;
  int axis;
  int PP;
  int ldt;
  BandTab bt;
};

// FIRST: (optionally p_new = z + beta p) -> T1 = M u, T2 = K u
// MID:   T1 <- M T1, T2 <- K T1 + M T2
// LAST:  out = K T1 + M T2, optional partial (dotv, out)
cudaError_t launch_stiff_first(const StiffLaunch& S, const double* u, const double* z, double* p_io,
                               const double* beta, int pmode, double* T1, double* T2, const int* done,
                               cudaStream_t st);
cudaError_t launch_stiff_mid(const StiffLaunch& S, double* T1, double* T2, const int* done, cudaStream_t st);
cudaError_t launch_stiff_last(const StiffLaunch& S, const double* T1, const double* T2, double* out,
                              const double* dotv, double* partial, const int* done, cudaStream_t st);
int stiff_tiles(const Dims& dims, int axis, int PP);

// Per-system descriptor of one batched stiffness sweep (fields unused by a
// stage are ignored).
struct StiffDesc {
  Dims dims;
  int axis, PP, ldt;
  BandTab bt;
  const double* u;
  const double* z;
  double* p_io;
  const double* beta;
  int pmode;
  double* T1;
  double* T2;
  double* out;
  const double* dotv;
  double* partial;
  const int* done;
};
// All systems of one launch share the degree p.
cudaError_t launch_stiff_batched(int p, int stage, const StiffDesc* sys, const long long* tile_prefix, int nsys,
                                 long long total_tiles, size_t smem, cudaStream_t st);

// Variable coefficient a = 1 + c prod_k s(x_k): the operator is
// A^ + c sum_k (M^s x .. x K^s_k x .. x M^s) with banded 1D matrices weighted by s.
struct WBandTab {
  const double* Msb;  // m * (2p+1) band rows of M^s
  const double* Ksb;  // m * (2p+1) band rows of K^s
  double c;
};
// FIRST: T1 = M u, T2 = K u, T3 = M^s u, T4 = K^s u (optional p update as above)
// MID:   T1 <- M T1, T2 <- K T1 + M T2, T3 <- M^s T3, T4 <- K^s T3 + M^s T4
// LAST:  out = K T1 + M T2 + c (K^s T3 + M^s T4), optional partial (dotv, out)
cudaError_t launch_vstiff_first(const StiffLaunch& S, const WBandTab& wb, const double* u, const double* z,
                                double* p_io, const double* beta, int pmode, double* T1, double* T2, double* T3,
                                double* T4, const int* done, cudaStream_t st);
cudaError_t launch_vstiff_mid(const StiffLaunch& S, const WBandTab& wb, double* T1, double* T2, double* T3,
                              double* T4, const int* done, cudaStream_t st);
cudaError_t launch_vstiff_last(const StiffLaunch& S, const WBandTab& wb, const double* T1, const double* T2,
                               const double* T3, const double* T4, double* out, const double* dotv,
                               double* partial, const int* done, cudaStream_t st);

// ---------------------------------------------------------------- PCG vectors
int vec_grid(long long N);
// x = 0, r = f, partial ||f||^2; a non-null state is reset to zero first.
cudaError_t launch_pcg_init(const double* f, double* x, double* r, long long N, double* partial, cudaStream_t st,
                            SolveState* state = nullptr);
cudaError_t launch_pcg_update(double* x, double* r, const double* p, const double* q, const SolveState* s,
                              long long N, double* partial, const int* done, cudaStream_t st);
// phase-specific reduction of `nparts` partial sums into the solve state
enum FinalizePhase : int { FP_FF = 0, FP_RZ0 = 1, FP_PQ = 2, FP_RR = 3, FP_RZ = 4, FP_RZ_FLEX = 5, FP_TRUE = 6 };
cudaError_t launch_finalize(SolveState* s, const double* partial, int nparts, int phase, double tol2, int maxit,
                            cudaStream_t st);
cudaError_t launch_residual(const double* f, const double* Au, long long N, double* partial, cudaStream_t st);

// Batched vector kernels (one descriptor per system).
struct VecDesc {
  const double* f;
  double* x;
  double* r;
  const double* p;
  const double* q;
  SolveState* st;
  long long N;
  double* part_rr;  // partial sums of ||f||^2 / ||r||^2 (vec_grid(N) entries)
  double* p_zero;   // batched init only: search direction to clear (may be null)
};
cudaError_t launch_gather_states(SolveState* const* src, SolveState* dst, int n, cudaStream_t st);
struct FinDesc {
  SolveState* st;
  const double* partial;
  int nparts;
};
cudaError_t launch_pcg_init_batched(const VecDesc* sys, const long long* prefix, int nsys, long long total_blocks,
                                    cudaStream_t st);
cudaError_t launch_pcg_update_batched(const VecDesc* sys, const long long* prefix, int nsys, long long total_blocks,
                                      cudaStream_t st);
cudaError_t launch_finalize_batched(const FinDesc* sys, int nsys, int phase, double tol2, int maxit, cudaStream_t st);

// ------------------------------------------------------ persistent engine
// One persistent launch walks a device work queue of item ranges: the tiles
// (or vector blocks, or the single reduction) of one system in one phase of
// one PCG iteration. Ranges are listed phase-major (iteration, phase, system),
// so an item waits only on items of its own system with earlier tickets.
enum PersistKind : int {
  PK_STIFF = 0,       // StiffDesc; arg = stage * 32 + p
  PK_FIN = 1,         // FinDesc; arg = finalize phase
  PK_UPD = 2,         // VecDesc (block = tile of the range)
  PK_PASS_D = 3,      // PassDesc<double, double, double>; arg = mode * 4 + ndot
  PK_PASS_F_IN = 4,   // PassDesc<float, double, float> (forward, first direction)
  PK_PASS_F_MID = 5,  // PassDesc<float, float, float>; arg = mode
  PK_PASS_F_OUT = 6   // PassDesc<float, float, double> (backward, first direction); arg = ndot
};

struct PRange {
  long long first;   // first ticket of the range
  int ntiles;        // items (tiles / blocks) in the range
  int kind;          // PersistKind
  int arg;
  int sys;           // index of the system's completion counter
  long long need;    // completed items of that system required before the range starts
  const void* desc;  // device address of the system's descriptor
  int desc_bytes;    // its size (copied to shared memory per item)
  int pad;
};

struct PQueue {
  unsigned long long head;  // next ticket
  int status;               // 0, or IFFD_ERR_TIMEOUT (8) when a bounded wait ran out
  int pad;
};

// Degrees the persistent launch carries (stiffness bodies instantiated).
constexpr int kPersistMinP = 2, kPersistMaxP = 8;

// Launches the persistent kernel over ranges[0..nranges) (total tickets
// `total`); done_cnt: one counter per system, zero at launch; q: zeroed.
// wait_limit bounds every wait (polls); smem: dynamic shared memory (the
// largest of the items'); grid: CTAs (at most the resident count).
cudaError_t launch_persistent(const PRange* ranges, int nranges, long long total, long long* done_cnt, PQueue* q,
                              long long wait_limit, double tol2, int maxit, size_t smem, int grid, cudaStream_t st);
// CTAs of the persistent kernel that fit on the GPU at once with smem bytes.
int persistent_grid(size_t smem);

}  // namespace iffd
