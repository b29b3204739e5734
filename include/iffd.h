/*
 * iffd.h -- C ABI of the GB300 (sm_103a) implementation of the Isogeometric
 * Fast Fourier-based Diagonalization (IFFD) preconditioner inside PCG for the
 * B-spline Galerkin Poisson system on [0,1]^d (arXiv 2512.20269).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Problem (Section 2): d in {2,3} directions, n elements per direction on a
 *   uniform grid, degree p, maximal smoothness C^{p-1}; on each end of each
 *   direction either homogeneous Dirichlet or natural (Neumann) conditions
 *   (the Dirichlet set D_k of direction k is any subset of {0,1}; at least one
 *   end of one direction must be Dirichlet, else A^ is singular). The basis of
 *   direction k has m_k = n_k + p - |D_k| functions; N = m_1 * ... * m_d.
 * - Vectors are float64 arrays of N entries in DEVICE memory, owned by the
 *   caller, contiguous, with direction 1 (x) fastest -- the lexicographic order
 *   of eq. "tp-B-basis": entry (i_1, .., i_d) sits at i_1 + m_1 (i_2 + m_2 i_3).
 * - The library owns only the plan (handle) and its device tables (a few
 *   hundred KB, plus 8 N bytes of eigenvalue reciprocals for FP64 IFFD plans).
 *   All large scratch memory is a caller-provided device buffer `ws` of at
 *   least iffd_workspace_bytes() bytes (256-byte aligned).
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Every call is asynchronous on that stream except iffd_setup (which
 *   synchronises it once after uploading the tables) and iffd_pcg_solve (which
 *   synchronises it to read the convergence state).
 * - Return value: an iffd_status. On error nothing is launched or the launch
 *   sequence stops at the failing launch; iffd_last_error() then returns a
 *   thread-local message. No exception crosses the ABI.
 * - The plan is bound to the CUDA device that was current at iffd_setup; every
 *   later call must run with that device current.
 */
#ifndef IFFD_H_
#define IFFD_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct iffd_plan* iffd_handle;

typedef enum {
  IFFD_OK = 0,
  IFFD_ERR_INVALID_ARG = 1,  /* null pointer, d not in {2,3}, p < 1, ... */
  IFFD_ERR_UNSUPPORTED = 2,  /* n <= p, p > 16, n too small for the edge blocks, size too large */
  IFFD_ERR_SINGULAR = 3,     /* all-Neumann problem: A^ singular (Section 3) */
  IFFD_ERR_WORKSPACE = 4,    /* ws is NULL or misaligned */
  IFFD_ERR_CUDA = 5,         /* a CUDA runtime call failed (message has the CUDA error) */
  IFFD_ERR_NOT_CONVERGED = 6,/* PCG reached maxit without the relative residual rtol */
  IFFD_ERR_BREAKDOWN = 7,    /* PCG breakdown: (p, A p) <= 0, (r, z) <= 0, or NaN/Inf */
  IFFD_ERR_TIMEOUT = 8       /* a bounded device wait expired (persistent engine launch) */
} iffd_status;

/* Arithmetic of the preconditioner transforms (the PCG vectors, residuals,
 * inner products and the stiffness apply are always float64). */
typedef enum {
  IFFD_PREC_FP64 = 0,           /* every transform step in float64 */
  IFFD_PREC_FP32_TRANSFORM = 1  /* transforms and eigenvalue scaling in float32 */
} iffd_precision;

typedef enum {
  IFFD_PRECOND_IFFD = 0,      /* eq. "preconditioner" with Q~, Lambda~ of Sections 4-6 */
  IFFD_PRECOND_EXACT_FD = 1,  /* eq. "exact_diagonalization" (dense Q per direction) */
  IFFD_PRECOND_NONE = 2       /* plain CG (z = r) */
} iffd_precond_kind;

typedef enum {
  IFFD_COEF_CONST = 0,        /* -Laplace: A = A^ = sum_k K_k x M x .. (eq. "system_matrix") */
  IFFD_COEF_SEPARABLE_SIN = 1 /* -div(a grad u), a = 1 + coef_amp prod_k sin(2 pi x_k), stiffness
                                 integrated with the tensor (p+1)-point Gauss rule (which factorises
                                 it exactly into A^ + coef_amp sum_k M^s x .. K^s_k .. x M^s);
                                 A != A^, the constant-coefficient IFFD stays the preconditioner, as
                                 for the geometry-mapped problems of Section 7 */
} iffd_coef_kind;

typedef struct {
  int precision;       /* iffd_precision */
  int precond;         /* iffd_precond_kind */
  double rtol;         /* stop when ||f - A u_k||_2 <= rtol ||f||_2 (recurrence residual); paper: 1e-8 */
  int maxit;           /* iteration cap */
  int coef;            /* iffd_coef_kind */
  int true_residual;   /* 1: iffd_pcg_solve recomputes ||f - A u||/||f|| at exit */
  int flexible;        /* 1: Polak-Ribiere beta (default for FP32 transforms) */
  double coef_amp;     /* amplitude c of IFFD_COEF_SEPARABLE_SIN (|c| < 1 keeps a > 0) */
  int autotune;        /* engine only: 1 tunes each (d, n, p) class at its first request (iffd_autotune) */
} iffd_options;

typedef struct {
  int iters;            /* number of products with A (Section 7 counts these) */
  double rel_res;       /* ||r_k|| / ||f|| of the recurrence residual at exit */
  double true_rel_res;  /* ||f - A u|| / ||f|| if options.true_residual, else -1 */
  int status;           /* iffd_status of the solve */
} iffd_pcg_info;

/* Fills *opt with the defaults: FP64, IFFD, rtol 1e-8, maxit 500, CONST,
 * true_residual 1, flexible 0, coef_amp 0.5, autotune 0. Returns
 * IFFD_ERR_INVALID_ARG on NULL. */
int iffd_default_options(iffd_options* opt);

/* Builds the plan for d directions with n_elems[k] elements each and degree p
 * (Section 2), computes on the host the 1D mass/stiffness matrices (Section 3),
 * the regular/remainder splitting and its eigendata (Sections 4-6: V_reg in the
 * special basis of eq. "special_basis", V_out, Q_out, Lambda_out, D~_reg,
 * Lambda_reg of Lemma 3) -- plus the dense Q_k of eq. "eigendecomposition" when
 * opt->precond == IFFD_PRECOND_EXACT_FD -- and uploads them to the current
 * device. FP64 IFFD plans also keep 1 / (sum of the eigenvalues of all
 * directions) for every DoF on the device (8 N bytes), so that the eigenvalue
 * scaling is a multiply. dirichlet[2k], dirichlet[2k+1] flag Dirichlet data
 * at x_k = 0 / 1 (0: natural condition); the transform of each direction
 * follows Table 1 for its (parity of p, D_k): DST-I / DST-II,III for
 * D_k = {0,1}, the six other cases through a zero-padded DFT of length 2n or
 * 4n. opt may be NULL (defaults). stream: see conventions.
 * Errors: INVALID_ARG, UNSUPPORTED (n <= p, p > 16, n too small for the edge
 * blocks of the special basis, transform too large for shared memory),
 * SINGULAR (no Dirichlet end at all), CUDA. *out is set only on success;
 * release it with iffd_destroy. */
int iffd_setup(int d, const int* n_elems, int p, const int* dirichlet, const iffd_options* opt, void* stream,
               iffd_handle* out);

/* iffd_setup with repeated interior knots (reduced regularity, Remark
 * "reduced_regularity" of Section 4). nrep[k] (k < d) is the number of
 * repeated breakpoints of direction k; reps lists them as (knot, extra) int
 * pairs, direction 0 first: the breakpoint knot/n_k (1 <= knot <= n_k - 1)
 * appears 1 + extra times in the knot vector (1 <= extra <= p - 1), so the
 * splines are C^{p-1-extra} there, and m_k = n_k + p + sum extra - |D_k|.
 * The regular space S^reg and its transform are those without repeated knots;
 * S^out grows by `extra` per repeated breakpoint (the jumps of the derivatives
 * of orders p - extra .. p - 1). V_reg gets a small dense block around every
 * repeated breakpoint, and the stiffness sweeps of such a direction use
 * general band rows throughout. nrep NULL: no repeated knots (iffd_setup).
 * Host arrays, read during the call only. Errors: as iffd_setup, plus
 * INVALID_ARG (negative count, reps NULL with a positive count) and
 * UNSUPPORTED (knot or extra out of range, a knot listed twice, a repeated
 * breakpoint too close to an end for the edge blocks, n_out above 16). */
int iffd_setup_knots(int d, const int* n_elems, int p, const int* dirichlet, const int* nrep, const int* reps,
                     const iffd_options* opt, void* stream, iffd_handle* out);

/* Device workspace needed by every call on this plan, in bytes. */
int iffd_workspace_bytes(iffd_handle h, size_t* bytes);

/* Tunes the launch geometry of the plan on this GPU (the paper has no
 * counterpart; it fixes no kernel design): for every direction, the pencils
 * per tile (2..32, within 200 KB of shared memory) and the radix sequence of
 * the FFT (greedy radix 8, radix 4, or the greedy sequence reversed) of the
 * transform pass, whether the pass runs as a persistent kernel that loads its
 * next tile asynchronously (where the pass reads its own arithmetic type) or,
 * for FP32 transforms where it applies, as the warp-FFT pass, and the pencils
 * per tile of the stiffness sweep. Each
 * candidate runs the plan's kernel on the workspace ws (iffd_workspace_bytes,
 * contents overwritten) on `stream`; the fastest of three timed launches wins.
 * Passes whose default launch has fewer than 4 x 152 CTAs (too small to fill
 * the GPU alone) keep the default geometry.
 * Choices are cached per size class for the life of the process, so plans of
 * the same class get the same geometry (and bitwise the same results) without
 * timing again. Synchronizes the stream. Results of a tuned plan equal those
 * of the untuned plan to rounding: tiles change the order of the partial
 * sums of the dot products, and the radix sequence changes FFT rounding.
 * Errors: INVALID_ARG, WORKSPACE (ws NULL or not 256-byte aligned), CUDA. */
int iffd_autotune(iffd_handle h, void* ws, void* stream);

/* Sets the launch geometry of direction `axis` by hand (the tuner's choices,
 * see iffd_autotune): pencils per tile of its transform pass and of its
 * stiffness sweep (2, 4, 8, 16 or 32; <= 0 keeps the current value) and the
 * schedule of its transform passes: `pipelined` 1 = persistent pipelined
 * kernel, 0 = one tile per CTA, 2 = the warp-FFT pass (D = {0,1} directions
 * whose FFT length is 64, 128, 256 or 512, FP64 plans up to 256: DST-II/III
 * with n_reg of that length, DST-I with 2 (n_reg + 1); each pencil pair is
 * transformed by the lanes of one warp, register butterflies, fixed tile;
 * opt-in for FP64 plans), 3 = double-float transforms for the whole plan
 * (FP64 IFFD plans whose every direction has a warp-FFT pass of length 64,
 * 128 or 256 or a transform run without Bluestein's convolution: the
 * warp-FFT pass or the block kernel in FP64-accurate arithmetic on pairs of
 * FP32 values; their default where the passes' tiles fill the GPU),
 * 4 = the paired FP32 warp-FFT pass (FFT length 64, 128 or 256:
 * every lane group carries two sequences, four pencils, at once; each
 * pencil's values are bitwise those of pipelined 2, and so are the partial
 * sums of the fused dot products; the default for the last direction of
 * FP32 plans when it qualifies), < 0 unchanged. Setting a tile size or pipelined 0/1 selects the block
 * kernel. The block-kernel geometry does not change any transformed value; it
 * changes the grouping of the partial sums of the dot products (the warp-FFT
 * pass rounds differently, within the FP32 or FP64 tolerance). The batched
 * engine runs FP64 systems on the block kernel. Errors: INVALID_ARG,
 * UNSUPPORTED (does not fit in 200 KB of shared memory; warp-FFT pass not
 * available for this direction). Do not call while work of the plan is in
 * flight. */
int iffd_set_geometry(iffd_handle h, int axis, int pencils_transform, int pencils_stiffness, int pipelined);

/* Launch geometry of direction `axis` (any pointer may be NULL): pencils per
 * tile of its transform pass (for the plan's precision) and of its stiffness
 * sweep, the radix sequence of its FFT (radices[0..*nstages), at most 12),
 * and the schedule of its transform passes (*pipelined = 1: persistent
 * pipelined kernel, each CTA loads its next tile asynchronously while it
 * transforms the current one; 2: warp-FFT pass; 3: double-float warp-FFT
 * pass; 4: paired FP32 warp-FFT pass; 5: double-float block kernel (the
 * reported tile and radices); 0: one tile per CTA). */
int iffd_get_tiles(iffd_handle h, int axis, int* pencils_transform, int* pencils_stiffness, int* radices,
                   int* nstages, int* pipelined);

/* Sizes of direction `axis` (0-based): m = n + p - |D| (plus the extra
 * multiplicities of repeated knots), n_reg and n_out of eq. "reg_space_dim". */
int iffd_get_dims(iffd_handle h, int axis, int* m, int* n_reg, int* n_out);

/* Copies the host-side 1D data of direction `axis` into caller HOST buffers
 * (any pointer may be NULL):
 *   M_band, K_band: m*(2p+1), band[i*(2p+1) + (j-i+p)] = M[i][j] (Section 3);
 *   lam: m, Lambda~ = [Lambda_reg (Lemma 3) | Lambda_out];
 *   dtilde: n_reg, diagonal of D~_reg (end of Section 6);
 *   Vreg: m*n_reg, V_reg in the special basis of Section 6 (row-major, dense):
 *       column j is special function j on the B-spline basis of S_{p,h,D};
 *   W: m*n_out, V_out Q_out (row-major). */
int iffd_get_1d(iffd_handle h, int axis, double* M_band, double* K_band, double* lam, double* dtilde,
                double* Vreg, double* W);

/* Host-only variant of iffd_get_1d that needs no plan and no GPU: runs the
 * same 1D setup for n elements, degree p and the Dirichlet flags
 * dirichlet[0..1] of one direction. m, n_reg, n_out receive the sizes (any may
 * be NULL); every array pointer may be NULL (call once with NULLs to size the
 * buffers). Same layouts and errors as iffd_get_1d / iffd_setup. */
int iffd_host_axis(int n, int p, const int* dirichlet, int* m, int* n_reg, int* n_out, double* M_band,
                   double* K_band, double* lam, double* dtilde, double* Vreg, double* W);

/* iffd_host_axis with nrep repeated interior breakpoints, listed as
 * (knot, extra) int pairs in reps (see iffd_setup_knots). Needs no GPU. */
int iffd_host_axis_knots(int n, int p, const int* dirichlet, int nrep, const int* reps, int* m, int* n_reg,
                         int* n_out, double* M_band, double* K_band, double* lam, double* dtilde, double* Vreg,
                         double* W);

/* Host-only: how the preconditioner passes of one direction carry its DST
 * (Table 1: DST-I for odd p, DST-II/III for even p, D = {0,1}) for the given
 * precision (IFFD_PREC_FP64 or IFFD_PREC_FP32_TRANSFORM). *L receives the
 * length of the complex DFT (two pencils per sequence: n_reg for DST-II/III,
 * 2 (n_reg + 1) for DST-I); *F the length of the FFT that runs: F == L for the
 * direct mixed-radix FFT, F > L (5-smooth, F >= 2L - 1) when the DFT runs as
 * Bluestein's chirp convolution because L has large prime factors; *pencils
 * (may be NULL) the pencils per tile. Same errors as iffd_setup. Needs no GPU. */
int iffd_host_transform(int n, int p, const int* dirichlet, int precision, int* L, int* F, int* pencils);

/* z = P^{-1} r: the IFFD preconditioner of eq. "preconditioner" (or the exact
 * FD of eq. "exact_diagonalization", or the identity, per opt->precond).
 * r, z: device, N float64 each, must not alias. ws: see conventions. */
int iffd_apply_preconditioner(iffd_handle h, const double* r, double* z, void* ws, void* stream);

/* Au = A u: A^ u with A^ = sum_k (M_d x .. x K_k x .. x M_1) (eq.
 * "system_matrix") for IFFD_COEF_CONST, or the variable-coefficient operator of
 * IFFD_COEF_SEPARABLE_SIN, applied matrix-free by banded sweeps. u, Au: device,
 * N float64 each, must not alias. */
int iffd_apply_stiffness(iffd_handle h, const double* u, double* Au, void* ws, void* stream);

/* Allocation-free variant of iffd_apply_stiffness (the paper has no
 * counterpart). It exists for callers that cannot allocate device memory at
 * the point where they need A^ u: a host framework whose caching allocator
 * owns all device memory and allows no side allocations, an embedded solver
 * with a device-memory budget fixed at start-up, or a latency-critical loop
 * that must not pay the implicit device synchronisation of cudaMalloc.
 * Same result as iffd_apply_stiffness(h, u, Au, ws, stream) for plans with
 * IFFD_COEF_CONST (other plans are rejected with IFFD_ERR_UNSUPPORTED), without a
 * workspace: the two N-vector temporaries live in a static device array of
 * 2 * IFFD_NOALLOC_MAX_DOFS doubles (16 MiB) inside the library, which every
 * GPU that loads the library's module holds until the process exits. The call
 * itself allocates nothing (no cudaMalloc / cudaFree).
 * - The checks run in the order of iffd_apply_stiffness (arguments, plan
 *   device, coefficient kind), then the size limit: plans with
 *   N > IFFD_NOALLOC_MAX_DOFS are rejected with IFFD_ERR_UNSUPPORTED and a
 *   message naming the limit.
 * - The first call on each device resolves the array's device address
 *   (cudaGetSymbolAddress, with that device current) and caches it with the
 *   CUDA context it belongs to; make that first call before any stream
 *   capture. A call that finds a different context current on the device
 *   (after cudaDeviceReset) resolves the address again.
 * - Every call shares the one array, so calls that overlap on the GPU (other
 *   streams, other plans, other host threads) race: order them on one stream
 *   or synchronise between them. The array keeps the last call's contents;
 *   nothing in it needs to start at zero.
 * u, Au: device, N float64 each, must not alias. */
#define IFFD_NOALLOC_MAX_DOFS (1 << 20)
int iffd_apply_stiffness_noalloc(iffd_handle h, const double* u, double* Au, void* stream);

/* Solves A u = f (A as in iffd_apply_stiffness) by PCG (Section 3) with zero initial guess and the stopping
 * rule ||r_k|| <= rtol ||f|| (Section 7), preconditioned per opt->precond.
 * f, u: device, N float64 each, must not alias; u is output only. info: HOST
 * pointer, filled on return (may be NULL). Synchronises `stream`. Returns
 * IFFD_OK, IFFD_ERR_NOT_CONVERGED or IFFD_ERR_BREAKDOWN (u then holds the last
 * iterate), or an argument / CUDA error.
 * All PCG scalars stay on the device; the host enqueues the iterations in
 * chunks and reads the solve state after each chunk (iterations enqueued past
 * convergence return at once). The first chunk is as long as the plan's last
 * converged solve, later chunks 4 iterations. A solve that repeats one of the
 * plan's two previous (f, u, ws) triples replays its chunks from CUDA graphs
 * captured on a private stream (bitwise the same kernels; not while per-launch
 * event timing is on). */
int iffd_pcg_solve(iffd_handle h, const double* f, double* u, void* ws, void* stream, iffd_pcg_info* info);

/* ---- General coefficient (stiffness of -div(C(x) grad u), A != A^) ----
 * Section 2's Galerkin form with a symmetric coefficient C(x) under the
 * integral, A_ij = int grad B_i . C grad B_j dx, integrated with the tensor
 * (p+1)-point Gauss rule of every element. A geometry map F of Section 7,
 * pulled back to the parameter domain, has this form with C = det(DF) DF^-1
 * DF^-T. The preconditioner stays the plan's IFFD (that of A^). */

/* Gauss points and weights of direction `axis` on [0, 1]: *nq = n (p + 1)
 * (element e owns points e (p+1) .. e (p+1) + p, increasing). x and w are
 * caller-owned host arrays of *nq entries, or NULL. Host only. Errors:
 * INVALID_ARG. */
int iffd_quad_points(iffd_handle h, int axis, int* nq, double* x, double* w);

/* Host only, no plan: the Gauss points x and weights w (nq = n (p+1)
 * entries) of one direction, and the dense nq x m row-major matrices B
 * (values) and D (first derivatives) of its kept B-splines there, expanded
 * from the sparse tables the device passes use (which are also checked
 * against their transposes). Arguments as iffd_host_axis_knots; any output
 * may be NULL (query nq and m first). Errors: INVALID_ARG, UNSUPPORTED. */
int iffd_host_quad_axis(int n, int p, const int* dirichlet, int nrep, const int* reps, int* nq, int* m, double* x,
                        double* w, double* B, double* D);

/* Bytes of the scratch workspace of the general-coefficient operator: 3D,
 * two arrays of nq_0 m_1 m_2 doubles and six of nq_0 nq_1 m_2 (about
 * 6 (p+1)^2 times the DoF count in doubles); 2D, four of nq_0 m_1. Values at
 * all Gauss points are never stored. Errors: INVALID_ARG. */
int iffd_general_workspace_bytes(iffd_handle h, size_t* bytes);

/* Au = A_C u on the device. C: device array of ncomp * nq_0 nq_1 (nq_2)
 * doubles at the tensor Gauss points (nq_k from iffd_quad_points, direction 0
 * fastest), component by component: ncomp = 1 is a scalar a(x) (C = a I);
 * ncomp = d (d + 1) / 2 is the upper triangle of the symmetric C row by row,
 * (C11, C12, C22) in 2D and (C11, C12, C13, C22, C23, C33) in 3D. u, Au:
 * device arrays of the plan's shape; they may not alias. gws: device scratch
 * of iffd_general_workspace_bytes, 256-byte aligned, caller-owned. Stream-
 * ordered, asynchronous. Errors: INVALID_ARG (NULL, aliasing, ncomp),
 * WORKSPACE, UNSUPPORTED (p > 11), CUDA. */
int iffd_apply_stiffness_general(iffd_handle h, const double* C, int ncomp, const double* u, double* Au, void* gws,
                                 void* stream);

/* PCG on A_C u = f (zero start) with the plan's preconditioner, the loop of
 * iffd_pcg_solve (same options, stopping rule, info and return values) with
 * A_C in place of A^. ws: the plan's workspace; gws: as above. Where the
 * eigenvalues of C lie in [c_lo, c_hi], c_lo A^ <= A_C <= c_hi A^, so the
 * condition number is at most c_hi / c_lo times that with A^. */
int iffd_pcg_solve_general(iffd_handle h, const double* C, int ncomp, const double* f, double* u, void* ws, void* gws,
                           void* stream, iffd_pcg_info* info);

/* Kernel kinds reported by the profiler (iffd_profile_read). */
typedef enum {
  IFFD_K_PRECOND_FWD = 0,    /* IFFD pass Q~^T along one direction */
  IFFD_K_PRECOND_FUSED = 1,  /* IFFD pass Q~^T, eigenvalue scaling, Q~ (last direction) */
  IFFD_K_PRECOND_BWD = 2,    /* IFFD pass Q~ along one direction (+ PCG dot products) */
  IFFD_K_STIFF_FIRST = 3,    /* stiffness sweep, slowest direction (+ p = z + beta p) */
  IFFD_K_STIFF_MID = 4,      /* stiffness sweep, middle direction (3D) */
  IFFD_K_STIFF_LAST = 5,     /* stiffness sweep along x (+ (p, A p) partial sums) */
  IFFD_K_PCG_UPDATE = 6,     /* x += alpha p, r -= alpha q, ||r||^2 partials */
  IFFD_K_PCG_INIT = 7,       /* x = 0, r = f, ||f||^2 partials */
  IFFD_K_FINALIZE = 8,       /* fixed-order reduction of partial sums + scalar updates */
  IFFD_K_FD_PASS = 9,        /* exact FD dense contraction pass */
  IFFD_K_VECTOR = 10,        /* copies, plain dot products, residual norm */
  IFFD_K_GENERAL = 11,       /* general-coefficient stiffness: sweeps, Gauss-point step, p-update */
  IFFD_K_KINDS = 12
} iffd_kernel_kind;

/* Per-kernel device timing of this plan's launches by CUDA events recorded on
 * the call's stream around every launch (off by default; costs one event pair
 * per launch). iffd_profile_enable(h, 1) starts recording, 0 stops;
 * iffd_profile_reset clears the totals. iffd_profile_read waits for the
 * recorded events and returns, for one iffd_kernel_kind, the number of
 * launches and their summed device time in milliseconds since the last reset
 * (name: static string, may be NULL). iffd_launch_count returns the number of
 * kernels this plan has launched since iffd_setup (always counted). */
int iffd_profile_enable(iffd_handle h, int enable);
int iffd_profile_reset(iffd_handle h);
int iffd_profile_read(iffd_handle h, int kind, long long* launches, double* ms, const char** name);
int iffd_launch_count(iffd_handle h, long long* count);

/* Releases the plan and its device tables (NULL is accepted). Must run with
 * the plan's device current; does not synchronise any stream. */
int iffd_destroy(iffd_handle h);

/* ---------------------------------------------------------------------------
 * Batched solves / continuous batching (many independent problems; the paper
 * solves one problem at a time and has no counterpart).
 * An engine owns a device arena of `budget_bytes` from which every admitted
 * request takes its workspace (iffd_engine_request_bytes). Each step
 * initialises the requests admitted since the previous step and advances every
 * active request by `iterations` PCG iterations; all active requests share the
 * launches of each phase (one batched launch per phase, the stiffness sweeps
 * grouped by degree), the per-iteration launch sequence is a CUDA graph that is
 * replayed while the set of requests is unchanged. After the step the finished
 * requests are retired (their workspace returns to the arena) and can be
 * collected with iffd_engine_poll. A request's kernels, tile decomposition and
 * reduction order are those of iffd_pcg_solve with the same options, so its
 * result does not depend on the other requests in the engine.
 * Only IFFD-preconditioned, constant-coefficient, Dirichlet cube/square
 * problems (d, n elements per direction, degree p) are served. */
typedef struct iffd_engine* iffd_engine_handle;

typedef struct {
  long long id;        /* request id returned by iffd_engine_submit */
  iffd_pcg_info info;  /* true_rel_res is -1 (not computed by the engine) */
} iffd_completion;

/* opt: precision, rtol, maxit, flexible and autotune are used (NULL =
 * defaults); with autotune, the plan of each (d, n, p) is tuned by
 * iffd_autotune at the first submit of that class. The arena
 * is allocated here (cudaMalloc of budget_bytes on the current device). The
 * engine runs on a stream of its own; every step first waits for the work
 * already enqueued on `stream` (so f may be produced there) and returns after
 * the step's work has finished. */
int iffd_engine_create(const iffd_options* opt, size_t budget_bytes, void* stream, iffd_engine_handle* out);
/* Workspace a request (d, n, p, dirichlet as in iffd_engine_submit) takes from
 * the arena (builds and caches the plan of the class if needed). */
int iffd_engine_request_bytes(iffd_engine_handle e, int d, int n, int p, const int* dirichlet, size_t* bytes);
/* Admits a request if its workspace fits the arena now: d directions with n
 * elements each, degree p, dirichlet[2k], dirichlet[2k+1] the Dirichlet flags
 * of direction k as in iffd_setup (NULL: Dirichlet on every face); f
 * (right-hand side) and u (solution, output) are caller-owned device arrays
 * of N float64 that must stay valid until the request completes. Returns
 * IFFD_ERR_WORKSPACE if the arena has no room now (resubmit after
 * completions) and IFFD_ERR_UNSUPPORTED if the request can never fit. */
int iffd_engine_submit(iffd_engine_handle e, int d, int n, int p, const int* dirichlet, const double* f, double* u,
                       long long* id);
/* One step (see above); *active receives the number of requests still
 * iterating. Synchronises the engine's stream once (to read the states). */
int iffd_engine_step(iffd_engine_handle e, int iterations, int* active);
/* Moves up to `capacity` completions into out; *count receives how many. */
int iffd_engine_poll(iffd_engine_handle e, iffd_completion* out, int capacity, int* count);
/* Active requests, free arena bytes, kernels launched so far (any may be NULL). */
int iffd_engine_stats(iffd_engine_handle e, int* active, size_t* bytes_free, long long* kernel_launches);
/* Launch mode of the engine's iterations (only while no request is active).
 * on = 1: every iffd_engine_step runs its `iterations` PCG iterations of all
 * active requests as ONE persistent kernel launch that walks a device work
 * queue of (request, phase, tile) items: CTAs take items in ticket order; an
 * item starts once its request has completed every earlier item (a
 * per-request counter); the device bodies, tiles and reduction orders are
 * those of the per-phase kernels, so each result is bitwise that of
 * iffd_pcg_solve with the same kernels (transform passes: the block kernel --
 * the engine's plans then run no warp-FFT pass; degrees 2..8). Every wait is
 * bounded by wait_limit polls of ~64 ns (<= 0: 2^26); a wait that runs out
 * makes the step return IFFD_ERR_TIMEOUT (that step's results are not valid)
 * instead of hanging. inject_stall = 1 is a test hook that makes one item
 * wait on a count that is never reached (so the timeout path runs).
 * on = 0: one captured graph of batched launches per iteration (default). */
int iffd_engine_set_persistent(iffd_engine_handle e, int on, long long wait_limit, int inject_stall);
int iffd_engine_destroy(iffd_engine_handle e);

/* ---------------------------------------------------------------------------
 * Batched solve of many systems in one call: PCG of Section 3 with the IFFD
 * preconditioner of eq. "preconditioner" (or the plan's own preconditioner),
 * for `count` plans, plan i with nrhs[i] right-hand sides. System (i, j),
 * j < nrhs[i], solves A_i u = f with f = f[i] + j N_i and writes u[i] + j N_i
 * (N_i the plan's DoF count): f[i] and u[i] are caller-owned DEVICE arrays of
 * nrhs[i] * N_i float64, right-hand side after right-hand side, x fastest
 * within each; u is output only (zero start). The right-hand sides of one plan
 * share that plan's device tables (no copy per right-hand side).
 * ws: caller-owned device workspace of iffd_batch_workspace_bytes() bytes,
 * 256-byte aligned (one plan workspace per system, in (i, j) order).
 * infos: HOST array of sum_i nrhs[i] entries, filled in (i, j) order (iters,
 * rel_res, status; true_rel_res when the plan's options ask for it, else -1).
 * Systems of IFFD-preconditioned constant-coefficient plans advance together
 * through the batched launches of the engine (below), one set of launches per
 * phase for all of them, grouped by the plans' solve options; the kernels,
 * tiles and reduction order of each system are those of iffd_pcg_solve on its
 * plan, so every u equals (bitwise) iffd_pcg_solve's on the same plan. Other
 * plans (exact FD, variable coefficient, FP64 warp-FFT geometry) are solved by
 * iffd_pcg_solve one after the other on their slice of ws. Waits for the work
 * already on `stream` and returns after every system has finished (the
 * batched part runs on library streams; it allocates small descriptor
 * buffers and a CUDA graph). Returns IFFD_OK if every system converged, else
 * the status of the first system (in (i, j) order) that did not (every info is
 * still filled), or an argument / workspace / CUDA error (INVALID_ARG: NULL or
 * aliasing arrays, negative counts, a plan of another device). The paper
 * solves one system at a time and has no batched counterpart. */
int iffd_batch_workspace_bytes(int count, const iffd_handle* plans, const int* nrhs, size_t* bytes);
int iffd_batch_solve(int count, const iffd_handle* plans, const double* const* f, double* const* u, const int* nrhs,
                     void* ws, void* stream, iffd_pcg_info* infos);

/* ---------------------------------------------------------------------------
 * Building blocks of the slab-decomposed solve of ONE problem over several
 * GPUs (one process per GPU; the Python module slab.py exchanges the data
 * between the ranks and sums the inner products). A rank holds a box of the
 * global grid of plan h: its slab of rows [z0, z0 + nz) of the slowest
 * direction, or, for the fused pass, a box with whole pencils along the
 * slowest direction. Boxes are float64 device arrays, direction 0 fastest;
 * box[k] / offset[k] give the extent and the global offset per direction
 * (direction 0 first; d entries, or 3 with trailing 1 / 0).
 *
 * iffd_apply_pass: one transform pass of the preconditioner of eq.
 * "preconditioner" along `axis` on a box holding whole pencils along it
 * (box[axis] = m_axis, offset[axis] = 0): mode 0 applies Q~^T, 1 applies Q~,
 * 2 (axis = d - 1 only) Q~^T, the division by the summed eigenvalues of all
 * directions (the box offset selects the eigenvalues of the other directions)
 * and Q~. in and out may alias. FP64 IFFD plans (FP64-pipe block kernel).
 * Errors: INVALID_ARG (box outside the grid, partial pencils, bad axis or
 * mode), UNSUPPORTED (other precisions or preconditioners), CUDA.
 *
 * iffd_slab_stiffness: Au = A^ u (eq. "system_matrix") on the rows
 * [z0, z0 + nz) of the slowest direction. u_ext holds u on the rows
 * [max(0, z0 - p), min(m, z0 + nz + p)) (the slab and its halo from the
 * neighbouring ranks), Au the nz rows; ws: device scratch of
 * iffd_slab_workspace_bytes(h, nz) bytes, 256-byte aligned. The sweep along
 * the slowest direction takes the global band rows of M and K; the sweeps
 * along the other directions are those of iffd_apply_stiffness. IFFD_COEF_CONST
 * plans. Errors: INVALID_ARG, WORKSPACE, UNSUPPORTED, CUDA.
 *
 * iffd_copy_box: dst box <- src box, both 3D arrays (dims, direction 0
 * fastest), boxes of extent ext at offsets src_off / dst_off (the packing of
 * the exchanges). Errors: INVALID_ARG (box outside an array), CUDA.
 *
 * iffd_vec_dot: *result (device) = (a, b) over n entries, a fixed reduction
 * order (per-block partial sums, then one block adds them in order); ws:
 * device scratch of iffd_vec_dot_workspace_bytes(). iffd_vec_axpby:
 * y = a x + b y (the PCG updates of Section 3 on a rank's part). */
int iffd_apply_pass(iffd_handle h, int axis, int mode, const int* box, const int* offset, const double* in,
                    double* out, void* stream);
int iffd_slab_workspace_bytes(iffd_handle h, int nz, size_t* bytes);
int iffd_slab_stiffness(iffd_handle h, int z0, int nz, const double* u_ext, double* Au, void* ws, void* stream);
int iffd_copy_box(const double* src, const int* src_dims, const int* src_off, double* dst, const int* dst_dims,
                  const int* dst_off, const int* ext, void* stream);
int iffd_vec_dot_workspace_bytes(size_t* bytes);
int iffd_vec_dot(const double* a, const double* b, long long n, double* result, void* ws, void* stream);
int iffd_vec_axpby(long long n, double a, const double* x, double b, double* y, void* stream);

/* Measures the arithmetic rate of the current GPU for the roofline of the
 * compute-bound kernels (the paper prints no timings and has no counterpart):
 * kind 0 = FP64 fused multiply-add, kind 1 = FP32 fused multiply-add, kind 2 =
 * packed FP32 pairs (fma.rn.f32x2: two FMAs per instruction). Every
 * thread of a grid of 4 CTAs x 256 threads per SM runs eight independent FMA
 * chains; *tflops receives 2 x FMAs / the best of three CUDA-event times
 * (~40 ms each) in TFLOP/s, *sm_count (may be NULL) the SM count read from the
 * device. Runs on `stream` and synchronises it; allocates and frees a few KB.
 * Errors: INVALID_ARG (kind not in 0..2, NULL tflops), CUDA. */
int iffd_measure_peak(int kind, void* stream, int* sm_count, double* tflops);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* iffd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* IFFD_H_ */
