/*
 * heat3d.h -- C ABI of libheat3d.so: a GB300 (sm_103a) solver for the forced
 * 3-D heat equation  u_t = nu Delta u + f  on [0,1]^3 with u = 0 on the
 * boundary (arXiv:1307.7867, Sec. 1, Eqs. 1-4), integrated in time by SDC,
 * two-level MLSDC and PFASST (Sec. 1.1) with multigrid solves of the
 * implicit-Euler substeps (Sec. 1.2).
 *
 * Conventions shared by every call:
 *  - Grid functions crossing this boundary are DENSE arrays of the N^3
 *    interior values, FP64, index ((k * N) + j) * N + i (x fastest, z
 *    slowest), with x_i = (i + 1) h, h = 1 / (N + 1), zero Dirichlet values
 *    on the boundary.  Inside the library fields are stored pitched.
 *  - Pointers documented as "device" must point to device memory of the
 *    context's device; "host or device" pointers are classified with
 *    cudaPointerGetAttributes (pageable or pinned host memory both work).
 *  - The caller owns every buffer it passes; the library never frees one.
 *    Device memory for resident state comes from ONE workspace the caller
 *    allocates (heat3d_workspace_size) and binds (heat3d_bind_workspace);
 *    the library allocates no device memory of its own.
 *  - Return codes: HEAT3D_OK (0) or a negative HEAT3D_E* code; a context
 *    keeps a message for the last failure (heat3d_last_error).
 *  - Work is enqueued on the context's CUDA stream.  Calls that read a
 *    convergence norm synchronise that stream; pfasst_run and heat3d_wait
 *    return with their results complete.  One host thread per context.
 */
#ifndef HEAT3D_H
#define HEAT3D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HEAT3D_OK 0
#define HEAT3D_EINVAL (-1)    /* bad argument or configuration */
#define HEAT3D_ENOMEM (-2)    /* workspace too small, or a request refused admission */
#define HEAT3D_ENOTCONV (-3)  /* a solve hit its V-cycle cap above its tolerance */
#define HEAT3D_ENAN (-4)      /* a residual norm was NaN or Inf */
#define HEAT3D_ETIMEOUT (-5)  /* a bounded device-side wait gave up */
#define HEAT3D_ECUDA (-6)     /* a CUDA runtime call failed */
#define HEAT3D_ESTATE (-7)    /* call made in the wrong state (e.g. no workspace bound) */

#define HEAT3D_FP64 0   /* every field and every smoother in FP64 */
#define HEAT3D_MIXED 1  /* FP32 V-cycles inside FP64 residual refinement */

#define HEAT3D_FORCING_NONE 0          /* f = 0 */
#define HEAT3D_FORCING_PAPER_LITERAL 1 /* Eq. 3 as printed: f = -Phi (sin t - nu pi^2 cos t) */
#define HEAT3D_FORCING_EXACT 2         /* f = -Phi (sin t - 3 nu pi^2 cos t): u = Phi cos t solves it */

#define HEAT3D_MAX_NODES 5

/* Stencil code (heat3d_level.order) of the fourth-order compact 19-point
 * (Mehrstellen) discretisation, the paper's fine-level stencil (Sec. 1):
 * W u' = nu L u + W f with L = (1/(6h^2)) (-24 u + 2 * faces + edges) and the
 * weighting matrix W = (6 u + faces) / 12.  SDC runs in this weighted form
 * (its collocation residual is the weighted one) and the FAS restriction
 * applies W^{-1} by multigrid (Sec. 1.2).  Fine level only. */
#define HEAT3D_COMPACT 19

/* One level of the space-time hierarchy (Sec. 1: PFASST coarsens nodes, mesh
 * and stencil order). */
typedef struct {
  int N;     /* interior points per axis; must be 2^k - 1 (multigrid halving), <= 1023 */
  int order; /* 2: 7-point Laplacian; 4: 13-point wide Laplacian (odd-reflection ghosts);
                HEAT3D_COMPACT: 19-point compact stencil (level 0 only) */
  int M;     /* Gauss-Lobatto nodes per step, both ends included, 2..5 */
} heat3d_level;

/* Multigrid settings for every implicit solve (Sec. 1.2). */
typedef struct {
  int nu1, nu2;   /* damped-Jacobi pre- and post-smoothing sweeps (V(2,1)) */
  int max_cycles; /* cap per solve, counted in refinement steps */
  double tol;     /* stop when max|b - A u| <= tol; tol < 0: exactly max_cycles cycles */
  int inner;      /* V-cycles per refinement step (per FP64 residual), >= 1; the
                     tolerance is checked after each step.  0 with HEAT3D_MIXED: chosen
                     per step (1-4) from the residuals seen so far and the contraction
                     per V-cycle of the previous step, with graph replay (use_graphs)
                     and tol >= 0; 3 on the other paths */
  double rel;     /* > 0 (with tol >= 0): inside an SDC sweep, item b's solves stop at
                     max(tol, rel * r_b), r_b = the collocation residual of the sweep's
                     incoming iterate (the paper leaves the solver tolerance open);
                     0: the fixed tol */
} heat3d_mg;

typedef struct {
  double nu;                /* diffusion coefficient */
  double T;                 /* end time of pfasst_run */
  double dt;                /* step (time slice) length */
  int nlevels;              /* 1: single-level SDC; 2: MLSDC (slices = 1) or PFASST */
  heat3d_level levels[2];   /* [0] fine, [1] coarse (N_f = 2 N_c + 1 or equal; nested nodes) */
  int sweeps_fine;          /* fine sweeps per iteration (nlevels = 1: sweeps per step) */
  int sweeps_coarse;        /* coarse sweeps per iteration and in the predictor */
  int slices;               /* PFASST time slices iterated together (1 = serial) */
  int iters;                /* MLSDC/PFASST iterations per block (cap when tol_sdc >= 0) */
  double tol_sdc;           /* stop when the fine collocation residual <= tol_sdc; < 0: fixed */
  int predictor;            /* 1: serial coarse predictor before the first iteration */
  heat3d_mg mg;
  int precision;            /* HEAT3D_FP64 or HEAT3D_MIXED */
  int forcing;              /* HEAT3D_FORCING_* */
  int batch;                /* state slots per level for sdc_sweep / serving (>= slices) */
  int device;               /* CUDA device ordinal */
  void* stream;             /* cudaStream_t for all work of this context (NULL: legacy) */
  int use_graphs;           /* 1: replay the solve cycles from captured CUDA graphs, with the
                               stop rule on the device and one host wait per chunk of cycles
                               (4 on grids below 127, else 1); same cycles and results as
                               without (needs a non-default stream; ignored on the legacy
                               stream) */
  int autotune;             /* 1: time the stencil launch shapes of every multigrid level at
                               heat3d_bind_workspace and keep the fastest (results identical).
                               The environment variable HEAT3D_SHAPE="kind,zc" (kind 1-26,
                               planes per block zc, or -1 / -2 for the chunk that fills one /
                               two waves of the GPU) forces one shape on every stencil of
                               grids with N >= 16 instead (testing); HEAT3D_TUNE_FILE=path
                               reuses the shapes recorded in that file for levels it lists
                               and appends the timed choices of the others */
  int fuse_coarse;          /* 1: run the coarse multigrid levels of a V-cycle in one kernel,
                               all levels in shared memory (results identical): the levels
                               with N <= 15, or N <= 7 or 3 when the autotuner times that
                               faster (the environment variable HEAT3D_FUSE_MAX=n forces n,
                               for testing) */
  int interp;               /* spatial interpolation of the coarse correction in the FAS
                               step (Sec. 1.1; the paper does not say which): 2 trilinear
                               (default); 4, 6, 8 the tensor-product 4-point (cubic),
                               6- or 8-point Lagrange midpoint rule on the odd extension
                               about the zero boundary.  With spatial coarsening the higher
                               orders cut the MLSDC / PFASST iterations several-fold */
  int persistent;           /* multigrid solves as one persistent cooperative kernel each
                               (residual, all V-cycles and the stop rule in one launch, grid
                               barriers between the steps; bitwise the results of the launch
                               sequence): -1 (default) on levels with 15 <= N <= 31, 1 on
                               levels with 15 <= N <= 63, 0 never.  Orders 2 and 4 only (the
                               compact stencil's levels use the launch sequence).  A grid
                               barrier that waits about 1 s gives up: HEAT3D_ETIMEOUT */
} heat3d_config;

typedef struct {
  long long vcycles;   /* V-cycles (refinement steps) over all solves */
  long long solves;    /* implicit solves */
  long long sweeps;    /* SDC sweeps on any level (a batched sweep counts once) */
  long long iters;     /* MLSDC / PFASST iterations */
  long long steps;     /* time steps completed (slices count one each) */
  int notconv;         /* solves that stopped at the cycle cap above tolerance */
  double residual;     /* last fine-level collocation residual computed (max over items) */
  double mg_residual;  /* last multigrid residual max|b - A u| */
  double seconds;      /* device time of the call, from CUDA events on the stream */
  double bytes;        /* algorithmic HBM bytes of the call's kernels (a counter) */
  long long vcycles_level[2]; /* V-cycles of solves on SDC level 0 (fine) and 1 (coarse) */
} heat3d_stats;

typedef struct heat3d_ctx heat3d_ctx;

/* Fills a config with the paper's fine/coarse hierarchy at N = 31/15 and V(2,1). */
void heat3d_config_default(heat3d_config* cfg);

/* Bytes of device workspace a context with this config needs. */
int heat3d_workspace_size(const heat3d_config* cfg, size_t* bytes);

/* Validates cfg and builds the host-side context (hierarchy, Gauss-Lobatto
 * nodes, integration matrices).  Allocates no device memory. */
int heat3d_init(const heat3d_config* cfg, heat3d_ctx** out);

/* Binds caller-owned device memory (>= heat3d_workspace_size, 256-byte
 * aligned) and zeroes it on the stream.  The memory must outlive the context. */
int heat3d_bind_workspace(heat3d_ctx* ctx, void* dptr, size_t bytes);

/* Releases host resources (graphs, events); never frees the workspace. */
int heat3d_destroy(heat3d_ctx* ctx);

/* Message of the last failure on ctx (never NULL; "" when none). */
const char* heat3d_last_error(const heat3d_ctx* ctx);

/* Replaces the stream every later call enqueues on. */
int heat3d_set_stream(heat3d_ctx* ctx, void* stream);

/* out = nu * Delta_h u on level `level`'s grid (Sec. 1 method of lines;
 * 7-point or wide stencil; nu L u, without W^{-1}, for the compact stencil).
 * u, out: device, dense N^3 FP64. */
int heat3d_apply_laplacian(heat3d_ctx* ctx, int level, const double* u, double* out);

/* Solves (I - c Delta_h) u = rhs ((W - c L) u = rhs for the compact
 * stencil) by V(nu1, nu2) multigrid cycles in the
 * context's precision (Sec. 1.2; coarsening to one unknown).  u is the warm
 * start and the result.  max_cycles/tol as in heat3d_mg.  rhs, u: device,
 * dense N^3 FP64.  Returns HEAT3D_ENOTCONV when tol >= 0 is not reached. */
int mg_vcycle(heat3d_ctx* ctx, int level, double c, const double* rhs, double* u, int max_cycles,
              double tol, heat3d_stats* stats);

/* Spreads the initial value u0 (host or device, dense N^3 FP64) to every
 * node of state slot `item` on `level`, sets the slot's step start t0 and
 * evaluates f^I at every node (the SDC initial iterate). */
int heat3d_set_state(heat3d_ctx* ctx, int level, int item, double t0, const double* u0);

/* Copies node `node` of slot `item` on `level` out to `out` (host or device)
 * or in from `in` (host or device; f^I of that node is re-evaluated). */
int heat3d_get_node(heat3d_ctx* ctx, int level, int item, int node, double* out);
int heat3d_set_node(heat3d_ctx* ctx, int level, int item, int node, const double* in);

/* One IMEX-Euler SDC sweep (Sec. 1.1, the sweep equation with the spectral
 * quadrature S) on slots [batch_begin, batch_begin + batch_count) of
 * `level`; on level 1 the slot's FAS correction (set by heat3d_fas_restrict)
 * is included. */
int sdc_sweep(heat3d_ctx* ctx, int level, int batch_begin, int batch_count, heat3d_stats* stats);

/* Collocation residual max_m max_x |U_0 + dt Q (F + f^E) (+ tau) - U_m| of
 * slot `item` on `level` (Sec. 1: the threshold applies to it). */
int heat3d_sdc_residual(heat3d_ctx* ctx, int level, int item, double* residual);

/* FAS coupling of slots [begin, begin + count) (Sec. 1.1): restriction of
 * the fine state to the coarse level by injection in space and time, coarse
 * f^I and the FAS correction tau; and the interpolation of the coarse
 * correction back (in space trilinear or the midpoint rule that
 * heat3d_config.interp selects, in time Lagrange) with f^I re-evaluated on
 * the fine level. */
int heat3d_fas_restrict(heat3d_ctx* ctx, int begin, int count);
int heat3d_fas_interpolate(heat3d_ctx* ctx, int begin, int count);

/* Sets the interval pfasst_run integrates: [t0, t0 + T] (T a multiple of
 * cfg.dt and of slices * dt).  The default is [0, cfg.T]. */
int heat3d_set_interval(heat3d_ctx* ctx, double t0, double T);

/* Integrates over [t0, t0 + T] (heat3d_set_interval; default [0, cfg.T]): single-level SDC (nlevels = 1), MLSDC
 * (slices = 1) or PFASST on blocks of `slices` time slices (Sec. 1.1).
 * u0 in, uT out: host or device, dense N_fine^3 FP64. */
int pfasst_run(heat3d_ctx* ctx, const double* u0, double* uT, heat3d_stats* stats);

/* ---------------------------------------------------------------------- */
/* Diagnostics (no counterpart in the paper).                               */
/* ---------------------------------------------------------------------- */

/* Kernels this library has launched in the process so far (all contexts). */
long long heat3d_kernel_launches(void);

#define HEAT3D_PROF_OFF 0
#define HEAT3D_PROF_JACOBI_FINE 1 /* damped-Jacobi sweeps on the finest multigrid level of SDC level 0 */
#define HEAT3D_PROF_RESID64_FINE 2 /* FP64 refinement residual on SDC level 0 */
#define HEAT3D_PROF_JACOBI_FINE_STORE 3 /* as 1, the sweeps that store the error (no FP64 update) */
/* Brackets every launch of one kernel class with CUDA events on the context's
 * stream from now on (HEAT3D_PROF_OFF stops and clears). */
int heat3d_profile(heat3d_ctx* ctx, int kernel_class);
/* Totals since heat3d_profile: summed device milliseconds, launches, and the
 * algorithmic bytes, FP64 pipe operations and flops of those launches.
 * Synchronises the stream. */
int heat3d_profile_read(heat3d_ctx* ctx, double* ms, long long* launches, double* bytes,
                        double* dp_ops, double* flops);

/* Self-test of the bounded grid barrier that the persistent solve kernel
 * (heat3d_config.persistent) waits on between its steps: a cooperative launch
 * of 4 blocks on `stream` (a cudaStream_t; NULL: legacy) meets at one barrier.
 * absent_block = -1: all arrive, HEAT3D_OK.  absent_block in 0..3: that block
 * returns without arriving, the others give up after about 1 s of waiting and
 * return, and the call reports HEAT3D_ETIMEOUT (the device stays usable).
 * Synchronises the stream; other values: HEAT3D_EINVAL. */
int heat3d_selftest_barrier(void* stream, int absent_block);

/* FP64 FMA throughput of the current device (fused multiply-adds per second,
 * one FP64-pipe operation each): independent FMA chains on 4 blocks of 512
 * threads per SM, best of three timed launches on `stream` (a cudaStream_t;
 * NULL: legacy).  No counterpart in the paper: it measures the denominator of
 * the FP64 stencil kernels' roofline (they are bound by the FP64 pipe, not by
 * memory).  Synchronises the stream; allocates no device memory.
 * HEAT3D_EINVAL for a NULL output, HEAT3D_ECUDA on a CUDA error. */
int heat3d_fp64_probe(void* stream, double* fma_per_s);

/* Self-test of the bounded mbarrier wait that the FP32 stencils' TMA plane
 * loader uses (no counterpart in the paper): one block of 64 threads waits
 * on a barrier that completes only if `arrive` is non-zero.  arrive != 0:
 * HEAT3D_OK at once; arrive = 0: every wait gives up after about 1 s of SM
 * clock cycles and the call returns HEAT3D_ETIMEOUT (the device stays
 * usable).  Synchronises `stream` (a cudaStream_t; NULL: legacy); allocates
 * no device memory; HEAT3D_ECUDA on a CUDA error. */
int heat3d_selftest_mbarrier(void* stream, int arrive);

/* ---------------------------------------------------------------------- */
/* Solve without any device allocation (no counterpart in the paper).       */
/* ---------------------------------------------------------------------- */

/* mg_vcycle for callers that cannot allocate device memory (a framework that
 * owns all device memory, a plugin given only its input and output buffers,
 * a loop with a memory budget fixed in advance): solves (I - c Delta_h) u =
 * rhs on an N^3 grid exactly as mg_vcycle does, with all scratch taken from a
 * static device array of 32 MiB inside this library (held on every GPU that
 * loads it until exit); no cudaMalloc, cudaFree or other allocating call.
 *  - N = 2^k - 1 <= 63; larger N returns HEAT3D_EINVAL.  order 2 or 4;
 *    precision HEAT3D_FP64 or HEAT3D_MIXED; c, max_cycles, tol as mg_vcycle.
 *  - rhs, u: host or device, dense N^3 FP64; u is the warm start and result.
 *  - Runs on the current device and `stream`.  Every call is synchronous:
 *    it waits for `stream` to finish before it returns, with u complete
 *    (host buffers are read and written on that stream).  So it can never be
 *    captured into a CUDA graph: called while `stream` (NULL: the legacy
 *    stream) is being captured it returns HEAT3D_EINVAL at once, without
 *    touching the stream, and the capture stays valid.
 *  - The first call on a device looks up the array's device address and sets
 *    up the solver state.
 *  - Calls share the array (it keeps the last call's contents; the solver
 *    clears what must start at zero).  Calls that overlap on the GPU race:
 *    serialise them.  stats->seconds is not measured (0).
 *  - Errors: HEAT3D_EINVAL (arguments, N), HEAT3D_ENOMEM (the solver state
 *    does not fit in the array), HEAT3D_ECUDA, or the solve's own code. */
int mg_vcycle_noalloc(int N, int order, int precision, double c, const double* rhs, double* u,
                      int max_cycles, double tol, void* stream, heat3d_stats* stats);
/* Message of the calling thread's last mg_vcycle_noalloc failure. */
const char* mg_vcycle_noalloc_last_error(void);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of independent heat-equation solves.        */
/* ---------------------------------------------------------------------- */

typedef struct {
  int device;
  void* pool;          /* device memory the server sub-allocates request state from */
  size_t pool_bytes;   /* admission is refused (queued) while the pool has no room */
  int max_active;      /* slots: requests resident at once */
  int sweeps;          /* SDC sweeps per step (fixed count) */
  int precision;       /* HEAT3D_FP64 or HEAT3D_MIXED */
  heat3d_mg mg;
} heat3d_server_config;

typedef struct {
  int N;                   /* interior points per axis (2^k - 1) */
  double nu, T, dt;        /* diffusion coefficient, horizon, step */
  int nmodes;              /* <= 8 sine modes of the initial value */
  int k[8][3];             /* mode numbers (k1, k2, k3) */
  double amp[8];           /* amplitudes */
} heat3d_request;

typedef struct heat3d_server heat3d_server;

int heat3d_server_create(const heat3d_server_config* cfg, heat3d_server** out);
/* Queues a request; returns at once with its ticket.  HEAT3D_ENOMEM if the
 * request could never fit in the pool. */
int heat3d_submit(heat3d_server* s, const heat3d_request* req, uint64_t* ticket);
/* *done = 1 once the ticket's solve has finished. */
int heat3d_poll(heat3d_server* s, uint64_t ticket, int* done);
/* Blocks until the ticket finishes; copies u(T) (host or device, dense N^3
 * FP64) and its statistics (NULL to skip either), then releases the ticket. */
int heat3d_wait(heat3d_server* s, uint64_t ticket, double* u_out, heat3d_stats* stats);
/* Latency percentiles (seconds, submit to completion) of finished requests. */
int heat3d_server_latency(heat3d_server* s, double* p50, double* p99, long long* completed);
int heat3d_server_destroy(heat3d_server* s);
const char* heat3d_server_last_error(const heat3d_server* s);

#ifdef __cplusplus
}
#endif
#endif /* HEAT3D_H */
