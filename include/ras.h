/*
 * ras.h - C ABI of the GB300 asynchronous Restricted Additive Schwarz solver.
 *
 * The library solves A x = b (Eq. 1) for a sparse matrix A (symmetric positive
 * definite for the Cholesky / CG / ILU(0)-PCG local solvers; any matrix with
 * nonsingular, pivot-free local blocks for the LU / GMRES local solvers of
 * the generic systems of Sec. 4.1) by Restricted Additive Schwarz (Sec. 2.1):
 * the unknowns are partitioned
 * into subdomains (Sec. 3.2.1), each subdomain is grown by `overlap` layers of
 * graph neighbours (Fig. 1), every subdomain solves its local problem on the
 * overlapped set and keeps only the values it owns. Subdomains run as CTAs of
 * one persistent kernel on one GPU. In RAS_SYNC mode iterations are separated
 * by a grid-wide barrier (the synchronous solver of Sec. 2.1 / Sec. 3.4); in
 * RAS_ASYNC mode every CTA publishes its owned values with release stores and
 * reads its neighbours' values with acquire loads whenever it is ready, with
 * no barrier (the asynchronous solver of Sec. 2.1 / Sec. 3.4). Convergence
 * uses the local criterion of Eq. 2 and the global criterion ||r|| < tol ||b||
 * verified after termination (Sec. 3.3.2).
 *
 * Conventions for every entry point:
 *  - Return value: a ras_status. Errors are returned, never raised or
 *    aborted. Pointers marked HOST are read on the CPU; DEVICE pointers must
 *    be CUDA device memory of the current device.
 *  - The caller owns every input buffer; the library deep-copies what it
 *    keeps, so inputs may be freed as soon as a call returns.
 *  - Work is issued on the stream given to ras_setup (NULL = legacy default
 *    stream). Calls that return results to the host synchronise that stream
 *    before returning.
 *  - A context must not be used by two host threads at the same time.
 */
#ifndef RAS_H
#define RAS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ras_ctx ras_ctx; /* opaque, owned by the library */

typedef enum {
  RAS_OK = 0,
  RAS_EINVAL = 1,   /* invalid argument (sizes, indices, pointers, options) */
  RAS_ENOMEM = 2,   /* host or device allocation failed */
  RAS_ENOTSPD = 3,  /* a local factorisation broke down: a non-positive pivot
                       (Cholesky, ILU(0)) or a zero pivot (LU), or a row of A_p
                       has no positive diagonal entry (local CG) */
  RAS_ENOCONV = 4,  /* max updates / restarts reached; x holds the last iterate */
  RAS_ETIMEOUT = 5, /* a device-side wait exceeded its limit; x is undefined */
  RAS_ECUDA = 6,    /* a CUDA runtime call failed */
  RAS_ENOTSUP = 7   /* valid but unsupported (e.g. local bandwidth too large) */
} ras_status;

/* RAS_SYNC: iterations separated by a grid-wide barrier. RAS_ASYNC: no
 * barrier; a subdomain stops when a device counter of locally converged
 * subdomains (Eq. 2) reaches P (the one-GPU form of the centralized detection
 * of Sec. 3.3.2). RAS_ASYNC_DECENTRAL: no barrier; decentralized, leader-based
 * detection (Sec. 3.3.2): a locally converged subdomain whose neighbours all
 * report local convergence raises a global flag, which every subdomain that
 * sees it on a neighbour raises too before it stops. Both asynchronous modes
 * then verify the global criterion on the frozen x and resume if it fails. */
typedef enum { RAS_SYNC = 0, RAS_ASYNC = 1, RAS_ASYNC_DECENTRAL = 2 } ras_mode;

/* Local solvers (Sec. 3.3.1): a banded Cholesky factorisation computed once
 * in ras_setup with triangular solves in every update, or `inner_iters` steps
 * of CG / ILU(0)-preconditioned CG from a zero initial guess. For general
 * (nonsymmetric) systems (Sec. 4.1): RAS_LOCAL_BANDLU, a banded LU
 * factorisation without pivoting (local half-bandwidth <= 112, else
 * RAS_ENOTSUP; a zero pivot gives RAS_ENOTSPD), applied like the Cholesky
 * factors; RAS_LOCAL_GMRES, `inner_iters` (1..32) steps of one GMRES cycle from
 * a zero initial guess (at most |Omega_p| steps). Banded Cholesky accepts
 * local half-bandwidths up to 160. */
typedef enum {
  RAS_LOCAL_BANDCHOL = 0,
  RAS_LOCAL_CG = 1,
  RAS_LOCAL_ILU0_CG = 2,
  RAS_LOCAL_BANDLU = 3,
  RAS_LOCAL_GMRES = 4
} ras_local_kind;

/* Precision of the local solve. The outer residual, the update of x and the
 * convergence tests are always FP64. RAS_FP32: factors / local matrix stored
 * and used in FP32. RAS_BF16_STORE: band factors stored in bfloat16, applied
 * in FP32 arithmetic (the banded solvers only). */
typedef enum { RAS_FP64 = 0, RAS_FP32 = 1, RAS_BF16_STORE = 2 } ras_prec;

/* Sparse matrix in CSR form. HOST pointers. row_ptr[n+1] (row_ptr[0] = 0,
 * non-decreasing, row_ptr[n] = nnz), col_idx[nnz] in [0, n) and strictly
 * ascending within each row, val[nnz]. The pattern must be structurally
 * symmetric and every row must hold its diagonal. */
typedef struct {
  int32_t n;
  int64_t nnz;
  const int32_t *row_ptr;
  const int32_t *col_idx;
  const double *val;
} ras_csr;

typedef struct {
  int32_t kind;        /* ras_local_kind */
  int32_t prec;        /* ras_prec */
  int32_t inner_iters; /* CG / PCG / GMRES steps per local solve (ignored by the
                          banded solvers) */
  int32_t reserved_;   /* set to 0 */
  double oras_alpha;   /* Optimized RAS (named as future work in Sec. 6): every
                          local matrix A_p takes, on each row, the row's couplings
                          to points outside Omega_p times oras_alpha onto its
                          diagonal, i.e. an exterior neighbour's value is replaced
                          by oras_alpha times the row's own (a Robin-type interface
                          condition; on the 5-point Laplacian the Robin parameter
                          p = (2/h)(1 - a)/(1 + a)). 0 = RAS. The outer residual
                          keeps A, so the solution is unchanged; a too large value
                          can make the iteration diverge (RAS_ENOCONV) or a local
                          factorisation fail (RAS_ENOTSPD). Must be finite. */
} ras_local_solver;

/* Result of one solve. */
typedef struct {
  int64_t iterations;     /* sync: RAS iterations k of the returned x^k;
                             async: median number of local updates */
  int64_t updates_min;    /* per-subdomain local-solve counts */
  int64_t updates_median;
  int64_t updates_max;
  double relres;          /* ||b - A x|| / ||b|| of the returned x, FP64, on device */
  double solve_ms;        /* device time of the solve (CUDA events) */
  int32_t restarts;       /* async: post-termination checks that failed */
  int32_t status;         /* same as the return value of the solve */
  double kernel_ms;       /* device time of the persistent RAS kernel alone */
  int64_t stale_updates;  /* async: local solves that saw no new neighbour data */
  int32_t error_site;     /* RAS_ETIMEOUT only: 1 grid barrier, 3 async idle wait,
                             4 whole-solve time limit, 5 staged-matrix copy (2 is not
                             used: the band copies complete by construction) */
  int32_t grid;           /* CTAs of the solve's persistent launch (on the dynamic
                             schedule every co-resident CTA slot takes subdomains by
                             ticket; the static plan gives each CTA a fixed set) */
} ras_solve_info;

/* ------------------------------------------------------------------------ */
/* Partitioners (Sec. 3.2.1). HOST memory, no GPU work.                      */
/* ------------------------------------------------------------------------ */

/* regular2d partition of an nx x ny grid (index y*nx + x): block column
 * floor(x*px/nx), block row floor(y*py/ny), part = row*px + column.
 * regular1d is px = 1. part[nx*ny] is written. */
ras_status ras_partition_regular2d(int32_t nx, int32_t ny, int32_t px, int32_t py,
                                   int32_t *part);

/* Seeded BFS-growth graph partition into num_parts parts (the stand-in for
 * the Metis partitioner of Sec. 3.2.1): random target sizes within +-30% of
 * n/num_parts, random seed vertices, round-robin breadth-first growth, and
 * leftover vertices joined to their smallest neighbouring part. Deterministic
 * for a given seed; bit-identical to the published rule on any host.
 * part[A->n] is written. */
ras_status ras_partition_bfs(const ras_csr *A, int32_t num_parts, uint64_t seed, int32_t *part);

/* ------------------------------------------------------------------------ */
/* Setup, solve, teardown (Algorithm 1: initialization_and_setup / solve).   */
/* ------------------------------------------------------------------------ */

/* Builds the overlapped subdomains Omega_p (O_p plus `overlap` graph layers,
 * Fig. 1), their restriction maps and local matrices (Sec. 3.2.2), factorises
 * the local matrices on the GPU (banded Cholesky in FP64, stored in the
 * requested precision) or the ILU(0) preconditioners, and uploads everything.
 * partition: HOST int32[A->n] with values in [0, num_parts), every part
 * non-empty. cuda_stream: a cudaStream_t or NULL. On failure *out = NULL.
 * Setup is not part of the solve timing (Sec. 3.1). */
ras_status ras_setup(const ras_csr *A, const int32_t *partition, int32_t num_parts,
                     int32_t overlap, const ras_local_solver *local_solver, void *cuda_stream,
                     ras_ctx **out);

/* Solves A x = b. b: DEVICE double[n]; x: DEVICE double[n], holds the initial
 * guess on entry and the solution on return. tol: relative residual target
 * (global criterion ||b - A x|| < tol ||b||, Sec. 3.3.2). mode: ras_mode.
 * max_updates: limit on local updates per subdomain (<= 0: 10^6).
 * info may be NULL. Synchronises the context's stream. RAS_ENOCONV leaves
 * the last iterate in x. */
ras_status ras_solve(ras_ctx *ctx, const double *b, double *x, double tol, int32_t mode,
                     int64_t max_updates, ras_solve_info *info);

/* Same as ras_solve with HOST b and x: copies b and x to the device, solves,
 * and copies x back, all on the context's stream. Pinned host memory gives
 * asynchronous copies; pageable memory works but is slower. */
ras_status ras_solve_host(ras_ctx *ctx, const double *b_host, double *x_host, double tol,
                          int32_t mode, int64_t max_updates, ras_solve_info *info);

/* Solves several independent systems in ONE persistent launch. All contexts
 * must share the local solver kind and precision and the stream of ctxs[0]
 * is used. b[i], x[i]: DEVICE arrays of ctxs[i]'s size. infos: num entries
 * or NULL. Returns the first non-OK status. */
ras_status ras_solve_batch(ras_ctx *const *ctxs, int32_t num, const double *const *b,
                           double *const *x, double tol, int32_t mode, int64_t max_updates,
                           ras_solve_info *infos);

/* Choice made by ras_autotune. */
typedef struct {
  int32_t cta_threads;  /* threads per CTA of the persistent kernel */
  int32_t staged;       /* 1: local matrix staged in shared memory (FP32 CG) */
  int32_t inner_iters;  /* CG / PCG steps per local solve */
  int32_t candidates;   /* configurations timed */
  double score;         /* best -ln(relres) per kernel millisecond */
  int32_t schedule;     /* 1 dynamic (CTAs take subdomains by ticket; synchronous
                           solves per iteration), 0 static assignment */
  int32_t grid;         /* CTAs of the tuned launch */
  int32_t per_cta;      /* static assignment: subdomains per CTA (dynamic: 0) */
  int32_t reserved_;
} ras_tune_result;

/* Launch-shape autotuner (not in the paper: the GPU counterpart of choosing
 * the local solver's parameters). For each candidate - CTA threads (128 / 256
 * for the banded solvers, 256 / 512 for CG and ILU-PCG, the shared-memory
 * staged FP32 CG), the launch shape (the dynamic ticket schedule on every
 * co-resident CTA slot, or the static assignment; a CTA cap of every slot or
 * half the subdomains, i.e. at least two subdomains per CTA), and with
 * tune_inner != 0 the inner step counts m/2, m, 2m - it runs the context's
 * system with a zero right-hand side from x = 1 (x_scratch: DEVICE double[n],
 * overwritten), `iters` updates and then `iters` more. With b = 0 the error is
 * x itself, dominated by the smoothest modes, so the second window's residual
 * reduction per millisecond of kernel time is the asymptotic rate that sets
 * time-to-solution. The best candidate is kept for every later solve. out may
 * be NULL. */
ras_status ras_autotune(ras_ctx *ctx, double *x_scratch, int32_t mode, int32_t iters,
                        int32_t tune_inner, ras_tune_result *out);

/* ------------------------------------------------------------------------ */
/* Continuous batching (serving)                                             */
/* ------------------------------------------------------------------------ */

/* Starts a solve on ctx without running it: records b, x (DEVICE, x holds
 * the initial guess) and tol, and initialises the solve state on the
 * context's stream (||b||^2 over every Omega_p and O_p, counters, the async
 * phase word). The context then advances only through ras_batch_step, which
 * may run it together with other contexts. */
ras_status ras_solve_begin(ras_ctx *ctx, const double *b, double *x, double tol);

/* Advances every listed context - each started with ras_solve_begin - in ONE
 * persistent launch (the batched launch of the subdomains of all systems, as
 * in ras_solve_batch) by at most step_limit local updates per subdomain
 * (RAS_ASYNC: the asynchronous solver of Sec. 2.1 with its convergence
 * detection, Sec. 3.3.2) or step_limit iterations (RAS_SYNC). Systems that
 * finished earlier are skipped. Between steps each x holds the current
 * iterate. Issued on the stream of ctxs[0] after the streams of the others.
 * done (HOST int32[num], may be NULL): 1 for systems finished (converged or
 * failed) by the end of this step. infos (HOST, may be NULL): filled for
 * finished systems. max_updates as in ras_solve. Returns the first non-OK
 * status among finished systems, or a launch error. */
ras_status ras_batch_step(ras_ctx *const *ctxs, int32_t num, int32_t mode, int64_t step_limit,
                          int64_t max_updates, int32_t *done, ras_solve_info *infos);

/* Releases a context (NULL is allowed). Synchronises its stream first. */
ras_status ras_destroy(ras_ctx *ctx);

/* ------------------------------------------------------------------------ */
/* Inspection (tests, tools)                                                 */
/* ------------------------------------------------------------------------ */

/* Maps of subdomain p, as built by ras_setup. Returned pointers are HOST
 * memory owned by the context and valid until ras_destroy:
 * omega[n_omega] (global ids of Omega_p, ascending), owned_mask[n_omega]
 * (1 where omega[t] is in O_p), iface[n_iface] (E_p: points outside Omega_p
 * coupled to it, ascending). */
ras_status ras_get_maps(const ras_ctx *ctx, int32_t p, const int32_t **omega, int32_t *n_omega,
                        const uint8_t **owned_mask, const int32_t **iface, int32_t *n_iface);

/* Sizes of the context: number of subdomains, global n, maximum local
 * half-bandwidth, and the bytes of device memory it holds. */
ras_status ras_get_info(const ras_ctx *ctx, int32_t *num_parts, int32_t *n, int32_t *max_bandwidth,
                        int64_t *device_bytes);

/* Per-subdomain local-update counts of the last solve: counts[num_parts]. */
ras_status ras_get_update_counts(const ras_ctx *ctx, int64_t *counts);

/* Launch shape the context uses: kernel_variant 0 banded triangular solves
 * (Cholesky or LU factors), 1 CG reading A_p from global memory, 2
 * ILU(0)-PCG, 3 CG with A_p staged in shared memory, 4 GMRES, 5 CG with A_p
 * staged in shared memory in diagonal-offset form (chosen for a 2D / 3D
 * stencil in lexicographic order, whose subdomains' rows are laid out on
 * grid boxes: no column indices); threads per
 * CTA; CTAs (one cooperative launch); CG / PCG / GMRES steps per local solve.
 * Any pointer may be NULL. */
ras_status ras_get_launch(const ras_ctx *ctx, int32_t *kernel_variant, int32_t *cta_threads,
                          int32_t *grid, int32_t *inner_iters);

/* Runtime breakdown of the last solve, per subdomain (the per-update timing
 * of Sec. 4's Figs. 3a-7a): ns[3*p+0] nanoseconds spent gathering the local
 * residual (reading neighbours' values), ns[3*p+1] in the local solve,
 * ns[3*p+2] in the restricted update and publish, summed over all updates of
 * subdomain p (device %globaltimer, measured by the CTA that ran it).
 * ns: HOST uint64[3 * num_parts]. RAS_EINVAL before the first solve. */
ras_status ras_get_phase_times(const ras_ctx *ctx, uint64_t *ns);

/* FP64 global relative residual ||b - A x|| / ||b|| computed on the device
 * (b, x DEVICE). Synchronises the context's stream. */
ras_status ras_relres(ras_ctx *ctx, const double *b, const double *x, double *relres);

/* No-allocation relative residual, for callers that cannot call cudaMalloc
 * (code running during CUDA graph capture, programs whose device memory
 * belongs to a fixed pool or custom allocator, loops that must not allocate
 * after start-up). The paper has no counterpart: it is an operational entry
 * point of this library. Computes ||b - A x||_2 / ||b||_2 (or ||b - A x||_2
 * when b = 0) in FP64 for a caller-held DEVICE CSR matrix (row_ptr[n+1],
 * col_idx, val, same rules as ras_csr) and DEVICE vectors b[n], x[n], and
 * writes it to the DEVICE double *relres, stream-ordered on cuda_stream
 * (NULL = legacy default stream); it does not synchronise. It allocates
 * nothing: its scratch (one pair of partial sums per 1024 rows) is a
 * 1 MiB file-scope device array that every GPU loading the library holds
 * until exit, so n may be at most 67,108,864 (larger n: RAS_EINVAL). The
 * first call on a device looks the array's address up with that device
 * current; make that first call before any stream capture (calls outside a
 * capture look it up again, so a cudaDeviceReset in between does no harm).
 * All calls share the array: calls that overlap on the GPU race and must be
 * ordered by the caller. */
ras_status ras_relres_noalloc(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                              const double *val, const double *b, const double *x, double *relres,
                              void *cuda_stream);

/* Static description of a status code. */
const char *ras_status_str(ras_status status);

#ifdef __cplusplus
}
#endif
#endif /* RAS_H */
