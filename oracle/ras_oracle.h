/*
 * CPU oracle for the Restricted Additive Schwarz (RAS) solver.
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, sequential FP64
 * restatement of the method, used to check the CUDA path. Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header or table with the CUDA library.
 *
 * Notation (Sec. 2.1, Fig. 1): O_p = rows owned by subdomain p (the
 * partition), Omega_p = O_p grown by `gamma` layers of graph neighbours (the
 * overlap), E_p = points outside Omega_p coupled to it (the external
 * interface, red points of Fig. 1). Local unknowns are Omega_p in ascending
 * global order.
 *
 * Return codes: 0 ok, 1 invalid argument, 3 local factorisation broke down
 * (Cholesky: not SPD; LU: zero pivot), 4 no convergence.
 */
#ifndef RAS_ORACLE_H
#define RAS_ORACLE_H
#include <stdint.h>

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOTSPD 3
#define OR_ENOCONV 4

/* local solver kinds and precisions */
#define OR_BANDCHOL 0
#define OR_CG 1
#define OR_ILU0_CG 2
#define OR_BANDLU 3 /* general matrices */
#define OR_GMRES 4  /* general matrices */
#define OR_FP64 0
#define OR_FP32 1
#define OR_BF16 2

/* SplitMix64 output k (0-based) of the stream with the given seed. */
uint64_t or_splitmix64(uint64_t seed, uint64_t k);
/* Round a double to bfloat16 (round to nearest even) and back to double. */
double or_round_bf16(double v);

/* Partitioners (Sec. 3.2.1). */
int or_partition_regular2d(int nx, int ny, int px, int py, int32_t *part);
int or_partition_bfs(int n, const int32_t *rp, const int32_t *ci, int P, uint64_t seed,
                     int32_t *part);

/* Overlap maps of subdomain p. omega/owned/iface need room for n entries. */
int or_overlap(int n, const int32_t *rp, const int32_t *ci, const int32_t *part, int P, int p,
               int gamma, int32_t *omega, int32_t *n_omega, uint8_t *owned, int32_t *iface,
               int32_t *n_iface);

/* Banded Cholesky. band[i*(w+1)+t] holds A[i][i-w+t] (t = 0..w); in place -> L. */
int or_band_cholesky(int n, int w, double *band);
/* Solve L L^T x = rhs in place (FP64). */
void or_band_solve(int n, int w, const double *L, double *x);
/* Same with factors rounded to `prec` (OR_FP32 / OR_BF16) and FP32 arithmetic. */
void or_band_solve_lowp(int n, int w, const double *L, int prec, double *x);

/* Banded LU without pivoting (general A_p with half-bandwidth w).
 * band[i*(2w+1)+t] holds A[i][i-w+t] (t = 0..2w); in place -> unit lower L
 * below the diagonal, U on and above it. */
int or_band_lu(int n, int w, double *band);
/* Solve L U x = rhs in place (FP64), and with rounded factors in FP32. */
void or_band_lu_solve(int n, int w, const double *LU, double *x);
void or_band_lu_solve_lowp(int n, int w, const double *LU, int prec, double *x);

/* Dense LU with partial pivoting: solves A x = b in place (A overwritten). */
int or_dense_lu_solve(int n, double *A, double *b);

/* m iterations of textbook CG on A d = rhs from d = 0 (FP64 or FP32 arithmetic). */
void or_cg(int n, const int32_t *rp, const int32_t *ci, const double *val, const double *rhs,
           int m, int prec, double *d);
/* m steps of GMRES (one cycle, Arnoldi with modified Gram-Schmidt, Givens
 * rotations) on A d = rhs from d = 0, FP64 or FP32 arithmetic. */
void or_gmres(int n, const int32_t *rp, const int32_t *ci, const double *val, const double *rhs,
              int m, int prec, double *d);
/* ILU(0) on the CSR pattern (IKJ order). lu has the pattern of A. */
int or_ilu0(int n, const int32_t *rp, const int32_t *ci, const double *val, double *lu);
/* m iterations of CG preconditioned by the ILU(0) factors, from d = 0. */
void or_pcg_ilu0(int n, const int32_t *rp, const int32_t *ci, const double *val,
                 const double *lu, const double *rhs, int m, int prec, double *d);

/* r = b - A x; returns ||r||_2^2 summed in index order. r may be NULL. */
double or_residual(int n, const int32_t *rp, const int32_t *ci, const double *val,
                   const double *b, const double *x, double *r);

/*
 * Synchronous RAS in correction form (Algorithm 1 with the RAS update of
 * Sec. 2.1). x holds x^0 on entry and the final iterate on exit. hist (may be
 * NULL) receives ||b - A x^k|| / ||b|| for k = 0..iters. nthreads > 1 runs the
 * independent local solves of one iteration in parallel (same result).
 */
int or_ras_sync(int n, const int32_t *rp, const int32_t *ci, const double *val, const double *b,
                const int32_t *part, int P, int gamma, int kind, int prec, int m, double tol,
                int max_iter, int nthreads, double *x, double *hist, int32_t *iters);
/*
 * Same with optimized (Robin-type) local matrices, the Optimized RAS the
 * paper names as future work (Sec. 6): in each local matrix A_p every value
 * of an exterior neighbour j in E_p is replaced by alpha times the value of
 * the row's own unknown, i.e. A_p[t][t] += alpha * sum_{j in E_p} A[i][j]
 * (i the global row of t). alpha = 0 is RAS (Dirichlet data at E_p); on the
 * 5-point Laplacian alpha is the ghost-value ratio of a Robin condition
 * du/dn + p u = 0 at the midpoint of the cut edge, p = (2/h)(1-alpha)/(1+alpha).
 * The residual stays that of A, so the fixed point is unchanged.
 */
int or_ras_sync_ex(int n, const int32_t *rp, const int32_t *ci, const double *val,
                   const double *b, const int32_t *part, int P, int gamma, int kind, int prec,
                   int m, double alpha, double tol, int max_iter, int nthreads, double *x,
                   double *hist, int32_t *iters);

/*
 * The same iteration split as Algorithm 1 splits it: or_ras_new does the
 * set-up (overlap maps, local matrices, factorisations; untimed in Sec. 3.1)
 * and keeps pointers to rp / ci / val (which must outlive the handle);
 * or_ras_iterate runs synchronous RAS iterations from x (the same arithmetic
 * as or_ras_sync_ex, which is new + iterate + free).
 */
typedef struct or_ras or_ras;
int or_ras_new(int n, const int32_t *rp, const int32_t *ci, const double *val,
               const int32_t *part, int P, int gamma, int kind, int prec, int m, double alpha,
               or_ras **out);
int or_ras_iterate(const or_ras *h, const double *b, double tol, int max_iter, int nthreads,
                   double *x, double *hist, int32_t *iters);
void or_ras_free(or_ras *h);

#endif
