/*
 * CPU oracle for the Restricted Additive Schwarz solver (plain C, FP64).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path. Every routine is
 * a direct, sequential restatement of its definition; nothing is blocked,
 * fused or reordered. Build flags: -O2 -ffp-contract=off (no FMA
 * contraction, so x86 and Arm hosts give identical results).
 *
 * Paper sections followed:
 *   Sec. 2.1 / Fig. 1   overlapping decomposition with overlap gamma, the
 *                       external interface (red points), and the RAS rule
 *                       "solve on the overlap, keep only owned values".
 *   Sec. 2.1            synchronous Schwarz: every subdomain uses x^k.
 *   Sec. 3.1, Alg. 1    partition, set up, then loop: local solve, exchange,
 *                       convergence check.
 *   Sec. 3.2.1          regular1d / regular2d partitions (a seeded
 *                       BFS-growth partitioner stands in for Metis).
 *   Sec. 3.3.1          direct local solves: Cholesky factorisation once,
 *                       triangular solves every iteration; or an iterative
 *                       local solver (CG).
 *   Sec. 4.1            a generic (nonsymmetric) system with LU or GMRES
 *                       local solves.
 *   Sec. 3.3.2, Eq. 2   local criterion ||r_p||^2 < tau^2 ||b_p||^2 and the
 *                       global criterion ||r|| < tau ||b||.
 */
#include "ras_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* random numbers and rounding                                               */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output k mixes the state
 * seed + (k+1) * golden-ratio increment. */
uint64_t or_splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static double or_u01(uint64_t seed, uint64_t k) {
  return (double)(or_splitmix64(seed, k) >> 11) * (1.0 / 9007199254740992.0);
}

/* bfloat16 keeps 8 significant bits and float's exponent range. Round the
 * significand to 8 bits, ties to even (rint in the default rounding mode). */
double or_round_bf16(double v) {
  if (v == 0.0 || !isfinite(v)) return v;
  int e;
  double f = frexp(v, &e); /* v = f * 2^e, 0.5 <= |f| < 1 */
  double q = rint(ldexp(f, 8));
  return ldexp(q, e - 8);
}

static float or_round_storage(double v, int prec) {
  if (prec == OR_BF16) return (float)or_round_bf16(v);
  return (float)v;
}

/* ------------------------------------------------------------------------ */
/* partitioners (Sec. 3.2.1)                                                 */
/* ------------------------------------------------------------------------ */

/* regular2d: block column floor(x*px/nx), block row floor(y*py/ny);
 * regular1d is px = 1 (row strips). */
int or_partition_regular2d(int nx, int ny, int px, int py, int32_t *part) {
  if (nx <= 0 || ny <= 0 || px <= 0 || py <= 0 || px > nx || py > ny) return OR_EINVAL;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      int bx = (int)(((int64_t)x * px) / nx);
      int by = (int)(((int64_t)y * py) / ny);
      part[(int64_t)y * nx + x] = by * px + bx;
    }
  return OR_OK;
}

/* BFS-growth partitioner, a seeded graph partitioner in place of Metis.
 * 1. Target sizes: w_p = 1 + 0.3 (2 u_p - 1), t_p = floor(n w_p / sum w);
 *    the remainder goes one each to p = 0, 1, ... (taken back the same way if
 *    negative).
 * 2. Seeds: v = floor(u_{P+p} n), probing v+1, v+2, ... (mod n) past
 *    assigned vertices.
 * 3. Rounds: each part below target claims the first unassigned neighbour of
 *    its FIFO front (scanning the front's row from its cursor); a front with
 *    none left is popped. Stop when a round claims nothing.
 * 4. Leftovers: sweeps in index order join an unassigned vertex to its
 *    smallest-size assigned neighbour part (ties: smallest id); a component
 *    with no assigned vertex starts from its lowest index in part
 *    argmin(size). */
int or_partition_bfs(int n, const int32_t *rp, const int32_t *ci, int P, uint64_t seed,
                     int32_t *part) {
  if (n <= 0 || P <= 0 || P > n) return OR_EINVAL;
  double *w = (double *)malloc(sizeof(double) * P);
  int64_t *target = (int64_t *)malloc(sizeof(int64_t) * P);
  int64_t *size = (int64_t *)calloc(P, sizeof(int64_t));
  int32_t *head = (int32_t *)malloc(sizeof(int32_t) * P);
  int32_t *tail = (int32_t *)malloc(sizeof(int32_t) * P);
  int32_t *next = (int32_t *)malloc(sizeof(int32_t) * n);
  int32_t *cursor = (int32_t *)malloc(sizeof(int32_t) * n);
  double W = 0.0;
  for (int p = 0; p < P; ++p) {
    w[p] = 1.0 + 0.3 * (2.0 * or_u01(seed, (uint64_t)p) - 1.0);
    W += w[p];
  }
  int64_t sum = 0;
  for (int p = 0; p < P; ++p) {
    target[p] = (int64_t)floor((double)n * w[p] / W);
    sum += target[p];
  }
  int64_t rem = (int64_t)n - sum;
  for (int p = 0; rem > 0; p = (p + 1) % P) { target[p]++; rem--; }
  for (int p = 0; rem < 0; p = (p + 1) % P)
    if (target[p] > 0) { target[p]--; rem++; }

  for (int i = 0; i < n; ++i) { part[i] = -1; next[i] = -1; cursor[i] = rp[i]; }
  for (int p = 0; p < P; ++p) { head[p] = -1; tail[p] = -1; }

  for (int p = 0; p < P; ++p) {
    int v = (int)floor(or_u01(seed, (uint64_t)(P + p)) * (double)n);
    if (v >= n) v = n - 1;
    while (part[v] != -1) v = (v + 1) % n;
    part[v] = p;
    size[p] = 1;
    head[p] = tail[p] = v;
  }

  for (;;) {
    int64_t claimed = 0;
    for (int p = 0; p < P; ++p) {
      if (size[p] >= target[p]) continue;
      while (head[p] != -1) {
        int f = head[p];
        int found = -1;
        while (cursor[f] < rp[f + 1]) {
          int j = ci[cursor[f]];
          cursor[f]++;
          if (part[j] == -1) { found = j; break; }
        }
        if (found >= 0) {
          part[found] = p;
          size[p]++;
          next[tail[p]] = found;
          tail[p] = found;
          claimed++;
          break;
        }
        head[p] = next[f]; /* pop f */
        if (head[p] == -1) tail[p] = -1;
      }
    }
    if (claimed == 0) break;
  }

  for (;;) {
    int changed = 1;
    while (changed) {
      changed = 0;
      for (int i = 0; i < n; ++i) {
        if (part[i] != -1) continue;
        int best = -1;
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
          int q = part[ci[k]];
          if (q < 0) continue;
          if (best < 0 || size[q] < size[best] || (size[q] == size[best] && q < best)) best = q;
        }
        if (best >= 0) { part[i] = best; size[best]++; changed = 1; }
      }
    }
    int i0 = -1;
    for (int i = 0; i < n; ++i)
      if (part[i] == -1) { i0 = i; break; }
    if (i0 < 0) break;
    int q = 0;
    for (int p = 1; p < P; ++p)
      if (size[p] < size[q]) q = p;
    part[i0] = q;
    size[q]++;
  }
  free(w); free(target); free(size); free(head); free(tail); free(next); free(cursor);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* overlap (Sec. 2.1, Fig. 1)                                                */
/* ------------------------------------------------------------------------ */

/* Omega_p: O_p plus every point within `gamma` graph steps of it (one layer
 * of neighbours per unit of overlap), ascending. E_p: points outside Omega_p
 * coupled to a point of Omega_p, ascending. */
int or_overlap(int n, const int32_t *rp, const int32_t *ci, const int32_t *part, int P, int p,
               int gamma, int32_t *omega, int32_t *n_omega, uint8_t *owned, int32_t *iface,
               int32_t *n_iface) {
  if (n <= 0 || p < 0 || p >= P || gamma < 0) return OR_EINVAL;
  int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * n);
  int32_t *front = (int32_t *)malloc(sizeof(int32_t) * n);
  int32_t *nfront = (int32_t *)malloc(sizeof(int32_t) * n);
  int nf = 0;
  for (int i = 0; i < n; ++i) {
    dist[i] = -1;
    if (part[i] == p) { dist[i] = 0; front[nf++] = i; }
  }
  for (int level = 1; level <= gamma; ++level) {
    int nn = 0;
    for (int a = 0; a < nf; ++a) {
      int v = front[a];
      for (int k = rp[v]; k < rp[v + 1]; ++k) {
        int j = ci[k];
        if (dist[j] == -1) { dist[j] = level; nfront[nn++] = j; }
      }
    }
    memcpy(front, nfront, sizeof(int32_t) * nn);
    nf = nn;
  }
  int no = 0;
  for (int i = 0; i < n; ++i)
    if (dist[i] >= 0) {
      omega[no] = i;
      owned[no] = (uint8_t)(part[i] == p);
      no++;
    }
  /* interface: mark with -2 */
  for (int t = 0; t < no; ++t) {
    int v = omega[t];
    for (int k = rp[v]; k < rp[v + 1]; ++k)
      if (dist[ci[k]] == -1) dist[ci[k]] = -2;
  }
  int ni = 0;
  for (int i = 0; i < n; ++i)
    if (dist[i] == -2) iface[ni++] = i;
  *n_omega = no;
  *n_iface = ni;
  free(dist); free(front); free(nfront);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* local direct solver: banded Cholesky (Sec. 3.3.1)                         */
/* ------------------------------------------------------------------------ */

#define BAND(L, w, i, j) ((L)[(int64_t)(i) * ((w) + 1) + ((j) - (i) + (w))])

/* Row-by-row (Cholesky-Banachiewicz) factorisation inside the band. */
int or_band_cholesky(int n, int w, double *band) {
  for (int i = 0; i < n; ++i) {
    int j0 = i - w > 0 ? i - w : 0;
    for (int j = j0; j <= i; ++j) {
      double s = BAND(band, w, i, j);
      int k0 = j0 > j - w ? j0 : j - w;
      if (k0 < 0) k0 = 0;
      for (int k = k0; k < j; ++k) s -= BAND(band, w, i, k) * BAND(band, w, j, k);
      if (j < i) {
        BAND(band, w, i, j) = s / BAND(band, w, j, j);
      } else {
        if (!(s > 0.0)) return OR_ENOTSPD;
        BAND(band, w, i, i) = sqrt(s);
      }
    }
  }
  return OR_OK;
}

/* Forward substitution L y = rhs, then backward substitution L^T x = y. */
void or_band_solve(int n, int w, const double *L, double *x) {
  for (int i = 0; i < n; ++i) {
    double s = x[i];
    int k0 = i - w > 0 ? i - w : 0;
    for (int k = k0; k < i; ++k) s -= BAND(L, w, i, k) * x[k];
    x[i] = s / BAND(L, w, i, i);
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    int k1 = i + w < n - 1 ? i + w : n - 1;
    for (int k = i + 1; k <= k1; ++k) s -= BAND(L, w, k, i) * x[k];
    x[i] = s / BAND(L, w, i, i);
  }
}

/* Same substitutions with every factor entry rounded to the storage
 * precision and FP32 arithmetic (the right-hand side is rounded to FP32). */
void or_band_solve_lowp(int n, int w, const double *L, int prec, double *x) {
  float *y = (float *)malloc(sizeof(float) * (n > 0 ? n : 1));
  for (int i = 0; i < n; ++i) y[i] = (float)x[i];
  for (int i = 0; i < n; ++i) {
    float s = y[i];
    int k0 = i - w > 0 ? i - w : 0;
    for (int k = k0; k < i; ++k) s -= or_round_storage(BAND(L, w, i, k), prec) * y[k];
    y[i] = s / or_round_storage(BAND(L, w, i, i), prec);
  }
  for (int i = n - 1; i >= 0; --i) {
    float s = y[i];
    int k1 = i + w < n - 1 ? i + w : n - 1;
    for (int k = i + 1; k <= k1; ++k) s -= or_round_storage(BAND(L, w, k, i), prec) * y[k];
    y[i] = s / or_round_storage(BAND(L, w, i, i), prec);
  }
  for (int i = 0; i < n; ++i) x[i] = (double)y[i];
  free(y);
}

/* ------------------------------------------------------------------------ */
/* local direct solver for general matrices: banded LU (Sec. 4.1 names LU   */
/* as the local solver for a generic system)                                 */
/* ------------------------------------------------------------------------ */

#define BANDG(U, w, i, j) ((U)[(int64_t)(i) * (2 * (w) + 1) + ((j) - (i) + (w))])

/* Doolittle LU without pivoting inside the band, row by row:
 *   l_ij = (a_ij - sum_{k<j} l_ik u_kj) / u_jj   for j < i (unit lower L),
 *   u_ij =  a_ij - sum_{k<i} l_ik u_kj           for j >= i,
 * where only |i-k|, |k-j| <= w contribute. A zero pivot u_ii stops it. */
int or_band_lu(int n, int w, double *band) {
  for (int i = 0; i < n; ++i) {
    int j0 = i - w > 0 ? i - w : 0;
    int j1 = i + w < n - 1 ? i + w : n - 1;
    for (int j = j0; j <= j1; ++j) {
      double s = BANDG(band, w, i, j);
      int k0 = j - w > j0 ? j - w : j0;
      int k1 = (i < j ? i : j) - 1;
      for (int k = k0; k <= k1; ++k) s -= BANDG(band, w, i, k) * BANDG(band, w, k, j);
      if (j < i) {
        BANDG(band, w, i, j) = s / BANDG(band, w, j, j);
      } else {
        if (j == i && !(fabs(s) > 0.0)) return OR_ENOTSPD;
        BANDG(band, w, i, j) = s;
      }
    }
  }
  return OR_OK;
}

/* Forward substitution with the unit lower L, then backward with U. */
void or_band_lu_solve(int n, int w, const double *LU, double *x) {
  for (int i = 0; i < n; ++i) {
    double s = x[i];
    int k0 = i - w > 0 ? i - w : 0;
    for (int k = k0; k < i; ++k) s -= BANDG(LU, w, i, k) * x[k];
    x[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    int k1 = i + w < n - 1 ? i + w : n - 1;
    for (int k = i + 1; k <= k1; ++k) s -= BANDG(LU, w, i, k) * x[k];
    x[i] = s / BANDG(LU, w, i, i);
  }
}

/* Same with the factors rounded to `prec` and FP32 arithmetic. */
void or_band_lu_solve_lowp(int n, int w, const double *LU, int prec, double *x) {
  float *y = (float *)malloc(sizeof(float) * (n > 0 ? n : 1));
  for (int i = 0; i < n; ++i) y[i] = (float)x[i];
  for (int i = 0; i < n; ++i) {
    float s = y[i];
    int k0 = i - w > 0 ? i - w : 0;
    for (int k = k0; k < i; ++k) s -= or_round_storage(BANDG(LU, w, i, k), prec) * y[k];
    y[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    float s = y[i];
    int k1 = i + w < n - 1 ? i + w : n - 1;
    for (int k = i + 1; k <= k1; ++k) s -= or_round_storage(BANDG(LU, w, i, k), prec) * y[k];
    y[i] = s / or_round_storage(BANDG(LU, w, i, i), prec);
  }
  for (int i = 0; i < n; ++i) x[i] = (double)y[i];
  free(y);
}

/* ------------------------------------------------------------------------ */
/* dense LU with partial pivoting (for small-grid checks)                    */
/* ------------------------------------------------------------------------ */

int or_dense_lu_solve(int n, double *A, double *b) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[(int64_t)i * n + k]) > fabs(A[(int64_t)piv * n + k])) piv = i;
    if (A[(int64_t)piv * n + k] == 0.0) return OR_EINVAL;
    if (piv != k) {
      for (int j = 0; j < n; ++j) {
        double t = A[(int64_t)k * n + j];
        A[(int64_t)k * n + j] = A[(int64_t)piv * n + j];
        A[(int64_t)piv * n + j] = t;
      }
      double t = b[k]; b[k] = b[piv]; b[piv] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      double l = A[(int64_t)i * n + k] / A[(int64_t)k * n + k];
      A[(int64_t)i * n + k] = l;
      for (int j = k + 1; j < n; ++j) A[(int64_t)i * n + j] -= l * A[(int64_t)k * n + j];
      b[i] -= l * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A[(int64_t)i * n + j] * b[j];
    b[i] = s / A[(int64_t)i * n + i];
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* local iterative solvers (Sec. 3.3.1: "or an iterative solver such as CG") */
/* ------------------------------------------------------------------------ */

/* Textbook conjugate gradients, m steps from d = 0:
 *   q = A p; alpha = rr / (p.q); d += alpha p; r -= alpha q;
 *   rr' = r.r; beta = rr'/rr; p = r + beta p.
 * Stops early only when r.r == 0. */
void or_cg(int n, const int32_t *rp, const int32_t *ci, const double *val, const double *rhs,
           int m, int prec, double *d) {
  if (prec == OR_FP64) {
    double *r = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    double *q = (double *)malloc(sizeof(double) * n);
    double rr = 0.0;
    for (int i = 0; i < n; ++i) { d[i] = 0.0; r[i] = rhs[i]; p[i] = rhs[i]; rr += r[i] * r[i]; }
    for (int it = 0; it < m && rr != 0.0; ++it) {
      double pq = 0.0;
      for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) s += val[k] * p[ci[k]];
        q[i] = s;
        pq += p[i] * s;
      }
      double alpha = rr / pq;
      double rr2 = 0.0;
      for (int i = 0; i < n; ++i) {
        d[i] += alpha * p[i];
        r[i] -= alpha * q[i];
        rr2 += r[i] * r[i];
      }
      double beta = rr2 / rr;
      for (int i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
      rr = rr2;
    }
    free(r); free(p); free(q);
  } else {
    float *r = (float *)malloc(sizeof(float) * n);
    float *p = (float *)malloc(sizeof(float) * n);
    float *q = (float *)malloc(sizeof(float) * n);
    float *x = (float *)malloc(sizeof(float) * n);
    float rr = 0.0f;
    for (int i = 0; i < n; ++i) {
      x[i] = 0.0f; r[i] = (float)rhs[i]; p[i] = r[i]; rr += r[i] * r[i];
    }
    for (int it = 0; it < m && rr != 0.0f; ++it) {
      float pq = 0.0f;
      for (int i = 0; i < n; ++i) {
        float s = 0.0f;
        for (int k = rp[i]; k < rp[i + 1]; ++k) s += or_round_storage(val[k], prec) * p[ci[k]];
        q[i] = s;
        pq += p[i] * s;
      }
      float alpha = rr / pq;
      float rr2 = 0.0f;
      for (int i = 0; i < n; ++i) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
        rr2 += r[i] * r[i];
      }
      float beta = rr2 / rr;
      for (int i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
      rr = rr2;
    }
    for (int i = 0; i < n; ++i) d[i] = (double)x[i];
    free(r); free(p); free(q); free(x);
  }
}

/* Working-precision rounding for the GMRES below: in FP32 mode every
 * operation's result is rounded to float. The operands are floats, so the
 * double result of + - * / and sqrt rounded once more to float is the
 * correctly rounded float result (double carries more than 2*24+2 bits;
 * S. A. Figueroa, "When is double rounding innocuous?", SIGNUM 1995). */
static double or_fl(int prec, double v) { return prec == OR_FP64 ? v : (double)(float)v; }

/* m steps of GMRES (Saad & Schultz 1986) on A d = rhs from d = 0, one cycle:
 * Arnoldi with modified Gram-Schmidt builds V (orthonormal) and the upper
 * Hessenberg H with A V_k = V_{k+1} H; Givens rotations reduce H to upper
 * triangular R and carry ||rhs|| e_1 along as g; then R y = g and
 * d = V_k y, the vector of the Krylov space K_k(A, rhs) with the least
 * residual 2-norm. Takes at most n steps (K_n is the whole space) and stops
 * early only on an exact breakdown (h_{j+1,j} == 0), where d is exact. FP32 mode: A's entries rounded to float and every
 * operation in float (emulated by or_fl). */
void or_gmres(int n, const int32_t *rp, const int32_t *ci, const double *val, const double *rhs,
              int m, int prec, double *d) {
  const int ld = m + 1;
  double *V = (double *)calloc((size_t)(m + 1) * (n > 0 ? n : 1), sizeof(double));
  double *w = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
  double *H = (double *)calloc((size_t)ld * (m > 0 ? m : 1), sizeof(double)); /* H[i + j*ld] */
  double *cs = (double *)calloc(m > 0 ? m : 1, sizeof(double));
  double *sn = (double *)calloc(m > 0 ? m : 1, sizeof(double));
  double *g = (double *)calloc(m + 1, sizeof(double));
  double *y = (double *)calloc(m > 0 ? m : 1, sizeof(double));
  for (int i = 0; i < n; ++i) d[i] = 0.0;
  double beta2 = 0.0;
  for (int i = 0; i < n; ++i) {
    double ri = or_fl(prec, rhs[i]);
    beta2 = or_fl(prec, beta2 + or_fl(prec, ri * ri));
  }
  double beta = or_fl(prec, sqrt(beta2));
  int k = 0;
  if (m > n) m = n; /* K_n is already the whole space */
  if (beta > 0.0) {
    for (int i = 0; i < n; ++i) V[i] = or_fl(prec, or_fl(prec, rhs[i]) / beta);
    g[0] = beta;
    for (int j = 0; j < m; ++j) {
      const double *vj = V + (size_t)j * n;
      for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e)
          s = or_fl(prec, s + or_fl(prec, or_fl(prec, val[e]) * vj[ci[e]]));
        w[i] = s;
      }
      for (int q = 0; q <= j; ++q) {
        const double *vq = V + (size_t)q * n;
        double h = 0.0;
        for (int i = 0; i < n; ++i) h = or_fl(prec, h + or_fl(prec, w[i] * vq[i]));
        H[q + j * ld] = h;
        for (int i = 0; i < n; ++i) w[i] = or_fl(prec, w[i] - or_fl(prec, h * vq[i]));
      }
      double hn2 = 0.0;
      for (int i = 0; i < n; ++i) hn2 = or_fl(prec, hn2 + or_fl(prec, w[i] * w[i]));
      const double hn = or_fl(prec, sqrt(hn2));
      H[j + 1 + j * ld] = hn;
      /* earlier rotations on column j, then the one that zeroes h_{j+1,j} */
      for (int q = 0; q < j; ++q) {
        const double a = H[q + j * ld], b = H[q + 1 + j * ld];
        H[q + j * ld] = or_fl(prec, or_fl(prec, cs[q] * a) + or_fl(prec, sn[q] * b));
        H[q + 1 + j * ld] = or_fl(prec, or_fl(prec, cs[q] * b) - or_fl(prec, sn[q] * a));
      }
      const double a = H[j + j * ld];
      const double den = or_fl(prec, sqrt(or_fl(prec, or_fl(prec, a * a) + or_fl(prec, hn * hn))));
      if (!(den > 0.0)) break; /* singular on the Krylov space: keep k steps */
      cs[j] = or_fl(prec, a / den);
      sn[j] = or_fl(prec, hn / den);
      H[j + j * ld] = den;
      H[j + 1 + j * ld] = 0.0;
      g[j + 1] = -or_fl(prec, sn[j] * g[j]);
      g[j] = or_fl(prec, cs[j] * g[j]);
      k = j + 1;
      if (hn == 0.0) break; /* exact breakdown: the Krylov space is invariant */
      double *vn = V + (size_t)(j + 1) * n;
      for (int i = 0; i < n; ++i) vn[i] = or_fl(prec, w[i] / hn);
    }
    for (int q = k - 1; q >= 0; --q) {
      double s = g[q];
      for (int t = q + 1; t < k; ++t) s = or_fl(prec, s - or_fl(prec, H[q + t * ld] * y[t]));
      y[q] = or_fl(prec, s / H[q + q * ld]);
    }
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int q = 0; q < k; ++q) s = or_fl(prec, s + or_fl(prec, y[q] * V[(size_t)q * n + i]));
      d[i] = s;
    }
  }
  free(V); free(w); free(H); free(cs); free(sn); free(g); free(y);
}

static int or_find(const int32_t *rp, const int32_t *ci, int row, int col) {
  for (int k = rp[row]; k < rp[row + 1]; ++k)
    if (ci[k] == col) return k;
  return -1;
}

/* ILU(0), IKJ order: for each row i and each k < i in its pattern,
 * a_ik /= a_kk, then a_ij -= a_ik a_kj for the j > k present in both rows. */
int or_ilu0(int n, const int32_t *rp, const int32_t *ci, const double *val, double *lu) {
  memcpy(lu, val, sizeof(double) * (size_t)rp[n]);
  for (int i = 0; i < n; ++i) {
    for (int kk = rp[i]; kk < rp[i + 1] && ci[kk] < i; ++kk) {
      int k = ci[kk];
      int dk = or_find(rp, ci, k, k);
      if (dk < 0 || lu[dk] == 0.0) return OR_ENOTSPD;
      lu[kk] /= lu[dk];
      for (int jj = kk + 1; jj < rp[i + 1]; ++jj) {
        int pos = or_find(rp, ci, k, ci[jj]);
        if (pos >= 0) lu[jj] -= lu[kk] * lu[pos];
      }
    }
    int di = or_find(rp, ci, i, i);
    if (di < 0 || !(lu[di] > 0.0)) return OR_ENOTSPD;
  }
  return OR_OK;
}

/* z = U^{-1} L^{-1} r with L unit lower and U upper from the ILU(0) factors,
 * in FP64 or with the factors rounded to FP32 and FP32 arithmetic. */
static void or_ilu0_apply_d(int n, const int32_t *rp, const int32_t *ci, const double *lu,
                            const double *r, double *z) {
  for (int i = 0; i < n; ++i) {
    double s = r[i];
    for (int k = rp[i]; k < rp[i + 1] && ci[k] < i; ++k) s -= lu[k] * z[ci[k]];
    z[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = z[i], dg = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      if (ci[k] > i) s -= lu[k] * z[ci[k]];
      else if (ci[k] == i) dg = lu[k];
    }
    z[i] = s / dg;
  }
}

static void or_ilu0_apply_f(int n, const int32_t *rp, const int32_t *ci, const double *lu,
                            int prec, const float *r, float *z) {
  for (int i = 0; i < n; ++i) {
    float s = r[i];
    for (int k = rp[i]; k < rp[i + 1] && ci[k] < i; ++k) s -= or_round_storage(lu[k], prec) * z[ci[k]];
    z[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    float s = z[i], dg = 0.0f;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      if (ci[k] > i) s -= or_round_storage(lu[k], prec) * z[ci[k]];
      else if (ci[k] == i) dg = or_round_storage(lu[k], prec);
    }
    z[i] = s / dg;
  }
}

/* Preconditioned CG, m steps from d = 0:
 *   z = M^{-1} r; p = z; q = A p; alpha = rz/(p.q); d += alpha p;
 *   r -= alpha q; z = M^{-1} r; rz' = r.z; beta = rz'/rz; p = z + beta p. */
void or_pcg_ilu0(int n, const int32_t *rp, const int32_t *ci, const double *val,
                 const double *lu, const double *rhs, int m, int prec, double *d) {
  if (prec == OR_FP64) {
    double *r = (double *)malloc(sizeof(double) * n);
    double *z = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    double *q = (double *)malloc(sizeof(double) * n);
    double rz = 0.0;
    for (int i = 0; i < n; ++i) { d[i] = 0.0; r[i] = rhs[i]; }
    or_ilu0_apply_d(n, rp, ci, lu, r, z);
    for (int i = 0; i < n; ++i) { p[i] = z[i]; rz += r[i] * z[i]; }
    for (int it = 0; it < m && rz != 0.0; ++it) {
      double pq = 0.0;
      for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) s += val[k] * p[ci[k]];
        q[i] = s;
        pq += p[i] * s;
      }
      double alpha = rz / pq;
      for (int i = 0; i < n; ++i) { d[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
      or_ilu0_apply_d(n, rp, ci, lu, r, z);
      double rz2 = 0.0;
      for (int i = 0; i < n; ++i) rz2 += r[i] * z[i];
      double beta = rz2 / rz;
      for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
      rz = rz2;
    }
    free(r); free(z); free(p); free(q);
  } else {
    float *r = (float *)malloc(sizeof(float) * n);
    float *z = (float *)malloc(sizeof(float) * n);
    float *p = (float *)malloc(sizeof(float) * n);
    float *q = (float *)malloc(sizeof(float) * n);
    float *x = (float *)malloc(sizeof(float) * n);
    float rz = 0.0f;
    for (int i = 0; i < n; ++i) { x[i] = 0.0f; r[i] = (float)rhs[i]; }
    or_ilu0_apply_f(n, rp, ci, lu, prec, r, z);
    for (int i = 0; i < n; ++i) { p[i] = z[i]; rz += r[i] * z[i]; }
    for (int it = 0; it < m && rz != 0.0f; ++it) {
      float pq = 0.0f;
      for (int i = 0; i < n; ++i) {
        float s = 0.0f;
        for (int k = rp[i]; k < rp[i + 1]; ++k) s += or_round_storage(val[k], prec) * p[ci[k]];
        q[i] = s;
        pq += p[i] * s;
      }
      float alpha = rz / pq;
      for (int i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
      or_ilu0_apply_f(n, rp, ci, lu, prec, r, z);
      float rz2 = 0.0f;
      for (int i = 0; i < n; ++i) rz2 += r[i] * z[i];
      float beta = rz2 / rz;
      for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
      rz = rz2;
    }
    for (int i = 0; i < n; ++i) d[i] = (double)x[i];
    free(r); free(z); free(p); free(q); free(x);
  }
}

/* ------------------------------------------------------------------------ */
/* residual and the synchronous RAS iteration                                */
/* ------------------------------------------------------------------------ */

double or_residual(int n, const int32_t *rp, const int32_t *ci, const double *val,
                   const double *b, const double *x, double *r) {
  double s2 = 0.0;
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = rp[i]; k < rp[i + 1]; ++k) s -= val[k] * x[ci[k]];
    if (r) r[i] = s;
    s2 += s * s;
  }
  return s2;
}

typedef struct {
  int no;          /* |Omega_p| */
  int32_t *omega;  /* global ids, ascending */
  uint8_t *owned;  /* owned[t]: omega[t] in O_p */
  int32_t *lrp;    /* A_p = A[Omega_p, Omega_p], local CSR */
  int32_t *lci;
  double *lval;
  int w;           /* half bandwidth of A_p */
  double *band;    /* Cholesky factor (or LU factors, width 2w+1), band layout */
  double *lu;      /* ILU(0) factors on the pattern of A_p */
} or_sub;

static void or_sub_free(or_sub *s) {
  free(s->omega); free(s->owned); free(s->lrp); free(s->lci); free(s->lval);
  free(s->band); free(s->lu);
}

/* Set up subdomain p: overlap maps, local matrix A_p (Sec. 3.2.2) and its
 * factorisation (done once, Sec. 3.3.1). */
static int or_sub_setup(int n, const int32_t *rp, const int32_t *ci, const double *val,
                        const int32_t *part, int P, int p, int gamma, int kind, double alpha,
                        int32_t *g2l, or_sub *s) {
  memset(s, 0, sizeof(*s));
  int32_t *omega = (int32_t *)malloc(sizeof(int32_t) * n);
  uint8_t *owned = (uint8_t *)malloc(n);
  int32_t *iface = (int32_t *)malloc(sizeof(int32_t) * n);
  int32_t no = 0, ni = 0;
  int rc = or_overlap(n, rp, ci, part, P, p, gamma, omega, &no, owned, iface, &ni);
  free(iface);
  if (rc) { free(omega); free(owned); return rc; }
  s->no = no;
  s->omega = omega;
  s->owned = owned;
  for (int t = 0; t < no; ++t) g2l[omega[t]] = t;
  int64_t nnz = 0;
  for (int t = 0; t < no; ++t) {
    int g = omega[t];
    for (int k = rp[g]; k < rp[g + 1]; ++k)
      if (g2l[ci[k]] >= 0) nnz++;
  }
  s->lrp = (int32_t *)malloc(sizeof(int32_t) * (no + 1));
  s->lci = (int32_t *)malloc(sizeof(int32_t) * (nnz > 0 ? nnz : 1));
  s->lval = (double *)malloc(sizeof(double) * (nnz > 0 ? nnz : 1));
  int64_t c = 0;
  int w = 0;
  s->lrp[0] = 0;
  for (int t = 0; t < no; ++t) {
    int g = omega[t];
    for (int k = rp[g]; k < rp[g + 1]; ++k) {
      int l = g2l[ci[k]];
      if (l < 0) continue;
      s->lci[c] = l;
      s->lval[c] = val[k];
      c++;
      int dd = t > l ? t - l : l - t;
      if (dd > w) w = dd;
    }
    s->lrp[t + 1] = (int32_t)c;
  }
  if (alpha != 0.0) {
    /* optimized (Robin-type) interface condition: every exterior neighbour
     * value u_j of row t is replaced by alpha * u_t, i.e. the exterior
     * couplings of the row, times alpha, join its diagonal */
    for (int t = 0; t < no; ++t) {
      int g = omega[t];
      double ext = 0.0;
      for (int k = rp[g]; k < rp[g + 1]; ++k)
        if (g2l[ci[k]] < 0) ext += val[k];
      for (int k = s->lrp[t]; k < s->lrp[t + 1]; ++k)
        if (s->lci[k] == t) s->lval[k] += alpha * ext;
    }
  }
  for (int t = 0; t < no; ++t) g2l[omega[t]] = -1;
  s->w = w;
  if (kind == OR_BANDCHOL) {
    size_t cnt = (size_t)(no > 0 ? no : 1) * (size_t)(w >= 0 ? w + 1 : 1);
    s->band = (double *)calloc(cnt, sizeof(double));
    for (int t = 0; t < no; ++t)
      for (int k = s->lrp[t]; k < s->lrp[t + 1]; ++k)
        if (s->lci[k] <= t) BAND(s->band, w, t, s->lci[k]) = s->lval[k];
    rc = or_band_cholesky(no, w, s->band);
  } else if (kind == OR_BANDLU) {
    size_t cnt = (size_t)(no > 0 ? no : 1) * (size_t)(2 * w + 1);
    s->band = (double *)calloc(cnt, sizeof(double));
    for (int t = 0; t < no; ++t)
      for (int k = s->lrp[t]; k < s->lrp[t + 1]; ++k) BANDG(s->band, w, t, s->lci[k]) = s->lval[k];
    rc = or_band_lu(no, w, s->band);
  } else if (kind == OR_ILU0_CG) {
    s->lu = (double *)malloc(sizeof(double) * (nnz > 0 ? nnz : 1));
    rc = or_ilu0(no, s->lrp, s->lci, s->lval, s->lu);
  }
  return rc;
}

/* delta = A_p^{-1} rhs (exactly, up to rounding) or m steps of (P)CG / GMRES. */
static void or_sub_solve(const or_sub *s, int kind, int prec, int m, double *rhs_delta) {
  if (kind == OR_BANDCHOL) {
    if (prec == OR_FP64) or_band_solve(s->no, s->w, s->band, rhs_delta);
    else or_band_solve_lowp(s->no, s->w, s->band, prec, rhs_delta);
  } else if (kind == OR_BANDLU) {
    if (prec == OR_FP64) or_band_lu_solve(s->no, s->w, s->band, rhs_delta);
    else or_band_lu_solve_lowp(s->no, s->w, s->band, prec, rhs_delta);
  } else {
    double *d = (double *)malloc(sizeof(double) * (s->no > 0 ? s->no : 1));
    if (kind == OR_CG) or_cg(s->no, s->lrp, s->lci, s->lval, rhs_delta, m, prec, d);
    else if (kind == OR_GMRES) or_gmres(s->no, s->lrp, s->lci, s->lval, rhs_delta, m, prec, d);
    else or_pcg_ilu0(s->no, s->lrp, s->lci, s->lval, s->lu, rhs_delta, m, prec, d);
    memcpy(rhs_delta, d, sizeof(double) * s->no);
    free(d);
  }
}

/* Synchronous RAS, correction form. For k = 0, 1, ...:
 *   r = b - A x^k; stop if ||r||^2 < tol^2 ||b||^2 (global criterion);
 *   for every p: delta_p = A_p^{-1} r[Omega_p];
 *                x^{k+1}[i] = x^k[i] + delta_p[i] for i in O_p only
 *   (values computed on the overlap are discarded: the "restricted" rule). */
int or_ras_sync(int n, const int32_t *rp, const int32_t *ci, const double *val, const double *b,
                const int32_t *part, int P, int gamma, int kind, int prec, int m, double tol,
                int max_iter, int nthreads, double *x, double *hist, int32_t *iters) {
  return or_ras_sync_ex(n, rp, ci, val, b, part, P, gamma, kind, prec, m, 0.0, tol, max_iter,
                        nthreads, x, hist, iters);
}

/* The set-up half of Algorithm 1 (initialization_and_setup): overlap maps,
 * local matrices and their factorisations for every subdomain, kept for
 * or_ras_iterate. Time spent here is not part of the solve (Sec. 3.1). */
struct or_ras {
  int n, P, kind, prec, m;
  const int32_t *rp, *ci;
  const double *val;
  or_sub *subs;
};

int or_ras_new(int n, const int32_t *rp, const int32_t *ci, const double *val,
               const int32_t *part, int P, int gamma, int kind, int prec, int m, double alpha,
               or_ras **out) {
  *out = NULL;
  if (n <= 0 || P <= 0 || gamma < 0 || !isfinite(alpha)) return OR_EINVAL;
  if (kind < OR_BANDCHOL || kind > OR_GMRES || prec < OR_FP64 || prec > OR_BF16) return OR_EINVAL;
  if (prec == OR_BF16 && kind != OR_BANDCHOL && kind != OR_BANDLU) return OR_EINVAL;
  for (int i = 0; i < n; ++i)
    if (part[i] < 0 || part[i] >= P) return OR_EINVAL;
  or_ras *h = (or_ras *)calloc(1, sizeof(or_ras));
  h->n = n; h->P = P; h->kind = kind; h->prec = prec; h->m = m;
  h->rp = rp; h->ci = ci; h->val = val;
  h->subs = (or_sub *)calloc(P, sizeof(or_sub));
  int32_t *g2l = (int32_t *)malloc(sizeof(int32_t) * n);
  for (int i = 0; i < n; ++i) g2l[i] = -1;
  int rc = OR_OK;
  for (int p = 0; p < P && rc == OR_OK; ++p)
    rc = or_sub_setup(n, rp, ci, val, part, P, p, gamma, kind, alpha, g2l, &h->subs[p]);
  free(g2l);
  if (rc != OR_OK) {
    or_ras_free(h);
    return rc;
  }
  *out = h;
  return OR_OK;
}

void or_ras_free(or_ras *h) {
  if (!h) return;
  for (int p = 0; p < h->P; ++p) or_sub_free(&h->subs[p]);
  free(h->subs);
  free(h);
}

/* The solve half: synchronous RAS iterations in correction form from x. */
int or_ras_iterate(const or_ras *h, const double *b, double tol, int max_iter, int nthreads,
                   double *x, double *hist, int32_t *iters) {
  if (max_iter < 0) return OR_EINVAL;
  const int n = h->n, P = h->P;
  double *r = (double *)malloc(sizeof(double) * n);
  double *xn = (double *)malloc(sizeof(double) * n);
  double b2 = 0.0;
  for (int i = 0; i < n; ++i) b2 += b[i] * b[i];
  double bn = sqrt(b2);
  int rc = OR_OK, k = 0;
  for (k = 0;; ++k) {
    double r2 = or_residual(n, h->rp, h->ci, h->val, b, x, r);
    if (hist) hist[k] = bn > 0.0 ? sqrt(r2) / bn : sqrt(r2);
    if (r2 < tol * tol * b2) break;
    if (k == max_iter) { rc = OR_ENOCONV; break; }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int p = 0; p < P; ++p) {
      const or_sub *s = &h->subs[p];
      double *loc = (double *)malloc(sizeof(double) * (s->no > 0 ? s->no : 1));
      for (int t = 0; t < s->no; ++t) loc[t] = r[s->omega[t]];
      or_sub_solve(s, h->kind, h->prec, h->m, loc);
      for (int t = 0; t < s->no; ++t)
        if (s->owned[t]) xn[s->omega[t]] = x[s->omega[t]] + loc[t];
      free(loc);
    }
    memcpy(x, xn, sizeof(double) * n);
  }
  *iters = k;
  free(r); free(xn);
  (void)nthreads;
  return rc;
}

int or_ras_sync_ex(int n, const int32_t *rp, const int32_t *ci, const double *val,
                   const double *b, const int32_t *part, int P, int gamma, int kind, int prec,
                   int m, double alpha, double tol, int max_iter, int nthreads, double *x,
                   double *hist, int32_t *iters) {
  *iters = 0;
  if (max_iter < 0) return OR_EINVAL;
  or_ras *h = NULL;
  int rc = or_ras_new(n, rp, ci, val, part, P, gamma, kind, prec, m, alpha, &h);
  if (rc != OR_OK) return rc;
  rc = or_ras_iterate(h, b, tol, max_iter, nthreads, x, hist, iters);
  or_ras_free(h);
  return rc;
}
