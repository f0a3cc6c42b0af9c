// Internal data layout shared by the host setup code and the device kernels.
//
// Device-side layout of one context (one linear system, P subdomains):
//   * per-subdomain descriptors SubDesc[P] and runtime state SubState[P];
//   * per-local-row arrays concatenated over subdomains, each subdomain padded
//     to a multiple of 32 rows (npad): gidx (global id of local row i),
//     ownf (1 when the row is owned, i.e. in O_p);
//   * the residual operator of Omega_p's rows in ELL form with GLOBAL columns
//     (rcol/rval, K entries per row, column-major inside a subdomain:
//     entry k of local row i at row_off*K + k*npad + i). It computes
//     r_p = b[Omega_p] - A[Omega_p, :] x, reading x on Omega_p and E_p;
//   * the owned-row list own_l (local ids);
//   * local-solver data: banded-Cholesky or banded-LU block records (fac), or the
//     local matrix A_p in ELL form with LOCAL columns (lcol/lval) plus ILU(0)
//     factors (luval) and level schedules, or the GMRES Krylov basis scratch.
#pragma once
#include <stdint.h>

namespace ras {

// kernel variants: kBand runs the banded triangular solves of both banded
// factorisations (Cholesky and LU share the record layout); kCGS is CG with
// A_p staged in shared memory
enum LocalKind : int32_t { kBand = 0, kCG = 1, kILU = 2, kCGS = 3, kGMRES = 4 };
enum Prec : int32_t { kF64 = 0, kF32 = 1, kBF16 = 2 };
enum Mode : int32_t { kSync = 0, kAsync = 1, kAsyncDecentral = 2 };
// status codes (mirror ras_status)
enum : int32_t { kOK = 0, kEINVAL = 1, kENOMEM = 2, kENOTSPD = 3, kENOCONV = 4, kETIMEOUT = 5,
                 kECUDA = 6, kENOTSUP = 7 };
// async per-system phases
enum : int32_t { kRun = 0, kDrain = 1, kCheck = 2, kDone = 3 };

#ifdef __CUDACC__
#define RAS_HD __host__ __device__
#else
#define RAS_HD
#endif

struct SubDesc {
  int32_t n;        // |Omega_p|
  int32_t npad;     // n rounded up to a multiple of 32
  int32_t n_own;    // |O_p|
  int32_t W;        // band: half-bandwidth w rounded up to a multiple of 4 (>= 4)
  int64_t row_off;  // offset of local row 0 in the per-row arrays (multiple of 32)
  int64_t own_off;  // offset into own_l
  int64_t fac_off;  // band: nb forward records, then nb backward records (32 x (W+32) each)
                    // (forward from L, backward from U = L^T (Cholesky) or U (LU))
  int64_t lev_off;  // ILU: offset into lev_ptr (forward levels, then backward)
  int64_t lrow_off; // ILU: offset into lev_rows (n forward rows, then n backward)
  int32_t nlev_f;   // ILU: number of forward / backward levels
  int32_t nlev_b;
  int32_t nbr_off;  // neighbour subdomains (system-local ids) in nbr[]
  int32_t n_nbr;
  int32_t tnbr_off;  // neighbours in a spanning tree of the subdomain graph (tnbr[])
  int32_t n_tnbr;
  // local rows on a grid box (SysDesc::grid > 0): box point (x, y, z) is
  // local row x + y bx + z bxy and global id g0 + x + y gs2 + z gs3
  int32_t g0;
  int32_t bx;
  int32_t bxy;
  int32_t pad_;
};

struct SubState {
  double bloc2;       // ||b||^2 over Omega_p (local criterion, Eq. 2)
  double bown2;       // ||b||^2 over O_p
  double part[2];     // owned-row residual^2 partials
  int64_t updates;    // local solves in the current solve
  int64_t step_updates;  // local solves in the current launch
  int64_t stale;      // async: solves that saw no new neighbour data
  uint64_t t_gather;  // accumulated ns in the residual gather
  uint64_t t_solve;   // accumulated ns in the local solve
  uint64_t t_update;  // accumulated ns in the restricted update + publish
  uint64_t nbr_seen;  // async: sum of neighbour versions at the last solve
  uint32_t version;   // async: 2 x published updates (release store); odd while the
                      // owned rows are being written (a sequence lock for readers)
  int32_t conv_epoch; // async: epoch in which Eq. 2 last held (-1: not converged)
  int32_t park_epoch;
  int32_t check_epoch;
  int32_t gconv_epoch;  // decentralized detection: epoch of the global flag (-1: none)
  uint32_t busy;        // async, dynamic schedule: 1 while a CTA holds the subdomain
  unsigned long long report;  // decentralized detection: (epoch << 32) | tree neighbour
                              // the convergence report was sent to (epoch -1: none)
};

struct SysState {
  double b2;          // ||b||^2
  double res2;        // last global residual^2
  int64_t iters;      // sync: completed RAS iterations
  uint32_t word;      // async: (epoch << 2) | phase
  int32_t status;
  int32_t done;       // sync: finished (converged or failed)
  int32_t nconv;      // async counters
  int32_t nparked;
  int32_t nchecked;
  int32_t restarts;
  int32_t result_alt; // sync: result left in xalt (copied back by the epilogue)
};

struct SysDesc {
  const double *b;
  double *x;     // initial guess in, result out
  double *xalt;  // sync double buffer
  int32_t n;
  int32_t P;
  int32_t K;     // ELL width
  // 2 or 3: A is a 2D / 3D stencil in lexicographic order (global strides
  // gs2, gs3) and every subdomain's local rows lie on a grid box (SubDesc g0,
  // bx, bxy; hole rows flagged in ownf); rcol / rval then hold each row's
  // entries in slot order: the diagonal, then the global offsets -gs3, -gs2,
  // -1, 1, gs2, gs3 (2D: without +-gs3), a missing entry as column g and
  // value 0. 0: the general layout
  int32_t grid;
  double tol2;
  const SubDesc *subs;
  SubState *sub;
  SysState *st;
  const int32_t *gidx;
  // per local row: 1 owned (O_p), 0 overlap, 2 hole row (local rows laid out
  // on a grid box: no point of Omega_p, residual and values zero)
  const uint8_t *ownf;
  const int32_t *rcol;
  const double *rval;
  const int32_t *own_l;
  const int32_t *own_g;  // global index of each owned row (same order as own_l)
  double *xg;    // per local row: the x value the last gather used (owned rows)
  const void *fac;
  const int32_t *lcol;
  const int16_t *lcol16;  // local columns as int16 (staged CG)
  // staged CG, paired layout (odd ELL width K, diagonal first): per subdomain
  // the K npad values are the diagonal, then (K-1)/2 blocks of npad value pairs
  // (entries 1+2q and 2+2q of a row); cpair holds the matching column pairs as
  // two int16 in one 32-bit word. Null when the plain ELL form is used.
  const float *vpair;
  const uint32_t *cpair;
  // staged CG, diagonal-offset form (grid > 0, largest local offset, bx in
  // 2D and bxy in 3D, at most kDiaMargin): per
  // subdomain K arrays of npad values of A_p, the diagonal first, then one
  // array per local offset -bxy, -bx, -1, 1, bx, bxy (2D: without +-bxy; zero
  // where a row has no entry in Omega_p there, unused slots zero with offset
  // 0). The kernel reads r[i + offset] and needs no column indices. Null
  // otherwise.
  const float *vdia;
  const void *lval;
  // ILU(0) factors in level order: forward sweep row e (lev_rows, forward
  // part) has its strictly lower entries at ilu_fcol / ilu_fval[k*npad + e]
  // (k < ilu_kl, column -1 = none), backward sweep row e its strictly upper
  // entries at ilu_bcol / ilu_bval[k*npad + e] (k < ilu_ku) and its diagonal
  // at ilu_bdiag[e]; per subdomain from row_off * ilu_kl, row_off * ilu_ku,
  // row_off. Values in the storage precision.
  const int32_t *ilu_fcol;
  const void *ilu_fval;
  const int32_t *ilu_bcol;
  const void *ilu_bval;
  const void *ilu_bdiag;
  int32_t ilu_kl, ilu_ku;
  const int32_t *lev_ptr;
  const int32_t *lev_rows;
  const int32_t *nbr;
  const int32_t *tnbr;  // spanning-tree neighbours (decentralized detection)
  // GMRES: Krylov basis scratch in the local-solve precision, kry_ld vectors
  // of npad entries per subdomain from row_off * kry_ld (vector q of local
  // row i at row_off * kry_ld + q * npad + i); kry_ld - 1 bounds the steps
  void *kry;
  int32_t kry_ld;
  int32_t gs2;  // grid strides (grid > 0)
  int32_t gs3;
  int32_t pad2_;
};

struct Item {
  int32_t sys;  // system index in the launch
  int32_t p;    // subdomain id within the system
  int32_t ls;   // index of `sys` in the owning CTA's system list
  int32_t pad_;
};

constexpr int kMaxCtaSys = 64;  // distinct systems per CTA in one launch
constexpr int kMaxEll = 8;      // ELL widths up to this are fully unrolled
constexpr int kIluHalf = 4;     // ILU(0): strictly lower / upper entries per row kept in registers
constexpr int kStagedRows = 6144;  // largest subdomain of the staged CG variant
constexpr int kRegRows = 11;       // staged diagonal-offset CG: rows per thread with r in registers
constexpr int kDiaMargin = 512;    // staged CG, diagonal-offset form: largest |offset|
                                   // (zero margins of this many values around r)
constexpr int kMaxBandW = 160;     // banded Cholesky: largest half-bandwidth
constexpr int kMaxBandLuW = 112;   // banded LU: largest half-bandwidth (factorisation window
                                   // of (w+1) x (2w+1) FP64 values in shared memory)
constexpr int kMaxGmres = 32;      // GMRES: most Arnoldi steps per local solve

struct GridCtl {
  unsigned int count;  // barrier arrivals
  unsigned int gen;    // barrier generation
  int fin_accum;       // systems finished since the last barrier
  int remaining;       // systems still running (sync: published by the barrier;
                       // async: decremented when a system finishes)
  int abort;           // set on any device-side error
  int status;          // first error code
  unsigned long long err_info;
  unsigned long long ticket;  // async, dynamic schedule: next ticket
};

struct Launch {
  SysDesc *sys;
  int32_t nsys;
  int32_t mode;
  const Item *items;
  const int32_t *cta_off;      // [G+1]
  const int32_t *cta_sys;      // distinct systems per CTA (sync decisions)
  const int32_t *cta_sys_off;  // [G+1]
  GridCtl *ctl;
  int64_t max_updates;         // per subdomain (async) / iterations (sync)
  int64_t step_limit;          // local updates (async) or iterations (sync) in this launch
  int64_t timeout_ns;          // limit on any device-side wait
  int64_t solve_limit_ns;      // limit on the whole launch (then RAS_ETIMEOUT)
  int32_t max_restarts;
  int32_t m;                   // CG / PCG steps
  int32_t Wmax;                // band: max W over the launch
  int32_t npad_max;
  int32_t persist;             // async: keep polling until every system is done
  int32_t kmax;                // largest ELL width over the launch
  int32_t nstages;             // band: copy pipeline depth in chain steps (4 or 6)
  int32_t fresh;               // async: update only after a neighbour published since the last update
  int32_t consistent;          // async: redo a gather that overlapped a neighbour's write (<= 2 times)
  int32_t dynamic;             // async, persistent: CTAs take items by ticket (no static assignment)
  int32_t nitems;              // items in the launch
  int32_t pad4_;
};

}  // namespace ras
