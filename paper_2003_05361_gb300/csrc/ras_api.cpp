// Host side of the GB300 RAS solver: the C ABI of include/ras.h.
//
//   * partitioners (Sec. 3.2.1): regular2d and the seeded BFS-growth graph
//     partitioner that stands in for Metis;
//   * the overlap / restriction-map builder (Sec. 2.1, Fig. 1; Sec. 3.2.2):
//     Omega_p = O_p grown by `overlap` layers of graph neighbours, the
//     external interface E_p, the local matrix A_p and the residual operator
//     of Omega_p's rows;
//   * local-solver setup (Sec. 3.3.1): banded Cholesky on the GPU, or ILU(0)
//     factors and level schedules for the preconditioned CG;
//   * launch planning (CTA count from occupancy, longest-processing-time
//     assignment of subdomains to CTAs) and the solve / batch-solve drivers
//     (Algorithm 1's solve loop runs inside one cooperative launch).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <memory>
#include <numeric>
#include <queue>
#include <thread>
#include <type_traits>
#include <vector>

#include "../../include/ras.h"
#include "ras_internal.h"
#include "ras_launch.h"

using namespace ras;

namespace {

// ---------------------------------------------------------------- utilities

int host_threads() {
  unsigned h = std::thread::hardware_concurrency();
  if (h == 0) h = 4;
  return (int)std::min(16u, h);
}

// Runs f(p) for p in [0, n) on a few host threads.
void parallel_for(int n, const std::function<void(int)> &f) {
  const int nt = std::min(host_threads(), std::max(n, 1));
  if (nt <= 1) {
    for (int p = 0; p < n; ++p) f(p);
    return;
  }
  std::atomic<int> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&]() {
      for (int p; (p = next.fetch_add(1)) < n;) f(p);
    });
  for (auto &t : th) t.join();
}

uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  // SplitMix64 (Steele, Lea & Flood 2014): state advanced k+1 times by the
  // golden-ratio increment, then the variant-13 finaliser.
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double unit_double(uint64_t z) { return (double)(z >> 11) * 0x1.0p-53; }

ras_status check_csr(const ras_csr *A) {
  if (!A || A->n <= 0 || !A->row_ptr || !A->col_idx || !A->val) return RAS_EINVAL;
  const int n = A->n;
  if (A->row_ptr[0] != 0 || (int64_t)A->row_ptr[n] != A->nnz) return RAS_EINVAL;
  for (int i = 0; i < n; ++i) {
    const int a = A->row_ptr[i], b = A->row_ptr[i + 1];
    if (b < a) return RAS_EINVAL;
    bool diag = false;
    for (int k = a; k < b; ++k) {
      const int c = A->col_idx[k];
      if (c < 0 || c >= n) return RAS_EINVAL;
      if (k > a && c <= A->col_idx[k - 1]) return RAS_EINVAL;
      if (c == i) diag = true;
      if (!std::isfinite(A->val[k])) return RAS_EINVAL;
    }
    if (!diag) return RAS_EINVAL;
  }
  // structural symmetry: (i, c) present => (c, i) present
  for (int i = 0; i < n; ++i)
    for (int k = A->row_ptr[i]; k < A->row_ptr[i + 1]; ++k) {
      const int c = A->col_idx[k];
      const int32_t *b = A->col_idx + A->row_ptr[c], *e = A->col_idx + A->row_ptr[c + 1];
      if (!std::binary_search(b, e, i)) return RAS_EINVAL;
    }
  return RAS_OK;
}

#define CUDA_TRY(expr)                                 \
  do {                                                 \
    cudaError_t e_ = (expr);                           \
    if (e_ != cudaSuccess) {                           \
      last_cuda_error() = e_;                          \
      return e_ == cudaErrorMemoryAllocation ? RAS_ENOMEM : RAS_ECUDA; \
    }                                                  \
  } while (0)

cudaError_t &last_cuda_error() {
  static thread_local cudaError_t e = cudaSuccess;
  return e;
}

int64_t env_int(const char *name, int64_t dflt) {
  const char *v = std::getenv(name);
  if (!v || !*v) return dflt;
  return std::strtoll(v, nullptr, 10);
}

// Host-side fault injection for the allocation-failure paths (nothing
// reaches the GPU): with RAS_FAULT_ALLOC=k (k >= 1) in the environment, the
// k-th device or pinned-host allocation counted on this thread since the
// start of the current ras_setup reports cudaErrorMemoryAllocation without
// allocating. Unset or 0: every call goes to the CUDA runtime.
thread_local int64_t t_alloc_count = 0;
bool inject_alloc_failure() {
  const int64_t k = env_int("RAS_FAULT_ALLOC", 0);
  return k > 0 && ++t_alloc_count == k;
}
cudaError_t dev_malloc(void **p, size_t bytes) {
  if (inject_alloc_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}
template <typename T> cudaError_t dev_malloc(T **p, size_t bytes) {
  return dev_malloc(reinterpret_cast<void **>(p), bytes);
}
template <typename T> cudaError_t host_malloc_pinned(T **p, size_t bytes) {
  if (inject_alloc_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(reinterpret_cast<void **>(p), bytes);
}

// A temporary device buffer freed when it goes out of scope (setup paths
// that return early on an error).
struct TmpDev {
  void *p = nullptr;
  ~TmpDev() {
    if (p) cudaFree(p);
  }
};

}  // namespace

// ---------------------------------------------------------------- context

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

struct LaunchPlan {
  int nt = 0, grid = 0, kmax = 0, nstages = 4;
  int grid_dyn = 0;  // CTAs of the dynamic asynchronous schedule (all co-resident slots)
  size_t smem = 0;
  int Wmax = 0, npad_max = 0;
  std::vector<Item> items;
  std::vector<int32_t> cta_off, cta_sys, cta_sys_off;
  // device copies
  Item *d_items = nullptr;
  int32_t *d_cta_off = nullptr, *d_cta_sys = nullptr, *d_cta_sys_off = nullptr;
  void release() {
    cudaFree(d_items);
    cudaFree(d_cta_off);
    cudaFree(d_cta_sys);
    cudaFree(d_cta_sys_off);
    d_items = nullptr;
    d_cta_off = d_cta_sys = d_cta_sys_off = nullptr;
  }
};

struct ras_ctx {
  cudaStream_t stream = nullptr;
  int n = 0, P = 0, K = 0, overlap = 0;
  ras_local_solver ls{};
  int maxw = 0;  // largest true local half-bandwidth
  int exec_kind = 0;  // kernel variant (LocalKind; kCGS for staged FP32 CG)
  int nt_pref = 0;    // preferred CTA threads of the CG / ILU variants (0: default)
  int sched = -1;     // schedule: -1 RAS_ASYNC_DYNAMIC / RAS_SYNC_DYNAMIC (default
                      // dynamic), 0 static assignment, 1 dynamic (tickets)
  int grid_cap = 0;   // cap on the CTAs of a launch (0: every co-resident slot); with the
                      // static assignment it sets the subdomains per CTA
  // host copies of the maps (inspection)
  std::vector<std::vector<int32_t>> omega, iface;
  std::vector<std::vector<uint8_t>> owned;
  std::vector<SubDesc> subs;
  std::vector<double> cost;  // per-subdomain work estimate for the launch plan
  // device data
  std::vector<DevBuf> bufs;
  SubDesc *d_subs = nullptr;
  SubState *d_sub = nullptr;
  SysState *d_st = nullptr;
  int16_t *d_lcol16 = nullptr;
  float *d_vpair = nullptr;     // staged CG, paired layout
  uint32_t *d_cpair = nullptr;
  float *d_vdia = nullptr;      // staged CG, diagonal-offset form
  bool dia = false;
  int grid = 0;                 // SysDesc::grid, gs2, gs3
  int32_t gs2 = 0, gs3 = 0;
  int32_t *d_own_g = nullptr;
  int32_t *d_gidx = nullptr, *d_rcol = nullptr, *d_own = nullptr, *d_lcol = nullptr,
          *d_levp = nullptr, *d_levr = nullptr, *d_nbr = nullptr, *d_tnbr = nullptr;
  uint8_t *d_ownf = nullptr;
  double *d_rval = nullptr, *d_xalt = nullptr, *d_xg = nullptr;
  void *d_fac = nullptr, *d_lval = nullptr;
  int32_t *d_ifc = nullptr, *d_ibc = nullptr;  // ILU(0) factors in level order
  void *d_ifv = nullptr, *d_ibv = nullptr, *d_ibd = nullptr;
  int32_t ilu_kl = 0, ilu_ku = 0;
  void *d_kry = nullptr;  // GMRES Krylov basis scratch
  int32_t kry_ld = 0;
  int64_t device_bytes = 0;
  // launch state
  LaunchPlan plan;
  SysDesc *d_sysdesc = nullptr;
  GridCtl *d_ctl = nullptr;
  SysDesc *h_sysdesc = nullptr;  // pinned staging
  GridCtl *h_ctl = nullptr;
  SysState *h_st = nullptr;
  SubState *h_sub = nullptr;
  double *d_bx = nullptr;  // device b and x for ras_solve_host
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evk0 = nullptr, evk1 = nullptr, ev_begin = nullptr;
  bool begun = false, finished = false;  // continuous-batching state
  uint64_t serial = next_serial();       // identity that survives address reuse
  static uint64_t next_serial() {
    static std::atomic<uint64_t> n(1);
    return n.fetch_add(1);
  }
  std::vector<int64_t> last_updates;
  std::vector<uint64_t> last_phase;  // 3 per subdomain: gather, solve, update ns

  template <typename T>
  ras_status alloc(T *&ptr, size_t count) {
    void *p = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = dev_malloc(&p, bytes);
    if (e != cudaSuccess) {
      last_cuda_error() = e;
      return RAS_ENOMEM;
    }
    bufs.push_back({p, bytes});
    device_bytes += (int64_t)bytes;
    ptr = static_cast<T *>(p);
    return RAS_OK;
  }
  template <typename T>
  ras_status upload(T *&ptr, const std::vector<T> &v) {
    ras_status s = alloc(ptr, v.size());
    if (s != RAS_OK) return s;
    if (!v.empty()) {
      cudaError_t e = cudaMemcpyAsync(ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice,
                                      stream);
      if (e != cudaSuccess) {
        last_cuda_error() = e;
        return RAS_ECUDA;
      }
    }
    return RAS_OK;
  }
  ~ras_ctx() {
    cudaStreamSynchronize(stream);
    plan.release();
    for (auto &b : bufs) cudaFree(b.p);
    cudaFreeHost(h_sysdesc);
    cudaFreeHost(h_ctl);
    cudaFreeHost(h_st);
    cudaFreeHost(h_sub);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (evk0) cudaEventDestroy(evk0);
    if (evk1) cudaEventDestroy(evk1);
    if (ev_begin) cudaEventDestroy(ev_begin);
  }
};

namespace {

size_t prec_bytes(int prec) { return prec == RAS_FP64 ? 8 : prec == RAS_FP32 ? 4 : 2; }

// Write value v in the storage precision at dst[k].
void store_prec(void *dst, size_t k, int prec, double v) {
  if (prec == RAS_FP64) {
    static_cast<double *>(dst)[k] = v;
  } else if (prec == RAS_FP32) {
    static_cast<float *>(dst)[k] = (float)v;
  } else {
    // bfloat16, round to nearest even from the float32 value
    float f = (float)v;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    static_cast<uint16_t *>(dst)[k] = (uint16_t)(u >> 16);
  }
}

// Per-subdomain maps built on the host.
struct SubMaps {
  std::vector<int32_t> omega;   // ascending global ids
  std::vector<uint8_t> owned;
  std::vector<int32_t> iface;   // ascending
  std::vector<int32_t> nbr;     // neighbouring subdomains (ascending, != p)
  int w = 0;                    // half-bandwidth of A_p in local order
  // local rows on a grid box (grid_embed): global id of local row i, -1 for
  // an inert hole row, and the local row of omega[t]; empty: row i = omega[i]
  std::vector<int32_t> slot_g, slot_of;
  int dims = 0;                 // grid dimension seen from Omega_p's rows (2, 3)
  int64_t s2 = 0, s3 = 0;       // global strides of y and z
  int32_t g0 = 0, bx = 0, bxy = 0;  // box origin (global id), row and plane lengths
};

// Lays the local rows of Omega_p out on the bounding box of Omega_p in grid
// coordinates when A is a 2D or 3D stencil in lexicographic order: the
// distinct distances |c - g| of the entries of Omega_p's rows are 1, s2 (and
// s3) with s2 | s3, and each entry moves one unit along one axis of
// x = g mod s2, y = (g / s2) mod (s3 / s2), z = g / s3. Local row
// ((z - z0) Wy + (y - y0)) Wx + (x - x0) then keeps the order of the global
// ids, and every entry of A_p sits at one of the fixed local offsets +-1,
// +-Wx, +-Wx Wy; box points outside Omega_p become hole rows (the corners
// that the breadth-first overlap leaves out). Returns false (m unchanged)
// when the pattern is not such a stencil, or the box has more than
// max_rows rows or over 1.25 |Omega_p|.
bool grid_embed(const ras_csr *A, SubMaps &m, int max_rows) {
  std::vector<int64_t> dist;
  for (int g : m.omega)
    for (int k = A->row_ptr[g]; k < A->row_ptr[g + 1]; ++k) {
      const int64_t d = std::abs((int64_t)A->col_idx[k] - g);
      if (d != 0 && std::find(dist.begin(), dist.end(), d) == dist.end()) {
        if (dist.size() == 3) return false;
        dist.push_back(d);
      }
    }
  std::sort(dist.begin(), dist.end());
  if (dist.size() < 2 || dist[0] != 1) return false;  // 1D: Omega_p is already contiguous
  const bool three = dist.size() == 3;
  const int64_t s2 = dist[1], s3 = three ? dist[2] : 0;
  if (three && s3 % s2 != 0) return false;
  auto coord = [&](int64_t g, int64_t *x) {
    x[0] = g % s2;
    x[1] = three ? (g / s2) % (s3 / s2) : g / s2;
    x[2] = three ? g / s3 : 0;
  };
  int64_t lo[3] = {INT64_MAX, INT64_MAX, INT64_MAX}, hi[3] = {-1, -1, -1}, a[3], b[3];
  for (int g : m.omega) {
    coord(g, a);
    for (int q = 0; q < 3; ++q) {
      lo[q] = std::min(lo[q], a[q]);
      hi[q] = std::max(hi[q], a[q]);
    }
    for (int k = A->row_ptr[g]; k < A->row_ptr[g + 1]; ++k) {
      coord(A->col_idx[k], b);
      int64_t moved = 0;
      for (int q = 0; q < 3; ++q) moved += std::abs(b[q] - a[q]);
      if (moved > 1) return false;  // wraps around a grid line or plane
    }
  }
  const int64_t wx = hi[0] - lo[0] + 1, wy = hi[1] - lo[1] + 1, wz = hi[2] - lo[2] + 1;
  const int64_t box = wx * wy * wz, n = (int64_t)m.omega.size();
  if (box > max_rows || 4 * box > 5 * n) return false;
  // every box point, holes included, must be a row of A
  if (hi[0] + hi[1] * s2 + hi[2] * s3 >= A->n) return false;
  m.dims = three ? 3 : 2;
  m.s2 = s2;
  m.s3 = s3;
  m.g0 = (int32_t)(lo[0] + lo[1] * s2 + lo[2] * s3);
  m.bx = (int32_t)wx;
  m.bxy = (int32_t)(wx * wy);
  m.slot_g.assign(box, -1);
  m.slot_of.resize(n);
  for (int64_t t = 0; t < n; ++t) {
    coord(m.omega[t], a);
    const int64_t sl = ((a[2] - lo[2]) * wy + (a[1] - lo[1])) * wx + (a[0] - lo[0]);
    m.slot_g[sl] = m.omega[t];
    m.slot_of[t] = (int32_t)sl;
  }
  return true;
}

// Omega_p by breadth-first layers from O_p over the graph of A (Fig. 1: one
// layer per unit of overlap); E_p = points outside Omega_p adjacent to it.
void build_maps(const ras_csr *A, const int32_t *part, const std::vector<int32_t> &owned_list,
                int p, int overlap, std::vector<int32_t> &mark, SubMaps &m) {
  const int tag = 2 * p + 1;  // mark[] == tag: in Omega_p; == tag+1: in E_p
  std::vector<int32_t> frontier(owned_list), next, all(owned_list);
  for (int v : owned_list) mark[v] = tag;
  for (int layer = 0; layer < overlap; ++layer) {
    next.clear();
    for (int v : frontier)
      for (int k = A->row_ptr[v]; k < A->row_ptr[v + 1]; ++k) {
        const int c = A->col_idx[k];
        if (mark[c] != tag) {
          mark[c] = tag;
          next.push_back(c);
        }
      }
    all.insert(all.end(), next.begin(), next.end());
    frontier.swap(next);
  }
  std::sort(all.begin(), all.end());
  m.omega = all;
  m.owned.resize(all.size());
  for (size_t t = 0; t < all.size(); ++t) m.owned[t] = part[all[t]] == p ? 1 : 0;
  m.iface.clear();
  for (int v : all)
    for (int k = A->row_ptr[v]; k < A->row_ptr[v + 1]; ++k) {
      const int c = A->col_idx[k];
      if (mark[c] != tag && mark[c] != tag + 1) {
        mark[c] = tag + 1;
        m.iface.push_back(c);
      }
    }
  std::sort(m.iface.begin(), m.iface.end());
  std::vector<int32_t> nb;
  for (int v : all)
    if (part[v] != p) nb.push_back(part[v]);
  for (int v : m.iface) nb.push_back(part[v]);
  std::sort(nb.begin(), nb.end());
  nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
  m.nbr = nb;
  // half-bandwidth in local (ascending global) order
  int w = 0;
  for (size_t i = 0; i < all.size(); ++i) {
    const int g = all[i];
    for (int k = A->row_ptr[g]; k < A->row_ptr[g + 1]; ++k) {
      auto it = std::lower_bound(all.begin(), all.end(), A->col_idx[k]);
      if (it != all.end() && *it == A->col_idx[k]) w = std::max(w, std::abs((int)(it - all.begin()) - (int)i));
    }
  }
  m.w = w;
}

inline int local_index(const std::vector<int32_t> &omega, int g) {
  auto it = std::lower_bound(omega.begin(), omega.end(), g);
  return (it != omega.end() && *it == g) ? (int)(it - omega.begin()) : -1;
}

// ILU(0) of a local CSR matrix (FP64), row by row: for each k < i in row i,
// l_ik = a_ik / u_kk, then a_ij -= l_ik u_kj for every j > k of row k that is
// also in row i (positions found through a scatter map of row i).
bool ilu0_local(int n, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci,
                std::vector<double> &a) {
  std::vector<int32_t> pos(n, -1), diag(n, -1);
  for (int i = 0; i < n; ++i)
    for (int k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] == i) diag[i] = k;
  for (int i = 0; i < n; ++i) {
    for (int k = rp[i]; k < rp[i + 1]; ++k) pos[ci[k]] = k;
    for (int kk = rp[i]; kk < rp[i + 1]; ++kk) {
      const int k = ci[kk];
      if (k >= i) break;
      const double ukk = a[diag[k]];
      if (ukk == 0.0) return false;
      const double lik = a[kk] / ukk;
      a[kk] = lik;
      for (int jj = diag[k] + 1; jj < rp[k + 1]; ++jj) {
        const int q = pos[ci[jj]];
        if (q >= 0) a[q] -= lik * a[jj];
      }
    }
    for (int k = rp[i]; k < rp[i + 1]; ++k) pos[ci[k]] = -1;
    if (!(a[diag[i]] > 0.0)) return false;
  }
  return true;
}

// Level sets of the unit-lower (forward) and upper (backward) triangular
// solves: level(i) = 1 + max level of the rows it depends on.
void level_schedule(int n, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci,
                    std::vector<int32_t> &ptr_f, std::vector<int32_t> &rows_f,
                    std::vector<int32_t> &ptr_b, std::vector<int32_t> &rows_b) {
  std::vector<int32_t> lev(n, 0);
  auto bucket = [&](std::vector<int32_t> &ptr, std::vector<int32_t> &rows) {
    const int nl = n ? *std::max_element(lev.begin(), lev.end()) + 1 : 0;
    ptr.assign(nl + 1, 0);
    for (int i = 0; i < n; ++i) ptr[lev[i] + 1]++;
    for (int l = 0; l < nl; ++l) ptr[l + 1] += ptr[l];
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    rows.assign(n, 0);
    for (int i = 0; i < n; ++i) rows[fill[lev[i]]++] = i;
  };
  for (int i = 0; i < n; ++i) {
    int l = 0;
    for (int k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] < i) l = std::max(l, lev[ci[k]] + 1);
    lev[i] = l;
  }
  bucket(ptr_f, rows_f);
  for (int i = n - 1; i >= 0; --i) {
    int l = 0;
    for (int k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] > i) l = std::max(l, lev[ci[k]] + 1);
    lev[i] = l;
  }
  bucket(ptr_b, rows_b);
}

// Longest-processing-time assignment of items to `grid` CTAs.
void assign_items(LaunchPlan &pl, const std::vector<Item> &items, const std::vector<double> &cost,
                  int grid) {
  const int ni = (int)items.size();
  std::vector<int> order(ni);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<std::vector<int>> per(grid);
  std::vector<std::vector<int>> sys_of(grid);
  using E = std::pair<double, int>;
  std::priority_queue<E, std::vector<E>, std::greater<E>> pq;
  for (int c = 0; c < grid; ++c) pq.push({0.0, c});
  std::vector<E> held;
  for (int idx : order) {
    const int s = items[idx].sys;
    // least-loaded CTA that can still take this item's system
    held.clear();
    int chosen = -1;
    while (!pq.empty()) {
      E e = pq.top();
      pq.pop();
      auto &ss = sys_of[e.second];
      if ((int)ss.size() < kMaxCtaSys || std::find(ss.begin(), ss.end(), s) != ss.end()) {
        chosen = e.second;
        per[chosen].push_back(idx);
        if (std::find(ss.begin(), ss.end(), s) == ss.end()) ss.push_back(s);
        pq.push({e.first + cost[idx], chosen});
        break;
      }
      held.push_back(e);
    }
    for (auto &e : held) pq.push(e);
    if (chosen < 0) {  // cannot happen while grid * kMaxCtaSys >= systems
      per[0].push_back(idx);
    }
  }
  pl.items.clear();
  pl.cta_off.assign(1, 0);
  pl.cta_sys.clear();
  pl.cta_sys_off.assign(1, 0);
  for (int c = 0; c < grid; ++c) {
    auto &v = per[c];
    std::sort(v.begin(), v.end(), [&](int a, int b) {
      return items[a].sys != items[b].sys ? items[a].sys < items[b].sys : items[a].p < items[b].p;
    });
    std::vector<int> sl;
    for (int idx : v) {
      Item it = items[idx];
      auto f = std::find(sl.begin(), sl.end(), it.sys);
      if (f == sl.end()) {
        sl.push_back(it.sys);
        f = sl.end() - 1;
      }
      it.ls = (int)(f - sl.begin());
      pl.items.push_back(it);
    }
    for (int s : sl) {
      bool lead = false;
      for (int idx : v)
        if (items[idx].sys == s && items[idx].p == 0) lead = true;
      pl.cta_sys.push_back(s);
      pl.cta_sys.push_back(lead ? 1 : 0);
    }
    pl.cta_off.push_back((int32_t)pl.items.size());
    pl.cta_sys_off.push_back((int32_t)(pl.cta_sys.size() / 2));
  }
}

ras_status plan_launch(LaunchPlan &pl, int kind, int prec, const std::vector<Item> &items,
                       const std::vector<double> &cost, int Wmax, int npad_max, int kmax,
                       cudaStream_t stream, int nt_pref = 0, int grid_cap = 0) {
  pl.release();
  int dev = 0, nsm = 0, max_smem = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (nt_pref <= 0) nt_pref = (int)env_int("RAS_CTA_THREADS", 0);  // 0: per-kind default
  pl.nt = main_threads(kind, prec, nt_pref);
  pl.Wmax = Wmax;
  pl.npad_max = npad_max;
  pl.kmax = kmax;
  // band: copy pipeline depth (chain steps in flight), reduced until the
  // shared memory fits, and down to 3 when that lets two CTAs share an SM
  // band: copy pipeline depth (chain steps in flight, 6 or 4): 4 when 6 does
  // not fit, or when 4 lets more CTAs share an SM and there are subdomains
  // enough to use them
  pl.nstages = env_int("RAS_BAND_STAGES", 6) >= 6 ? 6 : 4;
  pl.smem = main_smem_bytes(kind, prec, pl.nt, Wmax, npad_max, kmax, pl.nstages);
  if (kind == kBand && pl.nstages == 6 && pl.smem + 4096 > (size_t)max_smem) {
    pl.nstages = 4;
    pl.smem = main_smem_bytes(kind, prec, pl.nt, Wmax, npad_max, kmax, pl.nstages);
  }
  if (pl.smem + 4096 > (size_t)max_smem) return RAS_ENOTSUP;
  int occ = main_occupancy(kind, prec, pl.nt, pl.smem);
  if (occ <= 0) return RAS_ENOTSUP;
  if (kind == kBand && pl.nstages == 6 && (int64_t)items.size() > (int64_t)occ * nsm) {
    const size_t sm4 = main_smem_bytes(kind, prec, pl.nt, Wmax, npad_max, kmax, 4);
    const int occ4 = main_occupancy(kind, prec, pl.nt, sm4);
    if (occ4 > occ) {
      pl.nstages = 4;
      pl.smem = sm4;
      occ = occ4;
    }
  }
  int64_t cap = (int64_t)occ * nsm;
  const int64_t lim = env_int("RAS_MAX_CTAS", 0);
  if (lim > 0) cap = std::min<int64_t>(cap, lim);
  if (grid_cap > 0) cap = std::min<int64_t>(cap, grid_cap);
  // as many CTAs as give every CTA the same number of subdomains (the most
  // any CTA would get anyway): a synchronous iteration takes as long as its
  // fullest CTA either way, and in the asynchronous mode subdomains then
  // update at the same rate (unequal counts, e.g. 256 subdomains on 152 CTAs,
  // made some update twice as often as their neighbours, and the iteration
  // with CG-20 local solves then often failed to converge)
  const int64_t nit = (int64_t)items.size();
  const int64_t per = (nit + cap - 1) / std::max<int64_t>(cap, 1);
  pl.grid = (int)(per > 0 ? (nit + per - 1) / per : 0);
  if (pl.grid <= 0) return RAS_EINVAL;
  // the dynamic asynchronous schedule takes items by ticket, so it can use
  // every co-resident slot (e.g. 152 CTAs for 256 subdomains)
  pl.grid_dyn = (int)std::min<int64_t>(cap, nit);
  assign_items(pl, items, cost, pl.grid);
  auto up = [&](auto *&d, const auto &v) -> cudaError_t {
    using T = typename std::remove_reference<decltype(v)>::type::value_type;
    cudaError_t e = dev_malloc((void **)&d, std::max<size_t>(v.size(), 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, stream);
  };
  CUDA_TRY(up(pl.d_items, pl.items));
  CUDA_TRY(up(pl.d_cta_off, pl.cta_off));
  CUDA_TRY(up(pl.d_cta_sys, pl.cta_sys));
  CUDA_TRY(up(pl.d_cta_sys_off, pl.cta_sys_off));
  return RAS_OK;
}

SysDesc make_sysdesc(const ras_ctx *c, const double *b, double *x, double tol) {
  SysDesc s{};
  s.b = b;
  s.x = x;
  s.xalt = c->d_xalt;
  s.n = c->n;
  s.P = c->P;
  s.K = c->K;
  s.tol2 = tol * tol;
  s.subs = c->d_subs;
  s.sub = c->d_sub;
  s.st = c->d_st;
  s.gidx = c->d_gidx;
  s.ownf = c->d_ownf;
  s.rcol = c->d_rcol;
  s.rval = c->d_rval;
  s.own_l = c->d_own;
  s.own_g = c->d_own_g;
  s.xg = c->d_xg;
  s.fac = c->d_fac;
  s.lcol = c->d_lcol;
  s.lcol16 = c->d_lcol16;
  s.vpair = c->d_vpair;
  s.cpair = c->d_cpair;
  s.vdia = c->d_vdia;
  s.grid = c->grid;
  s.gs2 = c->gs2;
  s.gs3 = c->gs3;
  s.lval = c->d_lval;
  s.ilu_fcol = c->d_ifc;
  s.ilu_fval = c->d_ifv;
  s.ilu_bcol = c->d_ibc;
  s.ilu_bval = c->d_ibv;
  s.ilu_bdiag = c->d_ibd;
  s.ilu_kl = c->ilu_kl;
  s.ilu_ku = c->ilu_ku;
  s.lev_ptr = c->d_levp;
  s.lev_rows = c->d_levr;
  s.nbr = c->d_nbr;
  s.tnbr = c->d_tnbr;
  s.kry = c->d_kry;
  s.kry_ld = c->kry_ld;
  return s;
}

int64_t timeout_ns() { return env_int("RAS_TIMEOUT_MS", 20000) * 1000000ll; }

}  // namespace

// ========================================================================
// C ABI
// ========================================================================

extern "C" {

const char *ras_status_str(ras_status s) {
  switch (s) {
    case RAS_OK: return "ok";
    case RAS_EINVAL: return "invalid argument";
    case RAS_ENOMEM: return "out of memory";
    case RAS_ENOTSPD: return "local matrix not positive definite";
    case RAS_ENOCONV: return "no convergence within the update limit";
    case RAS_ETIMEOUT: return "device-side wait timed out";
    case RAS_ECUDA: return "CUDA runtime error";
    case RAS_ENOTSUP: return "unsupported configuration";
  }
  return "unknown status";
}

ras_status ras_partition_regular2d(int32_t nx, int32_t ny, int32_t px, int32_t py, int32_t *part) {
  if (!part || nx <= 0 || ny <= 0 || px <= 0 || py <= 0 || px > nx || py > ny) return RAS_EINVAL;
  for (int32_t y = 0; y < ny; ++y) {
    const int32_t by = (int32_t)(((int64_t)y * py) / ny);
    for (int32_t x = 0; x < nx; ++x)
      part[(int64_t)y * nx + x] = by * px + (int32_t)(((int64_t)x * px) / nx);
  }
  return RAS_OK;
}

ras_status ras_partition_bfs(const ras_csr *A, int32_t P, uint64_t seed, int32_t *part) {
  if (!A || !part || A->n <= 0 || P <= 0 || P > A->n || !A->row_ptr || !A->col_idx) return RAS_EINVAL;
  const int n = A->n;
  // target sizes from random weights in [0.7, 1.3]
  std::vector<double> wgt(P);
  double wsum = 0.0;
  for (int p = 0; p < P; ++p) {
    wgt[p] = 1.0 + 0.3 * (2.0 * unit_double(splitmix64_at(seed, (uint64_t)p)) - 1.0);
    wsum += wgt[p];
  }
  std::vector<int64_t> target(P), size(P, 0);
  int64_t tsum = 0;
  for (int p = 0; p < P; ++p) {
    target[p] = (int64_t)std::floor((double)n * wgt[p] / wsum);
    tsum += target[p];
  }
  for (int64_t rem = n - tsum, p = 0; rem != 0; p = (p + 1) % P) {
    if (rem > 0) { ++target[p]; --rem; }
    else if (target[p] > 0) { --target[p]; ++rem; }
  }
  std::fill(part, part + n, -1);
  std::vector<std::vector<int32_t>> queue(P);
  std::vector<size_t> qhead(P, 0);
  std::vector<int32_t> cursor(A->row_ptr, A->row_ptr + n);
  for (int p = 0; p < P; ++p) {
    int64_t v = (int64_t)std::floor(unit_double(splitmix64_at(seed, (uint64_t)(P + p))) * (double)n);
    if (v >= n) v = n - 1;
    while (part[v] != -1) v = (v + 1) % n;
    part[v] = p;
    size[p] = 1;
    queue[p].push_back((int32_t)v);
  }
  for (bool grew = true; grew;) {
    grew = false;
    for (int p = 0; p < P; ++p) {
      if (size[p] >= target[p]) continue;
      while (qhead[p] < queue[p].size()) {
        const int f = queue[p][qhead[p]];
        int got = -1;
        while (cursor[f] < A->row_ptr[f + 1]) {
          const int c = A->col_idx[cursor[f]++];
          if (part[c] == -1) { got = c; break; }
        }
        if (got < 0) { ++qhead[p]; continue; }
        part[got] = p;
        ++size[p];
        queue[p].push_back(got);
        grew = true;
        break;
      }
    }
  }
  for (;;) {
    for (bool changed = true; changed;) {
      changed = false;
      for (int i = 0; i < n; ++i) {
        if (part[i] != -1) continue;
        int best = -1;
        for (int k = A->row_ptr[i]; k < A->row_ptr[i + 1]; ++k) {
          const int q = part[A->col_idx[k]];
          if (q >= 0 && (best < 0 || size[q] < size[best] || (size[q] == size[best] && q < best)))
            best = q;
        }
        if (best >= 0) {
          part[i] = best;
          ++size[best];
          changed = true;
        }
      }
    }
    const int32_t *first = std::find(part, part + n, -1);
    if (first == part + n) break;
    const int q = (int)(std::min_element(size.begin(), size.end()) - size.begin());
    part[first - part] = q;
    ++size[q];
  }
  return RAS_OK;
}

ras_status ras_destroy(ras_ctx *ctx) {
  delete ctx;
  return RAS_OK;
}

ras_status ras_setup(const ras_csr *A, const int32_t *partition, int32_t P, int32_t overlap,
                     const ras_local_solver *lsv, void *cuda_stream, ras_ctx **out) {
  if (!out) return RAS_EINVAL;
  *out = nullptr;
  if (!partition || P <= 0 || overlap < 0 || !lsv) return RAS_EINVAL;
  if (lsv->kind < RAS_LOCAL_BANDCHOL || lsv->kind > RAS_LOCAL_GMRES) return RAS_EINVAL;
  if (lsv->prec < RAS_FP64 || lsv->prec > RAS_BF16_STORE) return RAS_EINVAL;
  const bool banded = lsv->kind == RAS_LOCAL_BANDCHOL || lsv->kind == RAS_LOCAL_BANDLU;
  if (lsv->prec == RAS_BF16_STORE && !banded) return RAS_EINVAL;
  if (!banded && lsv->inner_iters <= 0) return RAS_EINVAL;
  if (lsv->kind == RAS_LOCAL_GMRES && lsv->inner_iters > kMaxGmres) return RAS_EINVAL;
  if (!std::isfinite(lsv->oras_alpha)) return RAS_EINVAL;
  ras_status st = check_csr(A);
  if (st != RAS_OK) return st;
  const int n = A->n;
  std::vector<std::vector<int32_t>> owned_lists(P);
  for (int i = 0; i < n; ++i) {
    if (partition[i] < 0 || partition[i] >= P) return RAS_EINVAL;
    owned_lists[partition[i]].push_back(i);
  }
  for (int p = 0; p < P; ++p)
    if (owned_lists[p].empty()) return RAS_EINVAL;

  t_alloc_count = 0;  // allocation numbering of the fault-injection hook
  std::unique_ptr<ras_ctx> c(new ras_ctx());
  c->stream = (cudaStream_t)cuda_stream;
  c->n = n;
  c->P = P;
  c->overlap = overlap;
  c->ls = *lsv;
  int K = 0;
  for (int i = 0; i < n; ++i) K = std::max(K, A->row_ptr[i + 1] - A->row_ptr[i]);
  c->K = K;
  const int kind = lsv->kind, prec = lsv->prec;

  // ---- maps (parallel over subdomains; each worker has its own mark array)
  std::vector<SubMaps> maps(P);
  {
    const int nt = std::min(host_threads(), P);
    std::vector<std::vector<int32_t>> marks(nt, std::vector<int32_t>(n, -1));
    std::atomic<int> next(0);
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
      th.emplace_back([&, t]() {
        for (int p; (p = next.fetch_add(1)) < P;)
          build_maps(A, partition, owned_lists[p], p, overlap, marks[t], maps[p]);
      });
    for (auto &t : th) t.join();
  }

  // ---- local CG on a 2D / 3D stencil: local rows on grid boxes (all
  // subdomains or none), so that the residual gather computes every column
  // instead of loading it and the staged kernel can take A_p in diagonal-
  // offset form. A staged-size problem keeps its boxes within the staged limit
  if (kind == RAS_LOCAL_CG && (K == 5 || K == 7) && env_int("RAS_CG_GRID", 1) != 0) {
    size_t nmax = 0;
    for (int p = 0; p < P; ++p) nmax = std::max(nmax, maps[p].omega.size());
    const int max_rows =
        prec == RAS_FP32 && nmax <= (size_t)kStagedRows ? kStagedRows : INT32_MAX;
    std::atomic<int> fail(0);
    parallel_for(P, [&](int p) {
      if (!fail && !grid_embed(A, maps[p], max_rows)) fail = 1;
    });
    for (int p = 1; p < P && !fail; ++p)
      if (maps[p].dims != maps[0].dims || maps[p].s2 != maps[0].s2 || maps[p].s3 != maps[0].s3)
        fail = 1;
    if (!fail && (K < 1 + 2 * maps[0].dims ||
                  (int64_t)n + std::max(maps[0].s2, maps[0].s3) >= INT32_MAX))
      fail = 1;
    if (fail) {
      for (int p = 0; p < P; ++p) {
        maps[p].slot_g.clear();
        maps[p].slot_of.clear();
      }
    } else {
      c->grid = maps[0].dims;
      c->gs2 = (int32_t)maps[0].s2;
      c->gs3 = (int32_t)maps[0].s3;
    }
  }

  // ---- descriptors and offsets
  c->subs.resize(P);
  c->cost.resize(P);
  int64_t rows = 0, owns = 0, fac = 0, levp = 0, levr = 0;
  int nbrs = 0, Wmax = 0, npad_max = 0;
  const int m = std::max(lsv->inner_iters, 1);
  for (int p = 0; p < P; ++p) {
    SubDesc &d = c->subs[p];
    const SubMaps &mp = maps[p];
    d.n = (int32_t)(mp.slot_g.empty() ? mp.omega.size() : mp.slot_g.size());
    d.g0 = mp.g0;
    d.bx = mp.bx;
    d.bxy = mp.bxy;
    d.npad = (d.n + 31) / 32 * 32;
    d.n_own = (int32_t)owned_lists[p].size();
    d.W = (std::max(mp.w, 1) + 3) / 4 * 4;  // band records: W a multiple of 4
    d.row_off = rows;
    d.own_off = owns;
    d.fac_off = fac;
    d.nbr_off = nbrs;
    d.n_nbr = (int32_t)mp.nbr.size();
    rows += d.npad;
    owns += d.n_own;
    nbrs += d.n_nbr;
    if (banded) {
      if (mp.w > (kind == RAS_LOCAL_BANDLU ? kMaxBandLuW : kMaxBandW)) return RAS_ENOTSUP;
      fac += 2ll * (d.npad / 32) * 32 * (d.W + 32);  // forward and backward records
      Wmax = std::max(Wmax, d.W);
      c->cost[p] = (double)d.npad * (d.W + 1) * 2.0 + 12.0 * d.n * K;
    } else {
      c->cost[p] = kind == RAS_LOCAL_GMRES
                       ? (double)d.n * (K * (m + 1) + 4.0 * m * (m + 1))  // + CGS2 projections
                       : (double)d.n * K * (m + 1) * (kind == RAS_LOCAL_ILU0_CG ? 3.0 : 1.0);
    }
    c->maxw = std::max(c->maxw, mp.w);
    npad_max = std::max(npad_max, d.npad);
  }
  c->plan.Wmax = banded ? Wmax : 0;
  c->plan.npad_max = npad_max;
  c->exec_kind = banded ? kBand : kind == RAS_LOCAL_GMRES ? kGMRES : kind;
  if (kind == RAS_LOCAL_CG && prec == RAS_FP32 && K <= kMaxEll && npad_max <= kStagedRows &&
      env_int("RAS_CG_STAGE", 1) != 0)
    c->exec_kind = kCGS;

  // ---- per-row host arrays
  std::vector<int32_t> gidx(rows, 0), rcol(rows * K, 0), own(owns), nbr(nbrs);
  std::vector<uint8_t> ownf(rows, 0);
  std::vector<double> rval(rows * K, 0.0);
  std::vector<int32_t> lcol;
  std::vector<double> lval64, lu64;
  std::vector<double> band;  // FP64 bands for the GPU factorisation
  std::vector<int64_t> band_off(P, 0);
  const bool lu = kind == RAS_LOCAL_BANDLU;
  const double alpha = lsv->oras_alpha;
  if (!banded) {
    lcol.assign(rows * K, 0);
    lval64.assign(rows * K, 0.0);
    if (kind == RAS_LOCAL_ILU0_CG) lu64.assign(rows * K, 0.0);
  } else {
    int64_t bsz = 0;
    for (int p = 0; p < P; ++p) {
      band_off[p] = bsz;
      // Cholesky: lower half (ld = w+1); LU: the whole band (ld = 2w+1)
      bsz += (int64_t)c->subs[p].n * (lu ? 2 * maps[p].w + 1 : maps[p].w + 1);
    }
    band.assign(bsz, 0.0);
  }
  std::vector<std::vector<int32_t>> lev_ptr(P), lev_rows(P);
  std::atomic<int> ilu_fail(0);
  parallel_for(P, [&](int p) {
    const SubDesc &d = c->subs[p];
    const SubMaps &mp = maps[p];
    const int64_t ro = d.row_off;
    int t_own = 0;
    // local CSR of A_p (for ILU) built alongside the ELL arrays
    std::vector<int32_t> lrp, lci;
    std::vector<double> lva;
    if (kind == RAS_LOCAL_ILU0_CG) lrp.push_back(0);
    const bool emb = !mp.slot_g.empty();
    for (int i = 0; i < d.n; ++i) {
      if (emb && mp.slot_g[i] < 0) {
        // hole row of a grid box: flag 2, zero values, columns on itself
        gidx[ro + i] = mp.omega[0];
        ownf[ro + i] = 2;
        for (int k = 0; k < K; ++k) {
          rcol[ro * K + (int64_t)k * d.npad + i] = mp.omega[0];
          lcol[ro * K + (int64_t)k * d.npad + i] = i;
        }
        continue;
      }
      const int t = emb ? (int)(std::lower_bound(mp.omega.begin(), mp.omega.end(), mp.slot_g[i]) -
                                mp.omega.begin())
                        : i;
      const int g = mp.omega[t];
      gidx[ro + i] = g;
      ownf[ro + i] = mp.owned[t];
      if (mp.owned[t]) own[d.own_off + t_own++] = i;
      int k = 0, kl = 0, diag_kl = -1;
      int64_t diag_lva = -1;
      double ext = 0.0;  // couplings of row i to points outside Omega_p
      for (int e = A->row_ptr[g]; e < A->row_ptr[g + 1]; ++e, ++k) {
        const int col = A->col_idx[e];
        rcol[ro * K + (int64_t)k * d.npad + i] = col;
        rval[ro * K + (int64_t)k * d.npad + i] = A->val[e];
        int j = local_index(mp.omega, col);
        if (emb && j >= 0) j = mp.slot_of[j];
        if (j < 0) {
          ext += A->val[e];
          continue;
        }
        if (j == i) {
          diag_kl = kl;
          diag_lva = (int64_t)lva.size();
        }
        if (lu) {
          band[band_off[p] + (int64_t)i * (2 * mp.w + 1) + (j - i + mp.w)] = A->val[e];
        } else if (banded) {
          if (j <= i) band[band_off[p] + (int64_t)i * (mp.w + 1) + (j - i + mp.w)] = A->val[e];
        } else {
          lcol[ro * K + (int64_t)kl * d.npad + i] = j;
          lval64[ro * K + (int64_t)kl * d.npad + i] = A->val[e];
          if (kind == RAS_LOCAL_ILU0_CG) {
            lci.push_back(j);
            lva.push_back(A->val[e]);
          }
          ++kl;
        }
      }
      if (alpha != 0.0 && ext != 0.0) {
        // Optimized RAS: exterior neighbour values replaced by alpha times the
        // row's own value, so alpha * ext joins the local diagonal (the
        // residual operator rval keeps A)
        if (lu) band[band_off[p] + (int64_t)i * (2 * mp.w + 1) + mp.w] += alpha * ext;
        else if (banded) band[band_off[p] + (int64_t)i * (mp.w + 1) + mp.w] += alpha * ext;
        else {
          lval64[ro * K + (int64_t)diag_kl * d.npad + i] += alpha * ext;
          if (kind == RAS_LOCAL_ILU0_CG) lva[diag_lva] += alpha * ext;
        }
      }
      for (; k < K; ++k) rcol[ro * K + (int64_t)k * d.npad + i] = g;  // zero-valued padding
      if (emb) {
        // grid layout: the residual operator's entries in slot order (the
        // diagonal, then the global offsets in ascending order), a missing
        // entry as column g and value 0; grid_embed saw every entry of this
        // row move one unit along one axis, so each offset has its slot
        int64_t goff[8];
        int ns = 0;
        goff[ns++] = 0;
        if (mp.dims == 3) goff[ns++] = -mp.s3;
        goff[ns++] = -mp.s2;
        goff[ns++] = -1;
        goff[ns++] = 1;
        goff[ns++] = mp.s2;
        if (mp.dims == 3) goff[ns++] = mp.s3;
        double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        bool has[8] = {false, false, false, false, false, false, false, false};
        for (int e = A->row_ptr[g]; e < A->row_ptr[g + 1]; ++e) {
          const int64_t o = (int64_t)A->col_idx[e] - g;
          int q = 0;
          while (q + 1 < ns && goff[q] != o) ++q;
          v[q] += A->val[e];
          has[q] = true;
        }
        for (int q = 0; q < K; ++q) {
          const int64_t e = ro * K + (int64_t)q * d.npad + i;
          rcol[e] = q < ns && has[q] ? (int32_t)(g + goff[q]) : g;
          rval[e] = q < ns ? v[q] : 0.0;
        }
      }
      if (!banded)
        for (; kl < K; ++kl) lcol[ro * K + (int64_t)kl * d.npad + i] = i;
      if (kind == RAS_LOCAL_ILU0_CG) lrp.push_back((int32_t)lci.size());
    }
    for (int i = d.n; i < d.npad; ++i) {
      gidx[ro + i] = mp.omega[0];
      for (int k = 0; k < K; ++k) {
        rcol[ro * K + (int64_t)k * d.npad + i] = mp.omega[0];
        if (!banded) lcol[ro * K + (int64_t)k * d.npad + i] = i < d.n ? i : 0;
      }
    }
    for (size_t q = 0; q < mp.nbr.size(); ++q) nbr[d.nbr_off + q] = mp.nbr[q];
    if (kind == RAS_LOCAL_ILU0_CG) {
      std::vector<double> f = lva;
      if (!ilu0_local(d.n, lrp, lci, f)) {
        ilu_fail = 1;
        return;
      }
      // scatter the factors into the ELL layout (same column order as lcol)
      for (int i = 0; i < d.n; ++i)
        for (int e = lrp[i], kl = 0; e < lrp[i + 1]; ++e, ++kl)
          lu64[ro * K + (int64_t)kl * d.npad + i] = f[e];
      std::vector<int32_t> pf, rf, pb, rb;
      level_schedule(d.n, lrp, lci, pf, rf, pb, rb);
      lev_ptr[p] = pf;
      lev_ptr[p].insert(lev_ptr[p].end(), pb.begin(), pb.end());
      lev_rows[p] = rf;
      lev_rows[p].insert(lev_rows[p].end(), rb.begin(), rb.end());
    }
  });
  if (ilu_fail) return RAS_ENOTSPD;
  // local CG: every ELL row starts with its diagonal (the staged kernel reuses
  // p[i]); an SPD A_p has a positive diagonal in every row
  if (kind == RAS_LOCAL_CG) {
    std::atomic<int> nodiag(0);
    parallel_for(P, [&](int p) {
      const SubDesc &d = c->subs[p];
      for (int i = 0; i < d.n; ++i) {
        if (ownf[d.row_off + i] == 2) continue;  // hole row of a grid box
        const int64_t e0 = d.row_off * K + i;
        bool found = false;
        for (int kl = 0; kl < K && !found; ++kl) {
          const int64_t e = e0 + (int64_t)kl * d.npad;
          if (lcol[e] == i && lval64[e] > 0.0) {
            std::swap(lcol[e], lcol[e0]);
            std::swap(lval64[e], lval64[e0]);
            found = true;
          }
        }
        if (!found) nodiag = 1;
      }
    });
    if (nodiag) return RAS_ENOTSPD;
  }
  // staged CG, diagonal-offset form: local rows on grid boxes whose largest
  // local offset (bx in 2D, bxy in 3D) fits the zero margins around r
  c->dia = c->exec_kind == kCGS && c->grid > 0 && env_int("RAS_CG_DIA", 1) != 0;
  for (int p = 0; p < P && c->dia; ++p) {
    const SubDesc &d = c->subs[p];
    if ((c->grid == 3 ? d.bxy : d.bx) > kDiaMargin) c->dia = false;
  }
  std::vector<int32_t> levp_all, levr_all;
  if (kind == RAS_LOCAL_ILU0_CG) {
    for (int p = 0; p < P; ++p) {
      SubDesc &d = c->subs[p];
      d.lev_off = levp;
      d.lrow_off = levr;
      // forward pointer array has nlev_f + 1 entries, backward nlev_b + 1
      const std::vector<int32_t> &lp = lev_ptr[p];
      // split point: the forward array ends where its last entry equals n
      int nf = 0;
      while (lp[nf] != d.n) ++nf;
      d.nlev_f = nf;
      d.nlev_b = (int)lp.size() - (nf + 1) - 1;
      levp += (int64_t)lp.size();
      levr += (int64_t)lev_rows[p].size();
      levp_all.insert(levp_all.end(), lp.begin(), lp.end());
      levr_all.insert(levr_all.end(), lev_rows[p].begin(), lev_rows[p].end());
    }
  }
  std::vector<int> band_w(P);
  for (int p = 0; p < P; ++p) band_w[p] = maps[p].w;
  for (int p = 0; p < P; ++p) {
    c->omega.push_back(std::move(maps[p].omega));
    c->owned.push_back(std::move(maps[p].owned));
    c->iface.push_back(std::move(maps[p].iface));
  }

  // ---- device upload
  CUDA_TRY(cudaEventCreate(&c->ev0));
  CUDA_TRY(cudaEventCreate(&c->ev1));
  CUDA_TRY(cudaEventCreate(&c->evk0));
  CUDA_TRY(cudaEventCreate(&c->evk1));
  CUDA_TRY(cudaEventCreateWithFlags(&c->ev_begin, cudaEventDisableTiming));
  // spanning tree of the subdomain graph (breadth-first from subdomain 0, a
  // new root for every further component): the decentralized convergence
  // detection elects its leader along these edges
  std::vector<int32_t> tnbr;
  {
    std::vector<std::vector<int32_t>> tadj(P);
    std::vector<char> seen(P, 0);
    std::vector<int32_t> queue;
    queue.reserve(P);
    for (int r = 0; r < P; ++r) {
      if (seen[r]) continue;
      seen[r] = 1;
      queue.assign(1, r);
      for (size_t h = 0; h < queue.size(); ++h) {
        const int p = queue[h];
        for (int32_t q : maps[p].nbr) {
          if (seen[q]) continue;
          seen[q] = 1;
          tadj[p].push_back(q);
          tadj[q].push_back(p);
          queue.push_back(q);
        }
      }
    }
    for (int p = 0; p < P; ++p) {
      std::sort(tadj[p].begin(), tadj[p].end());
      c->subs[p].tnbr_off = (int32_t)tnbr.size();
      c->subs[p].n_tnbr = (int32_t)tadj[p].size();
      tnbr.insert(tnbr.end(), tadj[p].begin(), tadj[p].end());
    }
  }
  if ((st = c->upload(c->d_tnbr, tnbr)) != RAS_OK) return st;
  if ((st = c->upload(c->d_subs, c->subs)) != RAS_OK) return st;
  if ((st = c->alloc(c->d_sub, P)) != RAS_OK) return st;
  if ((st = c->alloc(c->d_st, 1)) != RAS_OK) return st;
  if ((st = c->upload(c->d_gidx, gidx)) != RAS_OK) return st;
  if ((st = c->upload(c->d_ownf, ownf)) != RAS_OK) return st;
  if ((st = c->upload(c->d_rcol, rcol)) != RAS_OK) return st;
  if ((st = c->upload(c->d_rval, rval)) != RAS_OK) return st;
  if ((st = c->upload(c->d_own, own)) != RAS_OK) return st;
  {
    std::vector<int32_t> own_g(own.size());
    for (int p = 0; p < P; ++p) {
      const SubDesc &d = c->subs[p];
      for (int t = 0; t < d.n_own; ++t) own_g[d.own_off + t] = gidx[d.row_off + own[d.own_off + t]];
    }
    if ((st = c->upload(c->d_own_g, own_g)) != RAS_OK) return st;
  }
  if ((st = c->upload(c->d_nbr, nbr)) != RAS_OK) return st;
  if ((st = c->alloc(c->d_xalt, n)) != RAS_OK) return st;
  if ((st = c->alloc(c->d_xg, (size_t)rows)) != RAS_OK) return st;
  if ((st = c->alloc(c->d_ctl, 1)) != RAS_OK) return st;
  if ((st = c->alloc(c->d_sysdesc, 1)) != RAS_OK) return st;
  CUDA_TRY(host_malloc_pinned(&c->h_sysdesc, sizeof(SysDesc)));
  CUDA_TRY(host_malloc_pinned(&c->h_ctl, sizeof(GridCtl)));
  CUDA_TRY(host_malloc_pinned(&c->h_st, sizeof(SysState)));
  CUDA_TRY(host_malloc_pinned(&c->h_sub, sizeof(SubState) * P));
  CUDA_TRY(cudaMemsetAsync(c->d_ctl, 0, sizeof(GridCtl), c->stream));
  CUDA_TRY(cudaMemsetAsync(c->d_xalt, 0, sizeof(double) * n, c->stream));

  if (banded) {
    // factorise on the GPU in FP64, then lay out the block records in the storage precision
    double *d_band = nullptr;
    BandJob *d_jobs = nullptr;
    LayoutJob *d_ljobs = nullptr;
    std::vector<BandJob> jobs(P);
    std::vector<LayoutJob> ljobs;
    int maxw = 0;
    for (int p = 0; p < P; ++p) {
      const SubDesc &d = c->subs[p];
      const int w = band_w[p];
      jobs[p] = {d.n, w, band_off[p]};
      maxw = std::max(maxw, w);
      for (int Kb = 0; Kb < d.npad / 32; ++Kb) {
        LayoutJob lj{};
        lj.n = d.n;
        lj.w = w;
        lj.W = d.W;
        lj.K = Kb;
        lj.nb = d.npad / 32;
        lj.band_off = band_off[p];
        lj.fac_off = d.fac_off;
        ljobs.push_back(lj);
      }
    }
    TmpDev t_band, t_jobs, t_ljobs;  // freed on every return below
    CUDA_TRY(dev_malloc(&t_band.p, std::max<size_t>(band.size(), 1) * sizeof(double)));
    CUDA_TRY(dev_malloc(&t_jobs.p, jobs.size() * sizeof(BandJob)));
    CUDA_TRY(dev_malloc(&t_ljobs.p, ljobs.size() * sizeof(LayoutJob)));
    d_band = static_cast<double *>(t_band.p);
    d_jobs = static_cast<BandJob *>(t_jobs.p);
    d_ljobs = static_cast<LayoutJob *>(t_ljobs.p);
    CUDA_TRY(cudaMemcpyAsync(d_band, band.data(), band.size() * sizeof(double),
                             cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(BandJob),
                             cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(d_ljobs, ljobs.data(), ljobs.size() * sizeof(LayoutJob),
                             cudaMemcpyHostToDevice, c->stream));
    void *d_fac = nullptr;
    const size_t fbytes = std::max<int64_t>(fac, 1) * prec_bytes(prec);
    cudaError_t e = dev_malloc(&d_fac, fbytes);
    if (e != cudaSuccess) {
      // the copies above read host vectors that outlive them only until return
      cudaStreamSynchronize(c->stream);
      return RAS_ENOMEM;
    }
    c->bufs.push_back({d_fac, fbytes});
    c->device_bytes += (int64_t)fbytes;
    c->d_fac = d_fac;
    e = lu ? launch_band_lu(d_jobs, P, maxw, d_band, c->d_ctl, c->stream)
           : launch_band_chol(d_jobs, P, maxw, d_band, c->d_ctl, c->stream);
    if (e == cudaSuccess)
      e = launch_band_layout(prec, lu, d_ljobs, (int)ljobs.size(), d_band, d_fac, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(GridCtl), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      last_cuda_error() = e;
      return RAS_ECUDA;
    }
    if (c->h_ctl->status != 0) return (ras_status)c->h_ctl->status;
  } else {
    std::vector<int32_t> &lc = lcol;
    if ((st = c->upload(c->d_lcol, lc)) != RAS_OK) return st;
    if (kind == RAS_LOCAL_CG && prec == RAS_FP32 && npad_max <= kStagedRows) {
      std::vector<int16_t> l16(lc.begin(), lc.end());
      if ((st = c->upload(c->d_lcol16, l16)) != RAS_OK) return st;
      if (c->dia) {
        // diagonal-offset form: slot 0 the diagonal, then one slot per local
        // offset -bxy, -bx, -1, 1, bx, bxy (2D: without +-bxy), zero where
        // the row has no entry in Omega_p there
        std::vector<float> vd(lval64.size(), 0.f);
        for (int p = 0; p < P; ++p) {
          const SubDesc &d = c->subs[p];
          const int64_t eb = d.row_off * K, np = d.npad;
          int loff[8], ns = 0;
          loff[ns++] = 0;
          if (c->grid == 3) loff[ns++] = -d.bxy;
          loff[ns++] = -d.bx;
          loff[ns++] = -1;
          loff[ns++] = 1;
          loff[ns++] = d.bx;
          if (c->grid == 3) loff[ns++] = d.bxy;
          for (int i = 0; i < d.n; ++i) {
            vd[eb + i] = (float)lval64[eb + i];  // the diagonal (slot 0 of lcol)
            for (int kl = 1; kl < K; ++kl) {
              const int64_t e = eb + (int64_t)kl * np + i;
              const int o = lc[e] - i;
              if (o == 0) continue;  // padding
              int q = 1;
              while (q + 1 < ns && loff[q] != o) ++q;  // every local entry has its slot
              vd[eb + (int64_t)q * np + i] += (float)lval64[e];
            }
          }
        }
        if ((st = c->upload(c->d_vdia, vd)) != RAS_OK) return st;
      } else if (K % 2 == 1 && K >= 3 && K <= 7) {
        // paired layout for the staged kernel (diagonal first, then pairs)
        std::vector<float> vp(lval64.size(), 0.f);
        std::vector<uint32_t> cp(lval64.size() / 2 + 1, 0u);
        for (int p = 0; p < P; ++p) {
          const SubDesc &d = c->subs[p];
          const int64_t eb = d.row_off * K, np = d.npad;
          for (int i = 0; i < d.npad; ++i) {
            vp[eb + i] = (float)lval64[eb + i];
            for (int q = 0; q < (K - 1) / 2; ++q) {
              const int64_t e1 = eb + (int64_t)(1 + 2 * q) * np + i, e2 = e1 + np;
              vp[eb + np + 2 * ((int64_t)q * np + i)] = (float)lval64[e1];
              vp[eb + np + 2 * ((int64_t)q * np + i) + 1] = (float)lval64[e2];
              cp[eb / 2 + (int64_t)q * np + i] =
                  (uint32_t)(uint16_t)lc[e1] | ((uint32_t)(uint16_t)lc[e2] << 16);
            }
          }
        }
        if ((st = c->upload(c->d_vpair, vp)) != RAS_OK) return st;
        if ((st = c->upload(c->d_cpair, cp)) != RAS_OK) return st;
      }
    }

    auto up_prec = [&](void *&dst, const std::vector<double> &src) -> ras_status {
      const size_t bytes = std::max<size_t>(src.size(), 1) * prec_bytes(prec);
      std::vector<unsigned char> tmp(bytes);
      for (size_t k = 0; k < src.size(); ++k) store_prec(tmp.data(), k, prec, src[k]);
      unsigned char *d = nullptr;
      ras_status s2 = c->upload(d, tmp);
      dst = d;
      return s2;
    };
    if ((st = up_prec(c->d_lval, lval64)) != RAS_OK) return st;
    if (kind == RAS_LOCAL_ILU0_CG) {
      {
        // level-order copies of the factors: forward rows keep their strictly
        // lower entries, backward rows their strictly upper ones and the
        // diagonal, each in the ELL order of the row
        int kl = 0, ku = 0;
        for (int p = 0; p < P; ++p) {
          const SubDesc &d = c->subs[p];
          for (int i = 0; i < d.n; ++i) {
            int nl = 0, nu = 0;
            for (int k = 0; k < K; ++k) {
              const int64_t e = d.row_off * K + (int64_t)k * d.npad + i;
              if (lu64[e] == 0.0) continue;
              if (lc[e] < i) ++nl;
              else if (lc[e] > i) ++nu;
            }
            kl = std::max(kl, nl);
            ku = std::max(ku, nu);
          }
        }
        kl = std::max(kl, 1);
        ku = std::max(ku, 1);
        c->ilu_kl = kl;
        c->ilu_ku = ku;
        std::vector<int32_t> fc(rows * kl, -1), bc(rows * ku, -1);
        std::vector<double> fv(rows * kl, 0.0), bv(rows * ku, 0.0), bd(rows, 1.0);
        for (int p = 0; p < P; ++p) {
          const SubDesc &d = c->subs[p];
          const int32_t *rf = levr_all.data() + d.lrow_off, *rb = rf + d.n;
          for (int e = 0; e < d.n; ++e) {
            int t = 0;
            const int i = rf[e];
            for (int k = 0; k < K; ++k) {
              const int64_t q = d.row_off * K + (int64_t)k * d.npad + i;
              if (lu64[q] != 0.0 && lc[q] < i) {
                fc[d.row_off * kl + (int64_t)t * d.npad + e] = lc[q];
                fv[d.row_off * kl + (int64_t)t * d.npad + e] = lu64[q];
                ++t;
              }
            }
            t = 0;
            const int ib = rb[e];
            for (int k = 0; k < K; ++k) {
              const int64_t q = d.row_off * K + (int64_t)k * d.npad + ib;
              if (lu64[q] == 0.0) continue;
              if (lc[q] > ib) {
                bc[d.row_off * ku + (int64_t)t * d.npad + e] = lc[q];
                bv[d.row_off * ku + (int64_t)t * d.npad + e] = lu64[q];
                ++t;
              } else if (lc[q] == ib) {
                bd[d.row_off + e] = lu64[q];
              }
            }
          }
        }
        if ((st = c->upload(c->d_ifc, fc)) != RAS_OK) return st;
        if ((st = c->upload(c->d_ibc, bc)) != RAS_OK) return st;
        if ((st = up_prec(c->d_ifv, fv)) != RAS_OK) return st;
        if ((st = up_prec(c->d_ibv, bv)) != RAS_OK) return st;
        if ((st = up_prec(c->d_ibd, bd)) != RAS_OK) return st;
      }
      if ((st = c->upload(c->d_levp, levp_all)) != RAS_OK) return st;
      if ((st = c->upload(c->d_levr, levr_all)) != RAS_OK) return st;
    }
    if (kind == RAS_LOCAL_GMRES) {
      // Krylov basis scratch: m+1 vectors per subdomain in the solve precision
      c->kry_ld = m + 1;
      const size_t cnt = (size_t)rows * c->kry_ld;
      if (prec == RAS_FP64) {
        double *q = nullptr;
        if ((st = c->alloc(q, cnt)) != RAS_OK) return st;
        c->d_kry = q;
      } else {
        float *q = nullptr;
        if ((st = c->alloc(q, cnt)) != RAS_OK) return st;
        c->d_kry = q;
      }
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
  }

  // ---- default launch plan: one system, all subdomains
  std::vector<Item> items(P);
  for (int p = 0; p < P; ++p) items[p] = {0, p, 0, 0};
  st = plan_launch(c->plan, c->exec_kind, prec, items, c->cost, c->plan.Wmax, npad_max, K, c->stream);
  if (st == RAS_ENOTSUP && c->exec_kind == kCGS) {  // staged variant does not fit: plain CG
    c->exec_kind = kind;
    st = plan_launch(c->plan, c->exec_kind, prec, items, c->cost, c->plan.Wmax, npad_max, K, c->stream);
  }
  c->sched = -1;
  c->grid_cap = 0;
  if (st != RAS_OK) return st;
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->last_updates.assign(P, 0);
  *out = c.release();
  return RAS_OK;
}

namespace {

// Runs one full solve of the systems described by `sysdesc` with plan `pl`.
ras_status run_solve(cudaStream_t stream, int kind, int prec, const LaunchPlan &pl,
                     SysDesc *d_sys, int nsys, GridCtl *d_ctl, GridCtl *h_ctl, int32_t mode,
                     int64_t max_updates, int m, cudaEvent_t ev0, cudaEvent_t ev1,
                     cudaEvent_t evk0, cudaEvent_t evk1, int *grid_out, int sched = -1) {
  Launch L{};
  L.sys = d_sys;
  L.nsys = nsys;
  L.mode = mode;
  L.items = pl.d_items;
  L.cta_off = pl.d_cta_off;
  L.cta_sys = pl.d_cta_sys;
  L.cta_sys_off = pl.d_cta_sys_off;
  L.ctl = d_ctl;
  L.max_updates = max_updates > 0 ? max_updates : 1000000;
  L.step_limit = (int64_t)1 << 62;
  L.timeout_ns = timeout_ns();
  L.solve_limit_ns = env_int("RAS_SOLVE_LIMIT_MS", 120000) * 1000000ll;
  // the leader-based scheme stops on any fully converged neighbourhood, so a
  // failed global check is routine there: it resumes until max_updates
  L.max_restarts = mode == RAS_ASYNC_DECENTRAL ? (1 << 30) : 8;
  L.fresh = (int32_t)env_int("RAS_ASYNC_FRESH", 0);
  L.consistent = (int32_t)env_int("RAS_ASYNC_CONSISTENT", 0);
  L.m = m;
  L.Wmax = pl.Wmax;
  L.npad_max = pl.npad_max;
  L.persist = 1;
  L.kmax = pl.kmax;
  L.nstages = pl.nstages;
  const int nitems = (int)pl.items.size();
  L.nitems = nitems;
  // solves run on the dynamic schedule unless the context chose the static
  // assignment (ras_autotune) or RAS_ASYNC_DYNAMIC=0 / RAS_SYNC_DYNAMIC=0;
  // synchronous launches take it when every CTA can hold the decision state
  // of every system
  const int dyn = sched >= 0 ? sched
                             : (env_int(mode == RAS_SYNC ? "RAS_SYNC_DYNAMIC" : "RAS_ASYNC_DYNAMIC",
                                        1) != 0 ? 1 : 0);
  L.dynamic = (dyn && (mode != RAS_SYNC || nsys <= kMaxCtaSys)) ? 1 : 0;
  std::memset(h_ctl, 0, sizeof(GridCtl));
  h_ctl->remaining = nsys;
  CUDA_TRY(cudaMemcpyAsync(d_ctl, h_ctl, sizeof(GridCtl), cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaEventRecord(ev0, stream));
  CUDA_TRY(launch_init(L, nitems, stream));
  CUDA_TRY(cudaEventRecord(evk0, stream));
  const int grid = L.dynamic ? pl.grid_dyn : pl.grid;
  if (grid_out) *grid_out = grid;
  CUDA_TRY(launch_main(kind, prec, pl.nt, L, grid, pl.smem, stream));
  CUDA_TRY(cudaEventRecord(evk1, stream));
  if (mode == RAS_SYNC) CUDA_TRY(launch_copyback(L, nitems, stream));
  CUDA_TRY(cudaEventRecord(ev1, stream));
  CUDA_TRY(launch_residual(L, nitems, stream));
  return RAS_OK;
}

ras_status finish_info(ras_ctx *c, const SysState &st, const GridCtl &ctl, const SubState *sub,
                       int32_t mode, ras_solve_info *info, float ms, float kms, int grid) {
  ras_status rs = RAS_OK;
  if (ctl.status != 0) rs = (ras_status)ctl.status;
  else if (st.status != 0) rs = (ras_status)st.status;
  std::vector<int64_t> u(c->P);
  int64_t stale = 0;
  c->last_phase.assign(3 * (size_t)c->P, 0);
  for (int p = 0; p < c->P; ++p) {
    u[p] = sub[p].updates;
    stale += sub[p].stale;
    c->last_phase[3 * p] = sub[p].t_gather;
    c->last_phase[3 * p + 1] = sub[p].t_solve;
    c->last_phase[3 * p + 2] = sub[p].t_update;
  }
  c->last_updates = u;
  if (info) {
    std::vector<int64_t> s(u);
    std::sort(s.begin(), s.end());
    info->updates_min = s.front();
    info->updates_max = s.back();
    info->updates_median = s[s.size() / 2];
    info->iterations = mode == RAS_SYNC ? st.iters : info->updates_median;
    info->relres = st.b2 > 0 ? std::sqrt(st.res2 / st.b2) : std::sqrt(st.res2);
    info->solve_ms = ms;
    info->restarts = st.restarts;
    info->status = rs;
    info->kernel_ms = kms;
    info->stale_updates = stale;
    info->error_site = ctl.status == RAS_ETIMEOUT ? (int32_t)ctl.err_info : 0;
    info->grid = grid;
  }
  return rs;
}

}  // namespace

ras_status ras_solve(ras_ctx *c, const double *b, double *x, double tol, int32_t mode,
                     int64_t max_updates, ras_solve_info *info) {
  if (!c || !b || !x || !(tol > 0.0) || (mode != RAS_SYNC && mode != RAS_ASYNC && mode != RAS_ASYNC_DECENTRAL)) return RAS_EINVAL;
  if (info) std::memset(info, 0, sizeof(*info));
  *c->h_sysdesc = make_sysdesc(c, b, x, tol);
  CUDA_TRY(cudaMemcpyAsync(c->d_sysdesc, c->h_sysdesc, sizeof(SysDesc), cudaMemcpyHostToDevice,
                           c->stream));
  int grid = 0;
  ras_status rs = run_solve(c->stream, c->exec_kind, c->ls.prec, c->plan, c->d_sysdesc, 1, c->d_ctl,
                            c->h_ctl, mode, max_updates, c->ls.inner_iters, c->ev0, c->ev1,
                            c->evk0, c->evk1, &grid, c->sched);
  if (rs != RAS_OK) return rs;
  CUDA_TRY(cudaMemcpyAsync(c->h_st, c->d_st, sizeof(SysState), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(GridCtl), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaMemcpyAsync(c->h_sub, c->d_sub, sizeof(SubState) * c->P, cudaMemcpyDeviceToHost,
                           c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  float ms = 0.f, kms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  cudaEventElapsedTime(&kms, c->evk0, c->evk1);
  return finish_info(c, *c->h_st, *c->h_ctl, c->h_sub, mode, info, ms, kms, grid);
}

ras_status ras_solve_host(ras_ctx *c, const double *b_host, double *x_host, double tol,
                          int32_t mode, int64_t max_updates, ras_solve_info *info) {
  if (!c || !b_host || !x_host) return RAS_EINVAL;
  if (!c->d_bx) {
    ras_status s = c->alloc(c->d_bx, 2 * (size_t)c->n);
    if (s != RAS_OK) return s;
  }
  double *db = c->d_bx, *dx = c->d_bx + c->n;
  CUDA_TRY(cudaMemcpyAsync(db, b_host, sizeof(double) * c->n, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(cudaMemcpyAsync(dx, x_host, sizeof(double) * c->n, cudaMemcpyHostToDevice, c->stream));
  ras_status rs = ras_solve(c, db, dx, tol, mode, max_updates, info);
  if (rs != RAS_OK && rs != RAS_ENOCONV) return rs;
  CUDA_TRY(cudaMemcpyAsync(x_host, dx, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return rs;
}

ras_status ras_solve_batch(ras_ctx *const *ctxs, int32_t num, const double *const *b,
                           double *const *x, double tol, int32_t mode, int64_t max_updates,
                           ras_solve_info *infos) {
  if (!ctxs || num <= 0 || !b || !x || !(tol > 0.0) || (mode != RAS_SYNC && mode != RAS_ASYNC && mode != RAS_ASYNC_DECENTRAL))
    return RAS_EINVAL;
  for (int s = 0; s < num; ++s)
    if (!ctxs[s] || !b[s] || !x[s] || ctxs[s]->exec_kind != ctxs[0]->exec_kind ||
        ctxs[s]->ls.prec != ctxs[0]->ls.prec || ctxs[s]->ls.inner_iters != ctxs[0]->ls.inner_iters)
      return RAS_EINVAL;
  ras_ctx *c0 = ctxs[0];
  cudaStream_t stream = c0->stream;
  std::vector<Item> items;
  std::vector<double> cost;
  std::vector<SysDesc> sd(num);
  int Wmax = 0, npad_max = 0, kmax = 0;
  for (int s = 0; s < num; ++s) {
    ras_ctx *c = ctxs[s];
    kmax = std::max(kmax, c->K);
    // one solve at a time per context: the state buffers are per context
    for (int t = 0; t < s; ++t)
      if (ctxs[t] == c) return RAS_EINVAL;
    sd[s] = make_sysdesc(c, b[s], x[s], tol);
    for (int p = 0; p < c->P; ++p) {
      items.push_back({s, p, 0, 0});
      cost.push_back(c->cost[p]);
    }
    Wmax = std::max(Wmax, c->plan.Wmax);
    npad_max = std::max(npad_max, c->plan.npad_max);
  }
  LaunchPlan pl;
  ras_status rs = plan_launch(pl, c0->exec_kind, c0->ls.prec, items, cost, Wmax, npad_max, kmax, stream);
  if (rs != RAS_OK) {
    pl.release();
    return rs;
  }
  SysDesc *d_sys = nullptr;
  GridCtl *d_ctl = nullptr;
  GridCtl h_ctl{};
  std::vector<SysState> hst(num);
  auto cleanup = [&]() {
    cudaStreamSynchronize(stream);
    cudaFree(d_sys);
    cudaFree(d_ctl);
    pl.release();
  };
  if (dev_malloc(&d_sys, sizeof(SysDesc) * num) != cudaSuccess ||
      dev_malloc(&d_ctl, sizeof(GridCtl)) != cudaSuccess) {
    cleanup();
    return RAS_ENOMEM;
  }
  cudaMemcpyAsync(d_sys, sd.data(), sizeof(SysDesc) * num, cudaMemcpyHostToDevice, stream);
  int grid = 0;
  rs = run_solve(stream, c0->exec_kind, c0->ls.prec, pl, d_sys, num, d_ctl, &h_ctl, mode,
                 max_updates, c0->ls.inner_iters, c0->ev0, c0->ev1, c0->evk0, c0->evk1, &grid);
  if (rs != RAS_OK) {
    cleanup();
    return rs;
  }
  cudaMemcpyAsync(&h_ctl, d_ctl, sizeof(GridCtl), cudaMemcpyDeviceToHost, stream);
  std::vector<std::vector<SubState>> hsub(num);
  for (int s = 0; s < num; ++s) {
    hsub[s].resize(ctxs[s]->P);
    cudaMemcpyAsync(&hst[s], ctxs[s]->d_st, sizeof(SysState), cudaMemcpyDeviceToHost, stream);
    cudaMemcpyAsync(hsub[s].data(), ctxs[s]->d_sub, sizeof(SubState) * ctxs[s]->P,
                    cudaMemcpyDeviceToHost, stream);
  }
  cudaError_t e = cudaStreamSynchronize(stream);
  float ms = 0.f, kms = 0.f;
  cudaEventElapsedTime(&ms, c0->ev0, c0->ev1);
  cudaEventElapsedTime(&kms, c0->evk0, c0->evk1);
  cleanup();
  if (e != cudaSuccess) return RAS_ECUDA;
  ras_status first = RAS_OK;
  for (int s = 0; s < num; ++s) {
    ras_status r = finish_info(ctxs[s], hst[s], h_ctl, hsub[s].data(), mode,
                               infos ? &infos[s] : nullptr, ms, kms, grid);
    if (first == RAS_OK && r != RAS_OK) first = r;
  }
  return first;
}

ras_status ras_solve_begin(ras_ctx *c, const double *b, double *x, double tol) {
  if (!c || !b || !x || !(tol > 0.0)) return RAS_EINVAL;
  *c->h_sysdesc = make_sysdesc(c, b, x, tol);
  CUDA_TRY(cudaMemcpyAsync(c->d_sysdesc, c->h_sysdesc, sizeof(SysDesc), cudaMemcpyHostToDevice,
                           c->stream));
  Launch L{};
  L.sys = c->d_sysdesc;
  L.nsys = 1;
  L.items = c->plan.d_items;
  CUDA_TRY(launch_init(L, (int)c->plan.items.size(), c->stream));
  CUDA_TRY(cudaEventRecord(c->ev_begin, c->stream));
  c->begun = true;
  c->finished = false;
  return RAS_OK;
}

namespace {

// Launch plan and device buffers of the last batch step on this host thread;
// reused while the same contexts, in the same order, are stepped.
struct StepCache {
  std::vector<uint64_t> key;  // serials of the stepped contexts, in order
  int32_t mode = -1;
  int64_t step_limit = -1, max_updates = -1;
  cudaGraphExec_t graph = nullptr;  // captured step sequence (null: launch directly)
  bool graph_failed = false;
  cudaStream_t cap_stream = nullptr;  // private stream the step is captured on
  LaunchPlan plan;
  SysDesc *d_sys = nullptr;
  GridCtl *d_ctl = nullptr;
  SysDesc *h_sys = nullptr;  // pinned
  GridCtl *h_ctl = nullptr;  // pinned
  SysState *h_st = nullptr;  // pinned
  int cap = 0;
  void release() {
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
    graph_failed = false;
    if (cap_stream) cudaStreamDestroy(cap_stream);
    cap_stream = nullptr;
    plan.release();
    cudaFree(d_sys);
    cudaFree(d_ctl);
    cudaFreeHost(h_sys);
    cudaFreeHost(h_ctl);
    cudaFreeHost(h_st);
    d_sys = nullptr;
    d_ctl = nullptr;
    h_sys = nullptr;
    h_ctl = nullptr;
    h_st = nullptr;
    cap = 0;
    key.clear();
  }
  ~StepCache() { release(); }
};
thread_local StepCache g_step;

}  // namespace

ras_status ras_batch_step(ras_ctx *const *ctxs, int32_t num, int32_t mode, int64_t step_limit,
                          int64_t max_updates, int32_t *done, ras_solve_info *infos) {
  if (!ctxs || num <= 0 || step_limit <= 0 || (mode != RAS_SYNC && mode != RAS_ASYNC && mode != RAS_ASYNC_DECENTRAL))
    return RAS_EINVAL;
  for (int s = 0; s < num; ++s) {
    if (!ctxs[s] || !ctxs[s]->begun || ctxs[s]->exec_kind != ctxs[0]->exec_kind ||
        ctxs[s]->ls.prec != ctxs[0]->ls.prec || ctxs[s]->ls.inner_iters != ctxs[0]->ls.inner_iters)
      return RAS_EINVAL;
    for (int t = 0; t < s; ++t)
      if (ctxs[t] == ctxs[s]) return RAS_EINVAL;
  }
  ras_ctx *c0 = ctxs[0];
  cudaStream_t stream = c0->stream;
  StepCache &sc = g_step;
  std::vector<uint64_t> key(num);
  for (int s = 0; s < num; ++s) key[s] = ctxs[s]->serial;
  if (key != sc.key) {
    sc.release();
    std::vector<Item> items;
    std::vector<double> cost;
    int Wmax = 0, npad_max = 0, kmax = 0;
    for (int s = 0; s < num; ++s) {
      ras_ctx *c = ctxs[s];
      for (int p = 0; p < c->P; ++p) {
        items.push_back({s, p, 0, 0});
        cost.push_back(c->cost[p]);
      }
      Wmax = std::max(Wmax, c->plan.Wmax);
      npad_max = std::max(npad_max, c->plan.npad_max);
      kmax = std::max(kmax, c->K);
    }
    ras_status rs = plan_launch(sc.plan, c0->exec_kind, c0->ls.prec, items, cost, Wmax, npad_max,
                                kmax, stream);
    if (rs != RAS_OK) {
      sc.release();
      return rs;
    }
    if (dev_malloc(&sc.d_sys, sizeof(SysDesc) * num) != cudaSuccess ||
        dev_malloc(&sc.d_ctl, sizeof(GridCtl)) != cudaSuccess ||
        host_malloc_pinned(&sc.h_sys, sizeof(SysDesc) * num) != cudaSuccess ||
        host_malloc_pinned(&sc.h_ctl, sizeof(GridCtl)) != cudaSuccess ||
        host_malloc_pinned(&sc.h_st, sizeof(SysState) * num) != cudaSuccess) {
      sc.release();
      return RAS_ENOMEM;
    }
    sc.cap = num;
    sc.key = key;
  }
  int running = 0;
  for (int s = 0; s < num; ++s) {
    sc.h_sys[s] = *ctxs[s]->h_sysdesc;
    if (!ctxs[s]->finished) ++running;
    if (ctxs[s]->stream != stream) CUDA_TRY(cudaStreamWaitEvent(stream, ctxs[s]->ev_begin, 0));
  }
  Launch L{};
  L.sys = sc.d_sys;
  L.nsys = num;
  L.mode = mode;
  L.items = sc.plan.d_items;
  L.cta_off = sc.plan.d_cta_off;
  L.cta_sys = sc.plan.d_cta_sys;
  L.cta_sys_off = sc.plan.d_cta_sys_off;
  L.ctl = sc.d_ctl;
  L.max_updates = max_updates > 0 ? max_updates : 1000000;
  L.step_limit = step_limit;
  L.timeout_ns = timeout_ns();
  L.solve_limit_ns = env_int("RAS_SOLVE_LIMIT_MS", 120000) * 1000000ll;
  // the leader-based scheme stops on any fully converged neighbourhood, so a
  // failed global check is routine there: it resumes until max_updates
  L.max_restarts = mode == RAS_ASYNC_DECENTRAL ? (1 << 30) : 8;
  L.fresh = (int32_t)env_int("RAS_ASYNC_FRESH", 0);
  L.consistent = (int32_t)env_int("RAS_ASYNC_CONSISTENT", 0);
  L.m = c0->ls.inner_iters;
  L.Wmax = sc.plan.Wmax;
  L.npad_max = sc.plan.npad_max;
  L.persist = 0;
  L.kmax = sc.plan.kmax;
  L.nstages = sc.plan.nstages;
  std::memset(sc.h_ctl, 0, sizeof(GridCtl));
  sc.h_ctl->remaining = running;
  const int nitems = (int)sc.plan.items.size();
  // The whole step: descriptors in (from pinned staging, read at execution
  // time), the persistent launch, copy-back, residual, state out.
  auto issue = [&](cudaStream_t sm) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(sc.d_sys, sc.h_sys, sizeof(SysDesc) * num,
                                    cudaMemcpyHostToDevice, sm);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sc.d_ctl, sc.h_ctl, sizeof(GridCtl), cudaMemcpyHostToDevice, sm);
    if (e == cudaSuccess)
      e = launch_main(c0->exec_kind, c0->ls.prec, sc.plan.nt, L, sc.plan.grid, sc.plan.smem, sm);
    if (e == cudaSuccess && mode == RAS_SYNC) e = launch_copyback(L, nitems, sm);
    if (e == cudaSuccess) e = launch_residual(L, nitems, sm);
    for (int s = 0; s < num && e == cudaSuccess; ++s)
      e = cudaMemcpyAsync(&sc.h_st[s], ctxs[s]->d_st, sizeof(SysState), cudaMemcpyDeviceToHost, sm);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sc.h_ctl, sc.d_ctl, sizeof(GridCtl), cudaMemcpyDeviceToHost, sm);
    return e;
  };
  if (sc.mode != mode || sc.step_limit != step_limit || sc.max_updates != max_updates) {
    if (sc.graph) cudaGraphExecDestroy(sc.graph);
    sc.graph = nullptr;
    sc.graph_failed = false;
    sc.mode = mode;
    sc.step_limit = step_limit;
    sc.max_updates = max_updates;
  }
  const bool use_graph = env_int("RAS_STEP_GRAPH", 1) != 0;
  if (use_graph && !sc.graph && !sc.graph_failed) {
    // captured on a private stream, so work other host threads put on the
    // caller's stream meanwhile is never swept into the graph
    cudaGraph_t gr = nullptr;
    cudaError_t e = sc.cap_stream ? cudaSuccess
                                  : cudaStreamCreateWithFlags(&sc.cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(sc.cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t ei = issue(sc.cap_stream);
      e = cudaStreamEndCapture(sc.cap_stream, &gr);
      if (ei != cudaSuccess) e = ei;
    }
    if (e == cudaSuccess && gr) e = cudaGraphInstantiate(&sc.graph, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      sc.graph = nullptr;
      sc.graph_failed = true;  // capture refused: launch directly from now on
      cudaGetLastError();
    }
  }
  if (sc.graph) CUDA_TRY(cudaGraphLaunch(sc.graph, stream));
  else CUDA_TRY(issue(stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  ras_status first = sc.h_ctl->status != 0 ? (ras_status)sc.h_ctl->status : RAS_OK;
  std::vector<int> newly;
  for (int s = 0; s < num; ++s) {
    const SysState &st = sc.h_st[s];
    const bool fin = mode == RAS_SYNC ? st.done != 0 : (st.word & 3u) == (uint32_t)kDone;
    if (fin && !ctxs[s]->finished) newly.push_back(s);
    if (fin) ctxs[s]->finished = true;
    if (done) done[s] = ctxs[s]->finished ? 1 : 0;
  }
  for (int s : newly) {
    ras_ctx *c = ctxs[s];
    CUDA_TRY(cudaMemcpyAsync(c->h_sub, c->d_sub, sizeof(SubState) * c->P, cudaMemcpyDeviceToHost,
                             stream));
  }
  if (!newly.empty()) CUDA_TRY(cudaStreamSynchronize(stream));
  for (int s : newly) {
    ras_ctx *c = ctxs[s];
    ras_solve_info tmp{};
    ras_status r = finish_info(c, sc.h_st[s], *sc.h_ctl, c->h_sub, mode, &tmp, 0.f, 0.f, sc.plan.grid);
    if (infos) infos[s] = tmp;
    if (first == RAS_OK && r != RAS_OK) first = r;
  }
  return first;
}

ras_status ras_autotune(ras_ctx *c, double *x_scratch, int32_t mode, int32_t iters,
                        int32_t tune_inner, ras_tune_result *out) {
  if (!c || !x_scratch || iters <= 0 || (mode != RAS_SYNC && mode != RAS_ASYNC && mode != RAS_ASYNC_DECENTRAL))
    return RAS_EINVAL;
  // homogeneous problem A x = 0 from x = 1: the error is x itself, dominated
  // by the smoothest modes, so a short window sees the asymptotic rate
  if (!c->d_bx) {
    ras_status s = c->alloc(c->d_bx, 2 * (size_t)c->n);
    if (s != RAS_OK) return s;
  }
  double *b = c->d_bx;
  CUDA_TRY(cudaMemsetAsync(b, 0, sizeof(double) * c->n, c->stream));
  // candidates: kernel variant and CTA threads, inner steps, and the launch
  // shape: asynchronous schedule (tickets on every slot, or the static
  // assignment) and a cap on the CTAs (every co-resident slot, or half of the
  // subdomains: two subdomains per CTA at least, fewer CTAs per SM)
  struct Cand {
    int exec_kind, nt, m, sched, grid_cap;
  };
  std::vector<Cand> cands;
  const int kind = c->ls.kind, prec = c->ls.prec, m0 = c->ls.inner_iters;
  std::vector<int> ms = {m0};
  const bool banded = kind == RAS_LOCAL_BANDCHOL || kind == RAS_LOCAL_BANDLU;
  if (tune_inner && !banded) {
    ms.push_back(std::max(1, m0 / 2));
    // GMRES: the Krylov scratch holds at most the set-up step count
    if (kind != RAS_LOCAL_GMRES) ms.push_back(2 * m0);
  }
  const bool async = mode != RAS_SYNC;
  const std::vector<std::pair<int, int>> shapes = {{1, 0}, {0, 0}, {0, (c->P + 1) / 2}};
  for (int m : ms) {
    std::vector<std::pair<int, int>> variants;  // (exec_kind, threads)
    if (banded) {
      variants = {{kBand, 128}, {kBand, 256}};
    } else {
      const int ek = kind == RAS_LOCAL_GMRES ? kGMRES : kind;
      variants = {{ek, 256}, {ek, 512}};
      if (kind == RAS_LOCAL_CG && prec == RAS_FP32 && c->d_lcol16) variants.push_back({kCGS, 512});
    }
    for (auto &v : variants)
      for (auto &sh : shapes) cands.push_back({v.first, v.second, m, sh.first, sh.second});
  }
  std::vector<Item> items(c->P);
  for (int p = 0; p < c->P; ++p) items[p] = {0, p, 0, 0};
  const Cand saved = {c->exec_kind, c->nt_pref, m0, c->sched, c->grid_cap};
  double best = -1.0;
  Cand pick = saved;
  int tried = 0, pick_grid = 0;
  for (const Cand &cd : cands) {
    LaunchPlan pl;
    if (plan_launch(pl, cd.exec_kind, prec, items, c->cost, c->plan.Wmax, c->plan.npad_max, c->K,
                    c->stream, cd.nt, cd.grid_cap) != RAS_OK) {
      pl.release();
      continue;
    }
    std::swap(pl, c->plan);
    const int ek = c->exec_kind, sk = c->sched;
    c->exec_kind = cd.exec_kind;
    c->ls.inner_iters = cd.m;
    c->sched = cd.sched;
    // window 1 (transient), then window 2 from its result (timed): the score
    // is the residual reduction per kernel millisecond of window 2
    CUDA_TRY(launch_fill(x_scratch, 1.0, c->n, c->stream));
    ras_solve_info info1{}, info{};
    ras_status rs = ras_solve(c, b, x_scratch, 1e-300, mode, iters, &info1);
    if (rs == RAS_OK || rs == RAS_ENOCONV) rs = ras_solve(c, b, x_scratch, 1e-300, mode, iters, &info);
    std::swap(pl, c->plan);
    c->exec_kind = ek;
    c->sched = sk;
    pl.release();
    if (rs != RAS_OK && rs != RAS_ENOCONV) continue;
    ++tried;
    const double red = std::log(std::max(info1.relres, 1e-300) / std::max(info.relres, 1e-300));
    const double score = red / std::max(info.kernel_ms, 1e-6);
    if (score > best) {
      best = score;
      pick = cd;
      pick_grid = info.grid;
    }
  }
  c->ls.inner_iters = pick.m;
  c->exec_kind = pick.exec_kind;
  c->nt_pref = pick.nt;
  c->sched = pick.sched;
  c->grid_cap = pick.grid_cap;
  if (pick.exec_kind != saved.exec_kind || pick.nt != saved.nt || pick.grid_cap != saved.grid_cap) {
    ras_status st = plan_launch(c->plan, c->exec_kind, prec, items, c->cost, c->plan.Wmax,
                                c->plan.npad_max, c->K, c->stream, c->nt_pref, c->grid_cap);
    if (st != RAS_OK) return st;
  }
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->cta_threads = c->plan.nt;
    out->staged = c->exec_kind == kCGS ? 1 : 0;
    out->inner_iters = c->ls.inner_iters;
    out->candidates = tried;
    out->score = best;
    out->schedule = pick.sched;
    out->grid = pick_grid;
    out->per_cta = pick.sched == 1
                       ? 0
                       : (int32_t)((c->P + c->plan.grid - 1) / std::max(c->plan.grid, 1));
  }
  return tried > 0 ? RAS_OK : RAS_ENOTSUP;
}

ras_status ras_get_maps(const ras_ctx *c, int32_t p, const int32_t **omega, int32_t *n_omega,
                        const uint8_t **owned_mask, const int32_t **iface, int32_t *n_iface) {
  if (!c || p < 0 || p >= c->P || !omega || !n_omega || !owned_mask || !iface || !n_iface)
    return RAS_EINVAL;
  *omega = c->omega[p].data();
  *n_omega = (int32_t)c->omega[p].size();
  *owned_mask = c->owned[p].data();
  *iface = c->iface[p].data();
  *n_iface = (int32_t)c->iface[p].size();
  return RAS_OK;
}

ras_status ras_get_info(const ras_ctx *c, int32_t *num_parts, int32_t *n, int32_t *max_bandwidth,
                        int64_t *device_bytes) {
  if (!c) return RAS_EINVAL;
  if (num_parts) *num_parts = c->P;
  if (n) *n = c->n;
  if (max_bandwidth) *max_bandwidth = c->maxw;
  if (device_bytes) *device_bytes = c->device_bytes;
  return RAS_OK;
}

ras_status ras_get_update_counts(const ras_ctx *c, int64_t *counts) {
  if (!c || !counts) return RAS_EINVAL;
  std::copy(c->last_updates.begin(), c->last_updates.end(), counts);
  return RAS_OK;
}

ras_status ras_get_launch(const ras_ctx *c, int32_t *kernel_variant, int32_t *cta_threads,
                          int32_t *grid, int32_t *inner_iters) {
  if (!c) return RAS_EINVAL;
  if (kernel_variant) *kernel_variant = c->exec_kind == kCGS && c->dia ? 5 : c->exec_kind;
  if (cta_threads) *cta_threads = c->plan.nt;
  if (grid) *grid = c->plan.grid;
  if (inner_iters) *inner_iters = c->ls.inner_iters;
  return RAS_OK;
}

ras_status ras_get_phase_times(const ras_ctx *c, uint64_t *ns) {
  if (!c || !ns) return RAS_EINVAL;
  if (c->last_phase.size() != 3 * (size_t)c->P) return RAS_EINVAL;
  std::copy(c->last_phase.begin(), c->last_phase.end(), ns);
  return RAS_OK;
}

ras_status ras_relres(ras_ctx *c, const double *b, const double *x, double *relres) {
  if (!c || !b || !x || !relres) return RAS_EINVAL;
  *c->h_sysdesc = make_sysdesc(c, b, const_cast<double *>(x), 1.0);
  CUDA_TRY(cudaMemcpyAsync(c->d_sysdesc, c->h_sysdesc, sizeof(SysDesc), cudaMemcpyHostToDevice,
                           c->stream));
  Launch L{};
  L.sys = c->d_sysdesc;
  L.nsys = 1;
  L.items = c->plan.d_items;
  const int nitems = (int)c->plan.items.size();
  CUDA_TRY(launch_init(L, nitems, c->stream));
  CUDA_TRY(launch_residual(L, nitems, c->stream));
  CUDA_TRY(cudaMemcpyAsync(c->h_st, c->d_st, sizeof(SysState), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  const SysState &st = *c->h_st;
  *relres = st.b2 > 0 ? std::sqrt(st.res2 / st.b2) : std::sqrt(st.res2);
  return RAS_OK;
}

}  // extern "C"
