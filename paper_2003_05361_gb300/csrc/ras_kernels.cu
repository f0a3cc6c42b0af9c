// Device code of the GB300 Restricted Additive Schwarz solver (sm_103a).
//
// Kernels:
//   band_chol_kernel     setup: banded Cholesky A_p = L L^T in FP64, one CTA per
//                        subdomain, sliding (w+1)x(w+1) window in shared memory
//                        (direct local solver of Sec. 3.3.1, factorised once).
//   band_lu_kernel       setup: banded LU A_p = L U without pivoting in FP64
//                        for general (nonsymmetric) systems, sliding
//                        (w+1)x(2w+1) window (the LU local solver of Sec. 4.1).
//   band_layout_kernel   setup: turns L and U into the per-block records read
//                        by the chained triangular solves ([inverse 32x32
//                        diagonal block | window operator]), rounded to the
//                        storage precision (FP64 / FP32 / BF16).
//   ras_init_kernel      per solve: ||b||^2 over Omega_p and O_p, state reset.
//   ras_sysnorm_kernel   per solve: per-system sums in a fixed order.
//   ras_main_kernel      the persistent RAS kernel, one CTA per group of
//                        subdomains. RAS_SYNC: iterations separated by a
//                        grid-wide barrier (synchronous Schwarz, Sec. 2.1).
//                        RAS_ASYNC: no barrier; owned values are published with
//                        a release store of a per-subdomain version counter and
//                        neighbours acquire it before reading (asynchronous
//                        Schwarz, Sec. 2.1 / one-sided exchange of Sec. 3.4);
//                        convergence by the local criterion of Eq. 2, a global
//                        converged counter (RAS_ASYNC) or flags flooded
//                        between neighbours (RAS_ASYNC_DECENTRAL), and the
//                        post-termination global check of Sec. 3.3.2.
//   ras_residual_kernel  ||b - A x||^2 partials over owned rows.
//   ras_copyback_kernel  moves a sync result left in the second buffer to x.
//
// Every device-side wait (grid barrier, the staged CG's mbarrier, idle
// polling) is bounded by a %globaltimer limit; on expiry the kernel records
// RAS_ETIMEOUT in GridCtl, raises the abort flag, drains its own bulk copies
// and returns. The band chain's cp.async copies are waited for with
// cp.async.wait_group, which completes by construction.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ras_convert.h"
#include "ras_internal.h"
#include "ras_launch.h"

namespace ras {

// --------------------------------------------------------------------------
// small PTX helpers
// --------------------------------------------------------------------------

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t atom_cas_acquire_u32(uint32_t *p, uint32_t cmp, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acquire.gpu.global.cas.b32 %0, [%1], %2, %3;"
               : "=r"(old)
               : "l"(p), "r"(cmp), "r"(v)
               : "memory");
  return old;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_s32(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_s32(int *p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_s32(const int *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ double ld_relaxed_f64(const double *p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void st_relaxed_f64(double *p, double v) {
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void set_error(GridCtl *c, int code, unsigned long long info) {
  if (atomicCAS(&c->status, 0, code) == 0) c->err_info = info;
  atomicExch(&c->abort, 1);
}

template <typename T> struct CTypeOf { using type = float; };
template <> struct CTypeOf<double> { using type = double; };

template <typename T> __device__ __forceinline__ T from_double(double v);
template <> __device__ __forceinline__ double from_double<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_double<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double v) {
  return __double2bfloat16(v);
}
__device__ __forceinline__ float to_ct(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_ct(float v) { return v; }
__device__ __forceinline__ double to_ct(double v) { return v; }

// The local right-hand side in the local-solve type: for FP32 by integer
// arithmetic on the bit patterns (ras_convert.h), off the slow FP64 unit.
template <typename CT> __device__ __forceinline__ CT rhs_from_f64(double v) { return (CT)v; }
template <> __device__ __forceinline__ float rhs_from_f64<float>(double v) { return f64_to_f32_rn(v); }

// Deterministic CTA reduction: butterfly inside each warp, then every thread
// adds the per-warp values in the same order, so all threads hold the same
// bit pattern. red must hold NT/32 values.
template <int NT, typename V>
__device__ __forceinline__ V block_sum(V v, V *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  V s = red[0];
#pragma unroll
  for (int i = 1; i < NT / 32; ++i) s += red[i];
  return s;
}

// Same deterministic sum with a single barrier: callers alternate between two
// buffers, so a buffer is rewritten only after every thread has passed the
// barrier of the reduction in between.
template <int NT, typename V>
__device__ __forceinline__ V block_sum_1b(V v, V *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  V s = red[0];
#pragma unroll
  for (int i = 1; i < NT / 32; ++i) s += red[i];
  return s;
}

template <int NT>
__device__ __forceinline__ void block_sum2(double &a, double &b, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = a;
    red[NT / 32 + (threadIdx.x >> 5)] = b;
  }
  __syncthreads();
  double sa = red[0], sb = red[NT / 32];
#pragma unroll
  for (int i = 1; i < NT / 32; ++i) {
    sa += red[i];
    sb += red[NT / 32 + i];
  }
  a = sa;
  b = sb;
}

// Fixed-order sum of the P per-subdomain partials of one system by one warp
// (lane-strided sequential sums, then a butterfly). Same bits in every CTA.
__device__ __forceinline__ double warp_sum_partials(const SubState *sub, int P, int slot,
                                                    bool relaxed) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int p = lane; p < P; p += 32)
    s += relaxed ? ld_relaxed_f64(&sub[p].part[slot]) : sub[p].part[slot];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// --------------------------------------------------------------------------
// grid barrier (co-resident CTAs of a cooperative launch)
// --------------------------------------------------------------------------

// All CTAs arrive; `fin` systems finished by this CTA since the last barrier
// are folded into GridCtl::remaining by the last arriver before it releases
// the generation, so every CTA reads the same `remaining` afterwards.
__device__ bool grid_barrier(GridCtl *c, int fin, int64_t timeout_ns, int *s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (fin) atomicAdd(&c->fin_accum, fin);
    const uint32_t gen = ld_acquire_u32(&c->gen);
    __threadfence();
    const unsigned int arrived = atomicAdd(&c->count, 1u);
    if (arrived == gridDim.x - 1) {
      c->count = 0;
      c->ticket = 0;  // next synchronous iteration of the dynamic schedule
      const int f = atomicExch(&c->fin_accum, 0);
      if (f) atomicSub(&c->remaining, f);
      __threadfence();
      st_release_u32(&c->gen, gen + 1);
    } else {
      const uint64_t t0 = gtimer();
      uint32_t spins = 0;
      while (ld_acquire_u32(&c->gen) == gen) {
        if ((++spins & 63u) == 0) {
          if (ld_relaxed_s32(&c->abort)) { ok = 0; break; }
          if ((int64_t)(gtimer() - t0) > timeout_ns) {
            set_error(c, kETIMEOUT, 1);
            ok = 0;
            break;
          }
        }
      }
    }
    if (ld_relaxed_s32(&c->abort)) ok = 0;
    s_flag[0] = ok;
    s_flag[1] = ld_relaxed_s32(&c->remaining);
  }
  __syncthreads();
  return s_flag[0] != 0;
}

// --------------------------------------------------------------------------
// asynchronous copies: 1D bulk copies (TMA) with an mbarrier for the staged CG,
// per-thread cp.async for the band chain
// --------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void bulk_copy_nobar_arrive(void *dst, const void *src, uint32_t bytes,
                                                       uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; returns false on timeout (error recorded by the caller).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int64_t timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (!mbar_try_wait(bar, parity))
    if ((int64_t)(gtimer() - t0) > timeout_ns) return false;
  return true;
}

// 16-byte asynchronous global -> shared copies (L2 only), tracked per thread
// by commit groups.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// --------------------------------------------------------------------------
// setup: banded Cholesky (FP64)
// --------------------------------------------------------------------------

// band (row-major, ld = w+1): band[i*ld + t] = A[i][i-w+t]; overwritten by L.
// Right-looking: for column j, L_jj = sqrt(a_jj), L_ij = a_ij / L_jj for
// i in (j, j+w], then a_ik -= L_ij L_kj on the trailing triangle. Rows j..j+w
// live in a circular window of shared memory (slot = row mod (w+1)).
__global__ void __launch_bounds__(256) band_chol_kernel(const BandJob *jobs, double *band,
                                                        GridCtl *ctl) {
  extern __shared__ __align__(16) double win[];
  __shared__ double s_piv;
  __shared__ int s_bad;
  const BandJob jb = jobs[blockIdx.x];
  const int n = jb.n, w = jb.w, ld = w + 1;
  double *B = band + jb.band_off;
  const int tid = threadIdx.x, NT = blockDim.x;
  for (int e = tid; e < ld * ld; e += NT) {
    const int r = e / ld;
    win[e] = r < n ? B[(int64_t)r * ld + (e % ld)] : 0.0;
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const int sj = j % ld;
    if (j > 0) {
      // row j-1 is final: write it out, load row j+w into its slot
      const int sp = (j - 1) % ld;
      const int rin = j + w;
      for (int t = tid; t < ld; t += NT) {
        B[(int64_t)(j - 1) * ld + t] = win[sp * ld + t];
        win[sp * ld + t] = rin < n ? B[(int64_t)rin * ld + t] : 0.0;
      }
      __syncthreads();
    }
    if (tid == 0) {
      const double a = win[sj * ld + w];
      if (!(a > 0.0)) {
        s_bad = 1;
      } else {
        const double d = sqrt(a);
        win[sj * ld + w] = d;
        s_piv = d;
      }
    }
    __syncthreads();
    if (s_bad) break;
    const double d = s_piv;
    const int nr = min(w, n - 1 - j);  // rows j+1 .. j+nr
    for (int q = tid; q < nr; q += NT) {
      const int i = j + 1 + q;
      win[(i % ld) * ld + (j - i + w)] /= d;
    }
    __syncthreads();
    for (int e = tid; e < nr * nr; e += NT) {
      const int qi = e / nr, qk = e % nr;
      if (qk > qi) continue;
      const int i = j + 1 + qi, k = j + 1 + qk;
      const int si = i % ld, sk = k % ld;
      win[si * ld + (k - i + w)] -= win[si * ld + (j - i + w)] * win[sk * ld + (j - k + w)];
    }
    __syncthreads();
  }
  if (s_bad) {
    if (tid == 0) set_error(ctl, kENOTSPD, (unsigned long long)blockIdx.x);
    return;
  }
  // flush the last row
  if (n > 0) {
    const int sl = (n - 1) % ld;
    for (int t = tid; t < ld; t += NT) B[(int64_t)(n - 1) * ld + t] = win[sl * ld + t];
  }
}

// --------------------------------------------------------------------------
// setup: banded LU without pivoting (FP64), for general A_p
// --------------------------------------------------------------------------

// band (row-major, ld = 2w+1): band[i*ld + t] = A[i][i-w+t]; overwritten by
// the unit lower L (t < w) and U (t >= w). Right-looking: for column j the
// pivot u_jj, the multipliers l_ij = a_ij / u_jj for i in (j, j+w], then
// a_ik -= l_ij u_jk on the trailing (w x w) block. Rows j..j+w live in a
// circular window of shared memory (slot = row mod (w+1)). A zero pivot
// stops the factorisation with kENOTSPD (no pivoting: the local matrices of
// an M-matrix, or of any diagonally dominant matrix, never need it).
__global__ void __launch_bounds__(256) band_lu_kernel(const BandJob *jobs, double *band,
                                                      GridCtl *ctl) {
  extern __shared__ __align__(16) double win[];
  __shared__ double s_piv;
  __shared__ int s_bad;
  const BandJob jb = jobs[blockIdx.x];
  const int n = jb.n, w = jb.w, ld = 2 * w + 1, nw = w + 1;
  double *B = band + jb.band_off;
  const int tid = threadIdx.x, NT = blockDim.x;
  for (int e = tid; e < nw * ld; e += NT) {
    const int r = e / ld;
    win[e] = r < n ? B[(int64_t)r * ld + (e % ld)] : 0.0;
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const int sj = j % nw;
    if (j > 0) {
      // row j-1 is final: write it out, load row j+w into its slot
      const int sp = (j - 1) % nw;
      const int rin = j + w;
      for (int t = tid; t < ld; t += NT) {
        B[(int64_t)(j - 1) * ld + t] = win[sp * ld + t];
        win[sp * ld + t] = rin < n ? B[(int64_t)rin * ld + t] : 0.0;
      }
      __syncthreads();
    }
    if (tid == 0) {
      const double u = win[sj * ld + w];
      if (!(fabs(u) > 0.0)) s_bad = 1;
      s_piv = u;
    }
    __syncthreads();
    if (s_bad) break;
    const double u = s_piv;
    const int nr = min(w, n - 1 - j);  // rows (and columns) j+1 .. j+nr
    for (int q = tid; q < nr; q += NT) {
      const int i = j + 1 + q;
      win[(i % nw) * ld + (j - i + w)] /= u;
    }
    __syncthreads();
    for (int e = tid; e < nr * nr; e += NT) {
      const int qi = e / nr, qk = e % nr;
      const int i = j + 1 + qi, k = j + 1 + qk;
      const int si = i % nw;
      win[si * ld + (k - i + w)] -= win[si * ld + (j - i + w)] * win[sj * ld + (k - j + w)];
    }
    __syncthreads();
  }
  if (s_bad) {
    if (tid == 0) set_error(ctl, kENOTSPD, (unsigned long long)blockIdx.x);
    return;
  }
  if (n > 0) {
    const int sl = (n - 1) % nw;
    for (int t = tid; t < ld; t += NT) B[(int64_t)(n - 1) * ld + t] = win[sl * ld + t];
  }
}

// --------------------------------------------------------------------------
// setup: operators of the blocked triangular solves
// --------------------------------------------------------------------------
//
// Rows are grouped in blocks of 32 (K = 0..nb-1; rows >= n are identity rows).
// With L_KK the diagonal block of the lower factor and W = the local
// half-bandwidth w, forward substitution block by block is
//   y_K = L_KK^{-1} (r_K - L_{K,left} y_left) = t_K - M_K y[32K-W, 32K),
//   t_K = L_KK^{-1} r_K,  M_K = L_KK^{-1} L[K rows, 32K-W .. 32K)   (32 x W)
// and backward substitution with the upper factor U
//   z_K = t'_K - M'_K z[32K+32, 32K+32+W),  t'_K = U_KK^{-1} y_K,
//   M'_K = U_KK^{-1} U[K rows, 32K+32 .. 32K+32+W)                   (32 x W).
// Cholesky: L from the band (ld = w+1), U = L^T, so U_KK^{-1} = (L_KK^{-1})^T.
// LU: unit lower L and U from one band (ld = 2w+1), U_KK inverted on its own.
// Per subdomain the storage is nb forward records, then nb backward records,
// each a column-major 32 x (32 + W) matrix (entry (l, j) at j*32 + l):
//   forward  record K = [ L_KK^{-1} | M_K  ],
//   backward record K = [ U_KK^{-1} | M'_K ],
// so that a chain step reads one contiguous record and every one of its
// 32 + W columns is applied to one broadcast value (the step's own right-hand
// side for the first 32, a finished window row for the rest).
template <typename T, bool LU>
__global__ void __launch_bounds__(32) band_layout_kernel(const LayoutJob *jobs,
                                                         const double *band, T *fac) {
  __shared__ double Lkk[32][33];
  __shared__ double X[32][33];              // L_KK^{-1}
  __shared__ double Y[LU ? 32 : 1][33];     // U_KK^{-1} (LU)
  const LayoutJob jb = jobs[blockIdx.x];
  const int l = threadIdx.x;
  const int n = jb.n, w = jb.w, W = jb.W, K = jb.K, nb = jb.nb, ld = LU ? 2 * w + 1 : w + 1;
  const double *Bd = band + jb.band_off;
  const int i = 32 * K + l;
  // entry (r, c) of the band, |c - r| <= w, r < n
  auto at = [&](int r, int c) -> double { return Bd[(int64_t)r * ld + (c - r + w)]; };
  for (int m = 0; m < 32; ++m) {
    double v = 0.0;
    const int jcol = 32 * K + m;
    if (i < n) {
      if (m < l && l - m <= w) v = at(i, jcol);
      else if (m == l) v = LU ? 1.0 : at(i, jcol);
    } else if (m == l) {
      v = 1.0;
    }
    Lkk[l][m] = v;
  }
  __syncwarp();
  {
    // lane m computes column m of the inverse by forward substitution
    const int m = l;
    double col[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      double s = (r == m) ? 1.0 : 0.0;
      if (r >= m) {
        for (int q = m; q < r; ++q) s -= Lkk[r][q] * col[q];
        col[r] = s / Lkk[r][r];
      } else {
        col[r] = 0.0;
      }
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) X[r][m] = col[r];
  }
  __syncwarp();
  if (LU) {
    // U_KK (row l, column m >= l), then lane m computes column m of its
    // inverse by backward substitution
    for (int m = 0; m < 32; ++m) {
      double v = 0.0;
      const int jcol = 32 * K + m;
      if (i < n) {
        if (m >= l && m - l <= w && jcol < n) v = at(i, jcol);
      } else if (m == l) {
        v = 1.0;
      }
      Lkk[l][m] = v;
    }
    __syncwarp();
    const int m = l;
    double col[32];
#pragma unroll
    for (int r = 31; r >= 0; --r) {
      double s = (r == m) ? 1.0 : 0.0;
      if (r <= m) {
        for (int q = r + 1; q <= m; ++q) s -= Lkk[r][q] * col[q];
        col[r] = s / Lkk[r][r];
      } else {
        col[r] = 0.0;
      }
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) Y[LU ? r : 0][m] = col[r];
    __syncwarp();
  }
  const int64_t rec = (int64_t)32 * (W + 32);
  T *F = fac + jb.fac_off + (int64_t)K * rec;
  T *Bk = fac + jb.fac_off + (int64_t)nb * rec + (int64_t)K * rec;
  for (int m = 0; m < 32; ++m) {
    F[m * 32 + l] = from_double<T>(X[l][m]);                           // L_KK^{-1}[l][m]
    Bk[m * 32 + l] = from_double<T>(LU ? Y[LU ? l : 0][m] : X[m][l]);  // U_KK^{-1}[l][m]
  }
  // M_K[l][c] = sum_{m <= l} Linv[l][m] L[32K+m][32K-W+c]
  for (int c = 0; c < W; ++c) {
    const int col = 32 * K - W + c;
    double s = 0.0;
    if (col >= 0)
      for (int m = 0; m <= l; ++m) {
        const int r = 32 * K + m;
        if (r < n && col >= r - w) s += X[l][m] * at(r, col);
      }
    F[(int64_t)(32 + c) * 32 + l] = from_double<T>(s);
  }
  // M'_K[l][c] = sum_{m >= l} Uinv[l][m] U[32K+m][32K+32+c]
  // (Cholesky: U[a][b] = L[b][a])
  for (int c = 0; c < W; ++c) {
    const int r = 32 * K + 32 + c;
    double s = 0.0;
    if (r < n)
      for (int m = l; m < 32; ++m) {
        const int col = 32 * K + m;
        if (col >= r - w) s += LU ? Y[LU ? l : 0][m] * at(col, r) : X[m][l] * at(r, col);
      }
    Bk[(int64_t)(32 + c) * 32 + l] = from_double<T>(s);
  }
}

// --------------------------------------------------------------------------
// per-solve helpers
// --------------------------------------------------------------------------

// One CTA per item: ||b||^2 over Omega_p and O_p, reset of the subdomain state.
__global__ void __launch_bounds__(128) ras_init_kernel(Launch L) {
  __shared__ double red[8];
  const Item it = L.items[blockIdx.x];
  const SysDesc S = L.sys[it.sys];
  const SubDesc D = S.subs[it.p];
  double a = 0.0, o = 0.0;
  for (int i = threadIdx.x; i < D.n; i += 128) {
    const uint8_t f = S.ownf[D.row_off + i];  // 1 owned, 0 overlap, 2 hole row
    const double v = f == 2 ? 0.0 : S.b[S.gidx[D.row_off + i]];
    a += v * v;
    if (f == 1) o += v * v;
  }
  block_sum2<128>(a, o, red);
  if (threadIdx.x == 0) {
    SubState &s = S.sub[it.p];
    s.bloc2 = a;
    s.bown2 = o;
    s.part[0] = s.part[1] = 0.0;
    s.updates = 0;
    s.step_updates = 0;
    s.stale = 0;
    s.nbr_seen = 0;
    s.t_gather = s.t_solve = s.t_update = 0;
    s.version = 0;
    s.conv_epoch = -1;
    s.park_epoch = -1;
    s.check_epoch = -1;
    s.gconv_epoch = -1;
    s.busy = 0;
    s.report = 0xffffffff00000000ull;  // epoch -1: no report
  }
}

// One warp per system: b2 = sum of the owned partials in subdomain order,
// state reset (what = 0), or res2 from part[0] (what = 1).
__global__ void ras_sysnorm_kernel(Launch L, int what) {
  const int s = blockIdx.x;
  if (s >= L.nsys) return;
  const SysDesc S = L.sys[s];
  const int lane = threadIdx.x;
  double acc = 0.0;
  for (int p = lane; p < S.P; p += 32) acc += what == 0 ? S.sub[p].bown2 : S.sub[p].part[0];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    if (what == 0) {
      S.st->b2 = acc;
      S.st->res2 = 0.0;
      S.st->iters = 0;
      S.st->word = kRun;
      S.st->status = 0;
      S.st->done = 0;
      S.st->nconv = 0;
      S.st->nparked = 0;
      S.st->nchecked = 0;
      S.st->restarts = 0;
      S.st->result_alt = 0;
    } else {
      S.st->res2 = acc;
    }
  }
}

// One CTA per item: owned-row residual partial of the system's x.
__global__ void __launch_bounds__(128) ras_residual_kernel(Launch L) {
  __shared__ double red[8];
  const Item it = L.items[blockIdx.x];
  const SysDesc S = L.sys[it.sys];
  const SubDesc D = S.subs[it.p];
  const int K = S.K;
  const int64_t eb = D.row_off * K;
  double o = 0.0, dummy = 0.0;
  for (int i = threadIdx.x; i < D.n; i += 128) {
    if (S.ownf[D.row_off + i] != 1) continue;
    double r = S.b[S.gidx[D.row_off + i]];
    for (int k = 0; k < K; ++k) {
      const int64_t e = eb + (int64_t)k * D.npad + i;
      r -= S.rval[e] * S.x[S.rcol[e]];
    }
    o += r * r;
  }
  block_sum2<128>(o, dummy, red);
  if (threadIdx.x == 0) S.sub[it.p].part[0] = o;
}

// One CTA per item: x[O_p] = xalt[O_p] for systems whose result is in xalt.
__global__ void __launch_bounds__(128) ras_copyback_kernel(Launch L) {
  const Item it = L.items[blockIdx.x];
  const SysDesc S = L.sys[it.sys];
  if (!S.st->result_alt) return;
  const SubDesc D = S.subs[it.p];
  for (int t = threadIdx.x; t < D.n_own; t += 128) {
    const int g = S.gidx[D.row_off + S.own_l[D.own_off + t]];
    S.x[g] = S.xalt[g];
  }
}

// --------------------------------------------------------------------------
// local solvers
// --------------------------------------------------------------------------

// Four consecutive values from 16-byte aligned shared memory.
__device__ __forceinline__ void ld4(const float *p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4 *>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2 *>(p);
  const double2 b = *reinterpret_cast<const double2 *>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// Columns of a band record each warp of an NW-warp CTA takes per chain step:
// ceil((W + 32) / NW) rounded up to a multiple of 4 (W itself is a multiple of
// 4), so every warp's first column, and the broadcast values it reads, are
// 16-byte aligned.
__host__ __device__ inline int band_cols_per_warp(int W, int NW) {
  return ((W + 32 + NW - 1) / NW + 3) / 4 * 4;
}

// Banded Cholesky solve L L^T delta = r by the whole CTA as two block chains:
// forward y_K = L_KK^{-1} r_K - M_K y_window, backward
// z_K = U_KK^{-1} y_K - M'_K z_window. A chain step applies the 32 + W columns
// of one record (see band_layout_kernel) to broadcast values: column j < 32 to
// row 32K + j of the step's own input (r in the forward pass, y in the
// backward pass, read from y before the step overwrites it), window column
// j = 32 + c to finished row 32K - W + c (forward) or 32K + 32 + c (backward).
// Warp w takes the contiguous columns [w tw, (w+1) tw) (band_cols_per_warp)
// and writes its 32 partial sums; after ONE barrier every warp adds the
// partials in the same fixed order, so all warps hold identical y_K. Window
// sums enter with a minus sign.
// Each warp streams its own columns of record s + D - 1 with 16-byte cp.async
// copies into a private D-slot ring while it computes step s; a copy is waited
// for by the thread that issued it and published to the warp by __syncwarp,
// so the chain needs no mbarrier and no second barrier. A slot is refilled one
// step after it was read, behind that step's barrier. Each warp keeps its own
// copy of the last 8 finished blocks in win (row g at g & 255, stored twice,
// at +0 and +256, so that a warp's window rows are one unwrapped run); window
// rows outside [0, npad) meet zero operator columns and read zero-initialised
// slots. y[0..npad) holds r on entry and delta on exit; part holds 2 NT
// partials.
template <typename T, typename CT, int NT, int D>
__device__ void band_solve_chain(const T *__restrict__ F, const T *__restrict__ Bs, int nb, int W,
                                 int twm, CT *y, CT *part, CT *win, T *ring) {
  constexpr int NW = NT / 32;
  constexpr int V = 16 / (int)sizeof(T);  // values per 16-byte copy
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NI = W + 32;
  const int tw = band_cols_per_warp(W, NW);
  const int j0 = warp * tw < NI ? warp * tw : NI;
  const int j1 = j0 + tw < NI ? j0 + tw : NI;
  const int cnt = j1 - j0;
  const int nd = (j1 < 32 ? j1 : 32) - (j0 < 32 ? j0 : 32);  // own-input columns
  const int nchunk = cnt * 32 / V;  // 16-byte chunks of this warp's columns
  const int64_t rec = (int64_t)32 * NI;
  const int slot_len = twm * 32;
  T *rw = ring + (size_t)warp * D * slot_len;
  CT *wy = win + warp * 512;  // two copies of an 8-block ring: reads never wrap
  for (int dir = 0; dir < 2; ++dir) {
    const T *src_l = (dir == 0 ? F : Bs) + (int64_t)j0 * 32 + lane * V;
    T *dst_l = rw + lane * V;
    // copies of chain step s into ring slot sl (one commit group, maybe empty)
    auto issue = [&](int s, int sl) {
      if (s < nb) {
        const T *src = src_l + (dir == 0 ? s : nb - 1 - s) * rec;
        T *dst = dst_l + sl * slot_len;
        for (int q0 = 0; q0 < nchunk; q0 += 128) {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (q0 + u * 32 + lane < nchunk) cp_async16(dst + (q0 + u * 32) * V, src + (q0 + u * 32) * V);
        }
      }
      cp_async_commit();
    };
#pragma unroll
    for (int q = 0; q < 16; ++q) wy[q * 32 + lane] = CT(0);
#pragma unroll
    for (int s = 0; s < D - 1; ++s) issue(s, s);
    int cur = 0;  // slot of step s
    for (int s = 0; s < nb; ++s) {
      issue(s + D - 1, cur == 0 ? D - 1 : cur - 1);
      asm volatile("cp.async.wait_group %0;" ::"n"(D - 1) : "memory");
      __syncwarp();
      const int K = dir == 0 ? s : nb - 1 - s;
      const T *sl = rw + cur * slot_len + lane;
      CT a[4] = {CT(0), CT(0), CT(0), CT(0)};
      int ii = 0;
      if (nd > 0) {
        const CT *ys = y + 32 * K + j0;  // own input rows 32K + j
        for (; ii < nd; ii += 4) {
          CT bv[4];
          ld4(ys + ii, bv);
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (ii + u < nd) a[u] += to_ct(sl[(ii + u) * 32]) * bv[u];
        }
        ii = nd;
      }
      if (ii < cnt) {
        // window row of column j: 32K - W - 32 + j (forward), 32K + j (backward)
        const int g0 = (dir == 0 ? 32 * K - W - 32 : 32 * K) + j0;
        const CT *ws = wy + (g0 & 255);
        for (; ii < cnt; ii += 4) {
          CT bv[4];
          ld4(ws + ii, bv);
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (ii + u < cnt) a[u] -= to_ct(sl[(ii + u) * 32]) * bv[u];
        }
      }
      CT *pb = part + (s & 1) * NT;
      pb[warp * 32 + lane] = (a[0] + a[1]) + (a[2] + a[3]);
      __syncthreads();
      // every warp forms the same y_K
      CT v = CT(0);
#pragma unroll
      for (int w = 0; w < NW; ++w) v += pb[w * 32 + lane];
      wy[(K & 7) * 32 + lane] = v;
      wy[256 + (K & 7) * 32 + lane] = v;
      if (warp == 0) y[32 * K + lane] = v;
      cur = cur + 1 == D ? 0 : cur + 1;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();  // y complete before the next pass reads it
  }
}

// m steps of textbook CG on A_p d = r from d = 0 (all threads). A_p in ELL
// with local columns; vectors in shared memory.
template <typename T, typename CT, int NT>
__device__ void cg_solve(const int32_t *lc, const T *lv, int K, int n, int npad, int m, CT *r,
                         CT *p, CT *q, CT *d, CT *red) {
  CT rr = CT(0);
  for (int i = threadIdx.x; i < npad; i += NT) {
    const CT v = i < n ? r[i] : CT(0);
    r[i] = v;
    p[i] = v;
    d[i] = CT(0);
    rr += v * v;
  }
  rr = block_sum<NT, CT>(rr, red);
  for (int it = 0; it < m && rr != CT(0); ++it) {
    CT pq = CT(0);
    for (int i = threadIdx.x; i < n; i += NT) {
      CT s = CT(0);
      for (int k = 0; k < K; ++k) s += to_ct(lv[(int64_t)k * npad + i]) * p[lc[(int64_t)k * npad + i]];
      q[i] = s;
      pq += p[i] * s;
    }
    pq = block_sum<NT, CT>(pq, red);
    const CT alpha = rr / pq;
    CT rn = CT(0);
    for (int i = threadIdx.x; i < n; i += NT) {
      d[i] += alpha * p[i];
      const CT ri = r[i] - alpha * q[i];
      r[i] = ri;
      rn += ri * ri;
    }
    rn = block_sum<NT, CT>(rn, red);
    const CT beta = rn / rr;
    rr = rn;
    for (int i = threadIdx.x; i < n; i += NT) p[i] = r[i] + beta * p[i];
    __syncthreads();
  }
}

// Two deterministic block sums with one barrier: callers alternate between
// two buffers of 2 NT/32 values (see block_sum_1b). The warp partials are
// stored as (a, b) pairs; after the barrier every warp reads them with one
// load (lane l takes pair l mod NT/32) and finishes with a butterfly over
// NT/32 lanes, so each thread does one shared load instead of NT/16, and
// every lane of every warp ends with the same bits (each butterfly level adds
// the same two values in both lanes of a pair).
template <int NT>
__device__ __forceinline__ void block_sum2f_1b(float &a, float &b, float *red) {
  constexpr int NW = NT / 32;
  static_assert(NW >= 1 && NW <= 32 && (NW & (NW - 1)) == 0, "power-of-two warp count");
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  float2 *red2 = reinterpret_cast<float2 *>(red);
  if ((threadIdx.x & 31) == 0) red2[threadIdx.x >> 5] = make_float2(a, b);
  __syncthreads();
  float2 v = red2[threadIdx.x & (NW - 1)];
#pragma unroll
  for (int o = NW / 2; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  a = v.x;
  b = v.y;
}

// m steps of CG on A_p d = r from d = 0 in the Chronopoulos-Gear
// arrangement (the same iterates as textbook CG in exact arithmetic, one
// synchronisation per step): with w = A r, gamma = (r, r), delta = (w, r),
//   p = r + beta p, s = w + beta s, d += alpha p, r -= alpha s,
//   w = A r, gamma' = (r, r), delta' = (w, r)   (one fused reduction),
//   beta' = gamma'/gamma, alpha' = gamma' / (delta' - beta' gamma'/alpha).
// A_p is staged in shared memory (FP32 values, the diagonal first in every
// row) in one of three forms: ELL with int16 local columns; PAIRED, the
// off-diagonal values and columns in pairs (one 64-bit and one 32-bit load
// per two entries); DIA, local rows on a grid box with row length bx and
// plane size bxy (grid3: a 3D box), one value array per local offset (the
// diagonal, then -bxy, -bx, -1, 1, bx, bxy; 2D without +-bxy) and no columns
// (entry e of row i multiplies r[i + offset e]; r has zero margins of
// kDiaMargin values on both sides, the front one cleared by the caller). r lives in shared memory (the operand of the products, read once
// per step per row and reused); p, s, d, w live in registers: thread t owns
// rows t, t + NT, ... On entry r holds the local residual (zero beyond n); on
// exit it holds d. KC > 0 is the ELL width known at compile time (KC = 0:
// runtime K). red holds 4 * NT/32 floats.
//
// RREG (diagonal-offset form): each thread also keeps r and the diagonal of
// its own rows in registers, so a step reads r from shared memory only at
// the neighbours (and stores it once): 9 instead of 12 shared accesses per
// row and step.
template <int NT, int RMAX, int KC, bool PAIRED, bool DIA = false, bool RREG = false>
__device__ void cg_solve_staged(const float *sval, const int16_t *scol, int K, int n, int npad,
                                int m, float *r, float *red, int bx = 0, int bxy = 0,
                                bool grid3 = false) {
  static_assert(!RREG || DIA, "own r in registers with the diagonal-offset form");
  static_assert(!PAIRED || (KC > 0 && KC % 2 == 1), "pairs need an odd compile-time width");
  static_assert(!DIA || (KC > 0 && !PAIRED), "the diagonal-offset form needs a compile-time width");
  const int tid = threadIdx.x;
  float *red0 = red, *red1 = red + 2 * (NT / 32);
  const float2 *vp = reinterpret_cast<const float2 *>(sval + npad);
  const uint32_t *cp = reinterpret_cast<const uint32_t *>(scol);
  float p[RMAX], s[RMAX], d[RMAX], w[RMAX], rr[RREG ? RMAX : 1], dg[RREG ? RMAX : 1];
  static_assert(!DIA || KC == 5 || KC == 7, "grid stencils have 5 or 7 entries");
  int off[DIA ? KC : 1];
  if constexpr (DIA) {
    if constexpr (KC == 5) {
      off[1] = -bx;
      off[2] = -1;
      off[3] = 1;
      off[4] = bx;
    } else {
      off[1] = grid3 ? -bxy : -bx;
      off[2] = grid3 ? -bx : -1;
      off[3] = grid3 ? -1 : 1;
      off[4] = grid3 ? 1 : bx;
      off[5] = grid3 ? bx : 0;
      off[6] = grid3 ? bxy : 0;
    }
    // the tail margin may hold a larger subdomain's values: clear it
    for (int i = npad + tid; i < npad + kDiaMargin; i += NT) r[i] = 0.f;
  }
  // w = A r and the two products of r
  auto product = [&](float &gam, float &del) {
    gam = 0.f;
    del = 0.f;
#pragma unroll
    for (int k = 0; k < RMAX; ++k) {
      const int i = tid + k * NT;
      float wi = 0.f;
      if (i < n) {
        const float ri = RREG ? rr[RREG ? k : 0] : r[i];
        wi = (RREG ? dg[RREG ? k : 0] : sval[i]) * ri;
        if constexpr (DIA) {
#pragma unroll
          for (int e = 1; e < KC; ++e) wi += sval[e * npad + i] * r[i + off[e]];
        } else if constexpr (PAIRED) {
#pragma unroll
          for (int q = 0; q < (KC - 1) / 2; ++q) {
            const float2 v = vp[q * npad + i];
            const uint32_t c = cp[q * npad + i];
            wi += v.x * r[c & 0xffffu];
            wi += v.y * r[c >> 16];
          }
        } else if constexpr (KC > 0) {
#pragma unroll
          for (int e = 1; e < KC; ++e) wi += sval[e * npad + i] * r[scol[e * npad + i]];
        } else {
          for (int e = 1; e < K; ++e) wi += sval[e * npad + i] * r[scol[e * npad + i]];
        }
        gam += ri * ri;
        del += wi * ri;
      }
      w[k] = wi;
    }
  };
#pragma unroll
  for (int k = 0; k < RMAX; ++k) {
    p[k] = 0.f;
    s[k] = 0.f;
    d[k] = 0.f;
  }
  __syncthreads();  // r complete, red buffers free
  if constexpr (RREG) {
#pragma unroll
    for (int k = 0; k < RMAX; ++k) {
      const int i = tid + k * NT;
      rr[k] = i < n ? r[i] : 0.f;
      dg[k] = i < n ? sval[i] : 0.f;
    }
  }
  float gam, del;
  product(gam, del);
  block_sum2f_1b<NT>(gam, del, red0);
  float alpha = gam != 0.f ? gam / del : 0.f, beta = 0.f;
  int buf = 1;
  for (int it = 0; it < m && gam != 0.f; ++it) {
#pragma unroll
    for (int k = 0; k < RMAX; ++k) {
      const int i = tid + k * NT;
      if (i < n) {
        const float ri = RREG ? rr[RREG ? k : 0] : r[i];
        p[k] = ri + beta * p[k];
        s[k] = w[k] + beta * s[k];
        d[k] += alpha * p[k];
        const float rn = ri - alpha * s[k];
        r[i] = rn;
        if constexpr (RREG) rr[k] = rn;
      }
    }
    __syncthreads();  // r complete before the product reads neighbours
    if (it + 1 == m) break;
    float g2, d2;
    product(g2, d2);
    block_sum2f_1b<NT>(g2, d2, buf ? red1 : red0);
    buf ^= 1;
    if (g2 == 0.f) break;
    beta = g2 / gam;
    alpha = g2 / (d2 - beta * g2 / alpha);
    gam = g2;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < RMAX; ++k) {
    const int i = tid + k * NT;
    if (i < npad) r[i] = i < n ? d[k] : 0.f;
  }
  __syncthreads();
}

// z = U^{-1} L^{-1} r with the ILU(0) factors, level by level.
// One triangular sweep of the ILU(0) solve: level rows e in
// [lptr[lv], lptr[lv+1]); the entries of level row e sit at index e
// (cc / vv[k*npad + e], column -1 = none), so a row's loads do not wait for
// its row number. BACK: U sweep (z[i] = (z[i] - sum) / d[e]), else L sweep
// (z[i] = r[i] - sum). With KE <= kIluHalf each thread's first rows of levels
// lv+1 and lv+2 are loaded into registers while level lv is computed, so the
// barriers between levels hide the load latency.
template <typename T, int NT, bool BACK>
struct IluRow {
  int i, c[kIluHalf];
  typename CTypeOf<T>::type v[kIluHalf], d;
  __device__ __forceinline__ void load(int e, int end, bool reg, const int32_t *__restrict__ lrow,
                                       const int32_t *__restrict__ cc, const T *__restrict__ vv,
                                       const T *__restrict__ dd, int KE, int npad) {
    using CT = typename CTypeOf<T>::type;
    i = -1;
    d = CT(1);
#pragma unroll
    for (int q = 0; q < kIluHalf; ++q) {
      c[q] = -1;
      v[q] = CT(0);
    }
    if (reg && e < end) {
      i = __ldg(lrow + e);
#pragma unroll
      for (int q = 0; q < kIluHalf; ++q)
        if (q < KE) {
          c[q] = __ldg(cc + (int64_t)q * npad + e);
          v[q] = to_ct(vv[(int64_t)q * npad + e]);
        }
      if (BACK) d = to_ct(dd[e]);
    }
  }
};

template <typename T, typename CT, int NT, bool BACK>
__device__ __forceinline__ void ilu_sweep(const int32_t *__restrict__ lptr, int nl,
                                          const int32_t *__restrict__ lrow,
                                          const int32_t *__restrict__ cc, const T *__restrict__ vv,
                                          const T *__restrict__ dd, int KE, int npad, const CT *r,
                                          CT *z) {
  constexpr int H = kIluHalf;
  if (nl <= 0) return;
  const int tid = threadIdx.x;
  const bool reg = KE <= H;
  // level bounds of lv, lv+1, lv+2: [a, b), [b, b2), [b2, b3)
  int a = __ldg(lptr), b = __ldg(lptr + 1);
  int b2 = nl > 1 ? __ldg(lptr + 2) : b;
  IluRow<T, NT, BACK> cur, nx1, nx2;
  cur.load(a + tid, b, reg, lrow, cc, vv, dd, KE, npad);
  nx1.load(b + tid, b2, reg, lrow, cc, vv, dd, KE, npad);
  for (int lv = 0; lv < nl; ++lv) {
    const int b3 = lv + 2 < nl ? __ldg(lptr + lv + 3) : b2;
    nx2.load(b2 + tid, b3, reg, lrow, cc, vv, dd, KE, npad);
    if (cur.i >= 0) {
      CT s = BACK ? z[cur.i] : r[cur.i];
#pragma unroll
      for (int q = 0; q < H; ++q)
        if (cur.c[q] >= 0) s -= cur.v[q] * z[cur.c[q]];
      z[cur.i] = BACK ? s / cur.d : s;
    }
    // rows beyond the first per thread (wide levels), or all rows when KE > H
    for (int e = a + tid + (reg ? NT : 0); e < b; e += NT) {
      const int i = __ldg(lrow + e);
      CT s = BACK ? z[i] : r[i];
      for (int q = 0; q < KE; ++q) {
        const int c = __ldg(cc + (int64_t)q * npad + e);
        if (c >= 0) s -= to_ct(vv[(int64_t)q * npad + e]) * z[c];
      }
      z[i] = BACK ? s / to_ct(dd[e]) : s;
    }
    __syncthreads();
    cur = nx1;
    nx1 = nx2;
    a = b;
    b = b2;
    b2 = b3;
  }
}

// z = U^{-1} L^{-1} r with the ILU(0) factors in level order.
template <typename T, typename CT, int NT>
__device__ __forceinline__ void ilu_apply(const SysDesc &S, const SubDesc &D, const int32_t *lptr_f,
                                          const int32_t *lrow_f, const int32_t *lptr_b,
                                          const int32_t *lrow_b, const CT *r, CT *z) {
  const int npad = D.npad, KL = S.ilu_kl, KU = S.ilu_ku;
  const int32_t *fc = S.ilu_fcol + D.row_off * KL;
  const T *fv = reinterpret_cast<const T *>(S.ilu_fval) + D.row_off * KL;
  const int32_t *bc = S.ilu_bcol + D.row_off * KU;
  const T *bv = reinterpret_cast<const T *>(S.ilu_bval) + D.row_off * KU;
  const T *bd = reinterpret_cast<const T *>(S.ilu_bdiag) + D.row_off;
  ilu_sweep<T, CT, NT, false>(lptr_f, D.nlev_f, lrow_f, fc, fv, bd, KL, npad, r, z);
  ilu_sweep<T, CT, NT, true>(lptr_b, D.nlev_b, lrow_b, bc, bv, bd, KU, npad, r, z);
}

// m steps of ILU(0)-preconditioned CG from d = 0 (all threads).
template <typename T, typename CT, int NT>
__device__ void pcg_solve(const SysDesc &S, const SubDesc &D, int m, CT *r, CT *z, CT *p, CT *q,
                          CT *d, CT *red) {
  const int K = S.K, n = D.n, npad = D.npad;
  const int32_t *lc = S.lcol + D.row_off * K;
  const T *lv = reinterpret_cast<const T *>(S.lval) + D.row_off * K;
  const int32_t *lptr_f = S.lev_ptr + D.lev_off;
  const int32_t *lptr_b = lptr_f + D.nlev_f + 1;
  const int32_t *lrow_f = S.lev_rows + D.lrow_off;
  const int32_t *lrow_b = lrow_f + n;
  for (int i = threadIdx.x; i < npad; i += NT) {
    if (i >= n) r[i] = CT(0);
    z[i] = CT(0);
    d[i] = CT(0);
  }
  __syncthreads();
  ilu_apply<T, CT, NT>(S, D, lptr_f, lrow_f, lptr_b, lrow_b, r, z);
  CT rz = CT(0);
  for (int i = threadIdx.x; i < npad; i += NT) {
    p[i] = z[i];
    rz += r[i] * z[i];
  }
  rz = block_sum<NT, CT>(rz, red);
  for (int it = 0; it < m && rz != CT(0); ++it) {
    CT pq = CT(0);
    for (int i = threadIdx.x; i < n; i += NT) {
      CT s = CT(0);
      for (int k = 0; k < K; ++k) s += to_ct(lv[(int64_t)k * npad + i]) * p[lc[(int64_t)k * npad + i]];
      q[i] = s;
      pq += p[i] * s;
    }
    pq = block_sum<NT, CT>(pq, red);
    const CT alpha = rz / pq;
    for (int i = threadIdx.x; i < n; i += NT) {
      d[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    __syncthreads();
    ilu_apply<T, CT, NT>(S, D, lptr_f, lrow_f, lptr_b, lrow_b, r, z);
    CT rn = CT(0);
    for (int i = threadIdx.x; i < n; i += NT) rn += r[i] * z[i];
    rn = block_sum<NT, CT>(rn, red);
    const CT beta = rn / rz;
    rz = rn;
    for (int i = threadIdx.x; i < n; i += NT) p[i] = z[i] + beta * p[i];
    __syncthreads();
  }
}

// GMRES work area in shared memory (after the four vectors): the Hessenberg
// matrix (column-major, kMaxGmres+1 rows), the Givens rotations, the
// least-squares right-hand side g, the projections / solution y, per-warp
// partial sums of the projections, and two ints.
template <typename CT, int NT>
struct GmresSmem {
  static constexpr int LDH = kMaxGmres + 1;
  static constexpr int H = 0, CS = H + LDH * kMaxGmres, SN = CS + kMaxGmres, G = SN + kMaxGmres,
                       Y = G + LDH, PART = Y + LDH, LEN = PART + (NT / 32) * LDH;
  static constexpr size_t bytes() { return (size_t)LEN * sizeof(CT) + 16; }
};

// m steps of GMRES on A_p d = r from d = 0, one cycle (Sec. 4.1 names GMRES
// as the iterative local solver for general systems; the method is Saad &
// Schultz's). Arnoldi builds the orthonormal basis V (global scratch, L2
// resident) and the Hessenberg matrix H; Givens rotations reduce H to upper
// triangular R while carrying ||r|| e_1 along as g; then R y = g and
// d = V_k y minimises ||r - A_p d|| over the Krylov space. Orthogonalisation
// is classical Gram-Schmidt applied twice: one block reduction of all j+1
// projections per pass instead of j+1 dependent ones, and with the second
// pass as accurate as modified Gram-Schmidt. At most n steps; an exact
// breakdown (h_{j+1,j} = 0) stops early with the exact solution. Thread t
// owns rows t, t+NT, ... of every vector, including its rows of V.
template <typename T, typename CT, int NT>
__device__ void gmres_solve(const int32_t *__restrict__ lc, const T *__restrict__ lv, int K, int n,
                            int npad, int m, CT *r, CT *w, CT *v, CT *d, CT *__restrict__ V,
                            CT *gs, CT *red) {
  using GS = GmresSmem<CT, NT>;
  constexpr int LDH = GS::LDH;
  CT *H = gs + GS::H, *cs = gs + GS::CS, *sn = gs + GS::SN, *g = gs + GS::G, *y = gs + GS::Y,
     *part = gs + GS::PART;
  int *flag = reinterpret_cast<int *>(gs + GS::LEN);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int mm = min(m, n);
  CT b2 = CT(0);
  for (int i = tid; i < npad; i += NT) {
    d[i] = CT(0);
    if (i < n) b2 += r[i] * r[i];
  }
  b2 = block_sum<NT, CT>(b2, red);  // same bit pattern in every thread
  const CT beta = sqrt(b2);
  if (!(beta > CT(0))) return;      // r = 0: d = 0
  for (int i = tid; i < npad; i += NT) {
    const CT x = i < n ? r[i] / beta : CT(0);
    v[i] = x;
    V[i] = x;
  }
  if (tid == 0) g[0] = beta;
  __syncthreads();
  int k = 0;
  for (int j = 0; j < mm; ++j) {
#pragma unroll 2
    for (int i = tid; i < n; i += NT) {  // w = A_p v_j
      CT s = CT(0);
      for (int e = 0; e < K; ++e) s += to_ct(lv[(int64_t)e * npad + i]) * v[lc[(int64_t)e * npad + i]];
      w[i] = s;
    }
    for (int pass = 0; pass < 2; ++pass) {
      // projections h_q = w . v_q (q <= j), four basis vectors per sweep over
      // the rows (independent load streams, rows unrolled so that the loads of
      // several rows are in flight together), all reduced together
      for (int q0 = 0; q0 <= j; q0 += 4) {
        const int nq = min(4, j + 1 - q0);
        const CT *__restrict__ vq = V + (int64_t)q0 * npad;
        CT s0 = CT(0), s1 = CT(0), s2 = CT(0), s3 = CT(0);
#pragma unroll 4
        for (int i = tid; i < n; i += NT) {
          const CT wi = w[i];
          s0 += wi * vq[i];
          if (nq > 1) s1 += wi * vq[npad + i];
          if (nq > 2) s2 += wi * vq[2 * (int64_t)npad + i];
          if (nq > 3) s3 += wi * vq[3 * (int64_t)npad + i];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          s0 += __shfl_xor_sync(0xffffffffu, s0, o);
          s1 += __shfl_xor_sync(0xffffffffu, s1, o);
          s2 += __shfl_xor_sync(0xffffffffu, s2, o);
          s3 += __shfl_xor_sync(0xffffffffu, s3, o);
        }
        if (lane == 0) {
          CT *pw = part + wid * LDH + q0;
          pw[0] = s0;
          if (nq > 1) pw[1] = s1;
          if (nq > 2) pw[2] = s2;
          if (nq > 3) pw[3] = s3;
        }
      }
      __syncthreads();
      for (int q = tid; q <= j; q += NT) {
        CT s = part[q];
        for (int u = 1; u < NT / 32; ++u) s += part[u * LDH + q];
        y[q] = s;
        H[q + j * LDH] = pass == 0 ? s : H[q + j * LDH] + s;
      }
      __syncthreads();
#pragma unroll 2
      for (int i = tid; i < n; i += NT) {  // w -= sum_q h_q v_q
        CT s = w[i];
        for (int q = 0; q <= j; ++q) s -= y[q] * V[(int64_t)q * npad + i];
        w[i] = s;
      }
      __syncthreads();  // y and part are rewritten by the next pass
    }
    CT h2 = CT(0);
    for (int i = tid; i < n; i += NT) h2 += w[i] * w[i];
    h2 = block_sum<NT, CT>(h2, red);
    const CT hn = sqrt(h2);
    if (tid == 0) {
      // earlier rotations on column j, then the one that zeroes h_{j+1,j}
      CT *hc = H + j * LDH;
      hc[j + 1] = hn;
      for (int q = 0; q < j; ++q) {
        const CT a = hc[q], b = hc[q + 1];
        hc[q] = cs[q] * a + sn[q] * b;
        hc[q + 1] = cs[q] * b - sn[q] * a;
      }
      const CT a = hc[j];
      const CT den = sqrt(a * a + hn * hn);
      int stop = 0;
      if (!(den > CT(0))) {
        stop = 2;  // singular on the Krylov space: keep the j steps so far
      } else {
        cs[j] = a / den;
        sn[j] = hn / den;
        hc[j] = den;
        hc[j + 1] = CT(0);
        g[j + 1] = -(sn[j] * g[j]);
        g[j] = cs[j] * g[j];
        if (!(hn > CT(0))) stop = 1;  // exact breakdown: the space is invariant
      }
      flag[0] = stop;
    }
    __syncthreads();
    const int stop = flag[0];
    if (stop == 2) break;
    k = j + 1;
    if (stop == 1 || k == mm) break;
    CT *__restrict__ vn = V + (int64_t)k * npad;
    for (int i = tid; i < n; i += NT) {
      const CT x = w[i] / hn;
      v[i] = x;
      vn[i] = x;
    }
    __syncthreads();
  }
  if (tid == 0) {  // R y = g, back substitution (k <= kMaxGmres)
    for (int q = k - 1; q >= 0; --q) {
      CT s = g[q];
      for (int t = q + 1; t < k; ++t) s -= H[q + t * LDH] * y[t];
      y[q] = s / H[q + q * LDH];
    }
  }
  __syncthreads();
#pragma unroll 2
  for (int i = tid; i < n; i += NT) {  // d = V_k y
    CT s = CT(0);
    for (int q = 0; q < k; ++q) s += y[q] * V[(int64_t)q * npad + i];
    d[i] = s;
  }
  __syncthreads();
}

// r_p = b[Omega_p] - A[Omega_p, :] x for the rows of one subdomain (thread t:
// rows t, t + NT, ...), written to rhs in the compute type; accumulates
// ||r||^2 over Omega_p and over its owned rows, and records for every owned
// row the x value used for its diagonal column (xg, used by the update).
// KC > 0: ELL width known at compile time; rows are then taken two at a time
// so that both rows' index / value loads, and then both rows' x loads, are in
// flight together (the gather is bound by memory latency, not bandwidth).
template <int KC, typename CT, int NT>
__device__ __forceinline__ void gather_rows(const SysDesc &S, const SubDesc &D, int K,
                                            const double *xcur, bool async, CT *rhs,
                                            double &a_loc, double &a_own) {
  const int64_t eb = D.row_off * K;
  if constexpr (KC > 0) {
    // the descriptors live in shared memory: keep what the loop needs in
    // registers (the stores below would otherwise force reloads)
    const int n = D.n, npad = D.npad;
    const int32_t *__restrict__ gidx = S.gidx + D.row_off;
    const uint8_t *__restrict__ ownf = S.ownf + D.row_off;
    const int32_t *__restrict__ rcol = S.rcol + eb;
    const double *__restrict__ rval = S.rval + eb;
    const double *__restrict__ bg = S.b;
    double *__restrict__ xg = S.xg + D.row_off;
    // R rows per thread and pass: the index loads of all R rows are issued
    // first, then x, b and the matrix values in one round of independent loads
    constexpr int R = 2;
    for (int i0 = threadIdx.x; i0 < npad; i0 += R * NT) {
      int cols[R][KC], g[R];
      bool live[R], own[R];
#pragma unroll
      for (int h = 0; h < R; ++h) {
        const int i = i0 + h * NT;
        live[h] = i < n;
        const int ii = live[h] ? i : 0;
        g[h] = gidx[ii];
        own[h] = live[h] && ownf[ii];  // no hole rows outside the grid layout
#pragma unroll
        for (int k = 0; k < KC; ++k) cols[h][k] = rcol[(int64_t)k * npad + ii];
      }
      double xs[R][KC], vs[R][KC], bb[R];
#pragma unroll
      for (int h = 0; h < R; ++h) {
        const int ii = live[h] ? i0 + h * NT : 0;
#pragma unroll
        for (int k = 0; k < KC; ++k) {
          xs[h][k] = async ? ld_relaxed_f64(xcur + cols[h][k]) : __ldcg(xcur + cols[h][k]);
          vs[h][k] = rval[(int64_t)k * npad + ii];
        }
        bb[h] = bg[g[h]];
      }
#pragma unroll
      for (int h = 0; h < R; ++h) {
        const int i = i0 + h * NT;
        if (i >= npad) continue;
        double r = 0.0;
        if (live[h]) {
          r = bb[h];
          double xd = 0.0;
#pragma unroll
          for (int k = 0; k < KC; ++k) {
            r -= vs[h][k] * xs[h][k];
            xd = cols[h][k] == g[h] ? xs[h][k] : xd;
          }
          if (own[h]) {
            xg[i] = xd;
            a_own += r * r;
          }
          if (async) a_loc += r * r;  // the local criterion (asynchronous only)
        }
        rhs[i] = rhs_from_f64<CT>(r);
      }
    }
  } else {
    for (int i = threadIdx.x; i < D.npad; i += NT) {
      double r = 0.0;
      if (i < D.n) {
        const int g = S.gidx[D.row_off + i];
        r = S.b[g];
        double xd = 0.0;
        for (int k = 0; k < K; ++k) {
          const int64_t e = eb + (int64_t)k * D.npad + i;
          const int c = S.rcol[e];
          const double xv = async ? ld_relaxed_f64(xcur + c) : __ldcg(xcur + c);
          r -= S.rval[e] * xv;
          xd = c == g ? xv : xd;
        }
        if (S.ownf[D.row_off + i]) {
          S.xg[D.row_off + i] = xd;
          a_own += r * r;
        }
        if (async) a_loc += r * r;  // the local criterion (asynchronous only)
      }
      rhs[i] = rhs_from_f64<CT>(r);
    }
  }
}

// The residual gather for local rows on a grid box (SysDesc::grid): local
// row i is box point x = i mod bx, y = (i / bx) mod (bxy / bx), z = i / bxy
// with global id g = g0 + x + y gs2 + z gs3, and rval holds the row's entries
// in slot order (the diagonal, then the global offsets -gs3, -gs2, -1, 1, gs2,
// gs3; 2D without +-gs3). No index is loaded: the loads of x (at g + offset,
// clamped into [0, n) where an entry is missing and its value zero), of the
// values, of b and of the row flag are all independent, so a row costs one
// memory round trip instead of two. Same results as gather_rows up to the
// order of the row's terms.
template <int KC, typename CT, int NT>
__device__ __forceinline__ void gather_rows_grid(const SysDesc &S, const SubDesc &D,
                                                 const double *xcur, bool async, CT *rhs,
                                                 double &a_loc, double &a_own) {
  static_assert(KC == 5 || KC == 7, "grid stencils have 5 or 7 entries");
  const int n = D.n, npad = D.npad;
  const uint8_t *__restrict__ ownf = S.ownf + D.row_off;
  const double *__restrict__ rval = S.rval + D.row_off * KC;
  const double *__restrict__ bg = S.b;
  double *__restrict__ xg = S.xg + D.row_off;
  const int bx = D.bx, by = D.bxy / D.bx, g0 = D.g0, s2 = S.gs2, s3 = S.gs3, nmax = S.n - 1;
  const bool g3 = S.grid == 3;
  int goff[KC];
  goff[0] = 0;
  if constexpr (KC == 5) {
    goff[1] = -s2;
    goff[2] = -1;
    goff[3] = 1;
    goff[4] = s2;
  } else {
    goff[1] = g3 ? -s3 : -s2;
    goff[2] = g3 ? -s2 : -1;
    goff[3] = g3 ? -1 : 1;
    goff[4] = g3 ? 1 : s2;
    goff[5] = g3 ? s2 : 0;
    goff[6] = g3 ? s3 : 0;
  }
  constexpr int R = 2;
  for (int i0 = threadIdx.x; i0 < npad; i0 += R * NT) {
    double xs[R][KC], vs[R][KC], bb[R];
    uint8_t f[R];
#pragma unroll
    for (int h = 0; h < R; ++h) {
      const int i = i0 + h * NT;
      const int ii = i < n ? i : 0;
      const int q = ii / bx, z = q / by;
      const int g = min(g0 + (ii - q * bx) + (q - z * by) * s2 + z * s3, nmax);
      f[h] = ownf[ii];
      bb[h] = bg[g];
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        const int c = min(max(g + goff[k], 0), nmax);
        xs[h][k] = async ? ld_relaxed_f64(xcur + c) : __ldcg(xcur + c);
        vs[h][k] = rval[(int64_t)k * npad + ii];
      }
    }
#pragma unroll
    for (int h = 0; h < R; ++h) {
      const int i = i0 + h * NT;
      if (i >= npad) continue;
      double r = 0.0;
      if (i < n && f[h] != 2) {
        r = bb[h];
#pragma unroll
        for (int k = 0; k < KC; ++k) r -= vs[h][k] * xs[h][k];
        if (f[h] == 1) {
          xg[i] = xs[h][0];
          a_own += r * r;
        }
        if (async) a_loc += r * r;  // the local criterion (asynchronous only)
      }
      rhs[i] = rhs_from_f64<CT>(r);
    }
  }
}

// --------------------------------------------------------------------------
// the persistent RAS kernel
// --------------------------------------------------------------------------


template <int KIND, typename T, int NT>
struct Smem {
  using CT = typename CTypeOf<T>::type;
  // band: copy rings | y | partials | window rings ; cg: r p q d ; ilu: r z p q d ;
  // staged cg: A_p values | A_p columns | p ; gmres: r w v d | GmresSmem
  static __host__ __device__ int band_twm(int Wmax) { return band_cols_per_warp(Wmax, NT / 32); }
  static __host__ __device__ size_t ylen(int Wmax, int npad_max) {
    return ((size_t)npad_max + 31) / 32 * 32;
  }
  static __host__ __device__ size_t vec_len(int npad_max) { return ((size_t)npad_max + 31) / 32 * 32; }
  static __host__ __device__ size_t bytes(int Wmax, int npad_max, int kmax, int nstages) {
    if (KIND == kBand) {
      size_t b = (size_t)(NT / 32) * nstages * band_twm(Wmax) * 32 * sizeof(T);  // copy rings
      b += ylen(Wmax, npad_max) * sizeof(CT);     // y (r / delta)
      b += 2 * NT * sizeof(CT);                   // partials, two buffers
      b += (size_t)(NT / 32) * 512 * sizeof(CT);  // per-warp window rings (two copies)
      return b;
    }
    if (KIND == kCGS) {
      // values (FP32) | columns (int16) | margin | p | margin ; K <= kmax <= kMaxEll
      const size_t vl = vec_len(npad_max);
      return (size_t)kmax * vl * 6 + (vl + 2 * kDiaMargin) * 4;
    }
    if (KIND == kGMRES) return 4 * vec_len(npad_max) * sizeof(CT) + GmresSmem<CT, NT>::bytes();
    const int nv = KIND == kCG ? 4 : 5;
    return nv * vec_len(npad_max) * sizeof(CT);
  }
};

// Resident CTAs per SM the register allocation is sized for: the 512-thread
// variants (staged CG: ~175 KB of shared memory) run one CTA per SM, the
// 256-thread variants two.
template <int NT> struct MinBlocks { static constexpr int value = NT >= 512 ? 1 : 2; };

template <int KIND, typename T, int NT>
__global__ void __launch_bounds__(NT, MinBlocks<NT>::value) ras_main_kernel(Launch L) {
  using CT = typename CTypeOf<T>::type;
  using SM = Smem<KIND, T, NT>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ SysDesc s_sys;
  __shared__ SubDesc s_sub;
  __shared__ double s_red[NT / 32 * 2];
  __shared__ __align__(16) CT s_redc[4 * (NT / 32)];
  __shared__ int s_flag[8];
  __shared__ int s_dyn[2];
  __shared__ uint32_t s_seq[32];  // async: neighbours' sequence values seen before the gather
  __shared__ __align__(8) uint64_t s_mbar[1];
  __shared__ int s_done[kMaxCtaSys];
  __shared__ int64_t s_iter0[kMaxCtaSys];

  const int tid = threadIdx.x;
  const int c = blockIdx.x;
  // static schedule: this CTA's items [i0, i1) and systems [cs0, cs1); the
  // dynamic schedules (more CTAs than the static plan) use neither
  const bool dyn = L.dynamic != 0;
  const int i0 = dyn ? 0 : L.cta_off[c], i1 = dyn ? 0 : L.cta_off[c + 1];
  const int cs0 = dyn ? 0 : L.cta_sys_off[c], cs1 = dyn ? 0 : L.cta_sys_off[c + 1];
  const int nls = dyn ? L.nsys : cs1 - cs0;  // systems this CTA decides for (sync)

  // shared-memory carve-up
  T *ring = nullptr;
  CT *ybuf = nullptr, *pbuf = nullptr, *v0 = nullptr, *v1 = nullptr, *v2 = nullptr, *v3 = nullptr,
     *v4 = nullptr, *wbuf = nullptr, *gsm = nullptr;
  const int twm = SM::band_twm(L.Wmax);
  if (KIND == kBand) {
    ring = reinterpret_cast<T *>(smem);
    ybuf = reinterpret_cast<CT *>(smem + (size_t)(NT / 32) * L.nstages * twm * 32 * sizeof(T));
    pbuf = ybuf + SM::ylen(L.Wmax, L.npad_max);
    wbuf = pbuf + 2 * NT;
  } else if (KIND == kCGS) {
    const size_t vl = SM::vec_len(L.npad_max);
    v0 = reinterpret_cast<CT *>(smem + (size_t)L.kmax * vl * 6) + kDiaMargin;  // p
  } else {
    const size_t vl = SM::vec_len(L.npad_max);
    CT *base = reinterpret_cast<CT *>(smem);
    v0 = base;
    v1 = base + vl;
    v2 = base + 2 * vl;
    v3 = base + 3 * vl;
    v4 = KIND == kILU ? base + 4 * vl : nullptr;
    if (KIND == kGMRES) gsm = base + 4 * vl;
  }
  uint32_t gcount = 0;
  if (KIND == kCGS) {
    // the front margin of p stays zero for the whole launch (the diagonal-
    // offset products read it for rows without an entry at that offset)
    for (int i = tid; i < kDiaMargin; i += NT) v0[i - kDiaMargin] = CT(0);
    if (tid == 0) {
      mbar_init(&s_mbar[0], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  if (tid == 0) s_flag[7] = -1;  // no system descriptor loaded yet
  for (int k = tid; k < nls; k += NT) {
    const int sys = dyn ? k : L.cta_sys[2 * (cs0 + k)];
    s_done[k] = L.sys[sys].st->done;  // systems finished in an earlier launch stay finished
    s_iter0[k] = L.sys[sys].st->iters;
  }
  __syncthreads();

  const bool async = L.mode != kSync;
  const bool decentral = L.mode == kAsyncDecentral;
  // wall-clock limit of the whole solve (each CTA measures from its own start)
  const uint64_t t_start = gtimer();
  auto past_deadline = [&]() -> bool {
    return (int64_t)(gtimer() - t_start) > L.solve_limit_ns;
  };

  // ---- one local update of subdomain `it`: gather, solve, restricted update
  // returns false on a device-side error (abort raised)
  auto update = [&](double *xcur, double *xnext, double &res_loc, double &res_own) -> bool {
    const SysDesc &S = s_sys;
    const SubDesc &D = s_sub;
    const int K = S.K;
    CT *rhs = KIND == kBand ? ybuf : v0;
    uint64_t t0 = 0, t1 = 0, t2 = 0;
    if (tid == 0) t0 = gtimer();
    if (KIND == kCGS && tid == 0) {
      // stage A_p (values, columns) while the residual is gathered
      const size_t vl = SM::vec_len(L.npad_max);
      const bool pr = S.vpair != nullptr, dia = S.vdia != nullptr;
      const uint32_t bv = (uint32_t)((size_t)K * D.npad * 4);
      const uint32_t bc = dia ? 0u : (uint32_t)((size_t)(pr ? K - 1 : K) * D.npad * 2);
      fence_proxy_async();
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&s_mbar[0])),
                   "r"(bv + bc)
                   : "memory");
      if (dia) {
        bulk_copy_nobar_arrive(smem, S.vdia + D.row_off * K, bv, &s_mbar[0]);
      } else if (pr) {
        bulk_copy_nobar_arrive(smem, S.vpair + D.row_off * K, bv, &s_mbar[0]);
        bulk_copy_nobar_arrive(smem + (size_t)L.kmax * vl * 4, S.cpair + D.row_off * K / 2, bc, &s_mbar[0]);
      } else {
        bulk_copy_nobar_arrive(smem, reinterpret_cast<const float *>(S.lval) + D.row_off * K, bv, &s_mbar[0]);
        bulk_copy_nobar_arrive(smem + (size_t)L.kmax * vl * 4, S.lcol16 + D.row_off * K, bc, &s_mbar[0]);
      }
    }
    double a_loc = 0.0, a_own = 0.0;
    for (int attempt = 0;; ++attempt) {
      a_loc = 0.0;
      a_own = 0.0;
      if (S.grid && K == 5) gather_rows_grid<5, CT, NT>(S, D, xcur, async, rhs, a_loc, a_own);
      else if (S.grid && K == 7) gather_rows_grid<7, CT, NT>(S, D, xcur, async, rhs, a_loc, a_own);
      else if (K == 5) gather_rows<5, CT, NT>(S, D, K, xcur, async, rhs, a_loc, a_own);
      else if (K == 7) gather_rows<7, CT, NT>(S, D, K, xcur, async, rhs, a_loc, a_own);
      else gather_rows<0, CT, NT>(S, D, K, xcur, async, rhs, a_loc, a_own);
      block_sum2<NT>(a_loc, a_own, s_red);
      // asynchronous mode: a gather that overlapped a neighbour's write of its
      // owned rows (its sequence value was odd, or moved) saw a mix of that
      // neighbour's old and new values; it is redone, at most twice
      if (!async || !L.consistent || attempt == 2 || D.n_nbr == 0 || D.n_nbr > 32) break;
      __threadfence();  // this thread's reads of x before the re-read below
      __syncthreads();
      if (tid < 32) {
        bool torn = false;
        if (tid < D.n_nbr) {
          const uint32_t now = ld_acquire_u32(&S.sub[S.nbr[D.nbr_off + tid]].version);
          torn = (s_seq[tid] & 1u) || now != s_seq[tid];
          s_seq[tid] = now;
        }
        torn = __any_sync(0xffffffffu, torn);
        if (tid == 0) s_flag[3] = torn ? 1 : 0;
      }
      __syncthreads();
      if (!s_flag[3]) break;
    }
    res_loc = a_loc;
    res_own = a_own;
    if (tid == 0) t1 = gtimer();
    // local solve
    CT *delta = rhs;
    if (KIND == kBand) {
      __syncthreads();
      const T *fac = reinterpret_cast<const T *>(S.fac);
      const int64_t rec = (int64_t)32 * (D.W + 32);
      const int nb = D.npad / 32;
      const T *F = fac + D.fac_off;
      if (L.nstages >= 6)
        band_solve_chain<T, CT, NT, 6>(F, F + nb * rec, nb, D.W, twm, ybuf, pbuf, wbuf, ring);
      else
        band_solve_chain<T, CT, NT, 4>(F, F + nb * rec, nb, D.W, twm, ybuf, pbuf, wbuf, ring);
    } else if (KIND == kCGS) {
      if (tid == 0) {
        const bool ok = mbar_wait(&s_mbar[0], gcount & 1u, L.timeout_ns);
        if (!ok) {
          set_error(L.ctl, kETIMEOUT, 5);
          mbar_wait(&s_mbar[0], gcount & 1u, L.timeout_ns);  // bounded drain of the copy
        }
        s_flag[4] = ok ? 1 : 0;
      }
      ++gcount;
      __syncthreads();
      if (!s_flag[4]) return false;
      const size_t vl = SM::vec_len(L.npad_max);
      const float *sv = reinterpret_cast<const float *>(smem);
      const int16_t *sc = reinterpret_cast<const int16_t *>(smem + (size_t)L.kmax * vl * 4);
      float *pv = reinterpret_cast<float *>(v0);
      float *rd = reinterpret_cast<float *>(s_redc);
      constexpr int RM = (kStagedRows + NT - 1) / NT;
      // subdomains of up to kRegRows rows per thread keep their r in registers
      constexpr int RR = RM < kRegRows ? RM : kRegRows;
      if (S.vdia && K == 5 && D.n <= RR * NT)
        cg_solve_staged<NT, RR, 5, false, true, true>(sv, sc, K, D.n, D.npad, L.m, pv, rd, D.bx,
                                                      D.bxy);
      else if (S.vdia && K == 5)
        cg_solve_staged<NT, RM, 5, false, true>(sv, sc, K, D.n, D.npad, L.m, pv, rd, D.bx, D.bxy);
      else if (S.vdia && K == 7)
        cg_solve_staged<NT, RM, 7, false, true>(sv, sc, K, D.n, D.npad, L.m, pv, rd, D.bx, D.bxy,
                                                S.grid == 3);
      else if (S.vpair && K == 5) cg_solve_staged<NT, RM, 5, true>(sv, sc, K, D.n, D.npad, L.m, pv, rd);
      else if (S.vpair && K == 7) cg_solve_staged<NT, RM, 7, true>(sv, sc, K, D.n, D.npad, L.m, pv, rd);
      else if (S.vpair && K == 3) cg_solve_staged<NT, RM, 3, true>(sv, sc, K, D.n, D.npad, L.m, pv, rd);
      else if (K == 5) cg_solve_staged<NT, RM, 5, false>(sv, sc, K, D.n, D.npad, L.m, pv, rd);
      else if (K == 7) cg_solve_staged<NT, RM, 7, false>(sv, sc, K, D.n, D.npad, L.m, pv, rd);
      else cg_solve_staged<NT, RM, 0, false>(sv, sc, K, D.n, D.npad, L.m, pv, rd);
      delta = v0;
    } else if (KIND == kCG) {
      const int32_t *lc = S.lcol + D.row_off * K;
      const T *lv = reinterpret_cast<const T *>(S.lval) + D.row_off * K;
      __syncthreads();
      cg_solve<T, CT, NT>(lc, lv, K, D.n, D.npad, L.m, v0, v1, v2, v3, s_redc);
      delta = v3;
    } else if (KIND == kGMRES) {
      const int32_t *lc = S.lcol + D.row_off * K;
      const T *lv = reinterpret_cast<const T *>(S.lval) + D.row_off * K;
      CT *V = reinterpret_cast<CT *>(S.kry) + D.row_off * S.kry_ld;
      __syncthreads();
      gmres_solve<T, CT, NT>(lc, lv, K, D.n, D.npad, min(L.m, S.kry_ld - 1), v0, v1, v2, v3, V, gsm,
                             s_redc);
      delta = v3;
    } else {
      __syncthreads();
      pcg_solve<T, CT, NT>(S, D, L.m, v0, v1, v2, v3, v4, s_redc);
      delta = v4;
    }
    if (tid == 0) t2 = gtimer();
    if (async && L.consistent) {
      // sequence value odd while the owned rows change
      if (tid == 0) {
        SubState &me = S.sub[s_flag[5]];
        st_relaxed_u32(&me.version, (uint32_t)(2 * me.updates + 1));
        __threadfence();
      }
      __syncthreads();
    }
    // restricted prolongation: only owned rows are written (RAS). x_g + delta
    // on an owned row is the owned part of the local solution computed from
    // the very values this gather read, whatever other subdomains (or delays)
    // did to x meanwhile. Four rows per thread and pass, loads first.
    {
      const int32_t *__restrict__ own = S.own_l + D.own_off;
      const int32_t *__restrict__ owng = S.own_g + D.own_off;
      const double *__restrict__ xgl = S.xg + D.row_off;
      const int no = D.n_own;
      constexpr int U = 4;
      for (int t0 = tid; t0 < no; t0 += U * NT) {
        int li[U], gg[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int t = t0 + u * NT;
          li[u] = t < no ? own[t] : 0;
          gg[u] = t < no ? owng[t] : 0;
        }
        double xn[U];
#pragma unroll
        for (int u = 0; u < U; ++u) xn[u] = xgl[li[u]] + (double)delta[li[u]];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (t0 + u * NT < no) {
            if (async) st_relaxed_f64(xnext + gg[u], xn[u]);
            else __stcg(xnext + gg[u], xn[u]);
          }
        }
      }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      // atomics: on the dynamic schedules a subdomain's updates run on
      // different CTAs
      SubState &ph = S.sub[s_flag[5]];
      atomicAdd(reinterpret_cast<unsigned long long *>(&ph.t_gather), t1 - t0);
      atomicAdd(reinterpret_cast<unsigned long long *>(&ph.t_solve), t2 - t1);
      atomicAdd(reinterpret_cast<unsigned long long *>(&ph.t_update), gtimer() - t2);
    }
    return true;
  };

  auto load_item = [&](int it) {
    __syncthreads();  // everyone is done with the previous item's shared state
    if (tid == 0) {
      const Item item = L.items[it];
      if (item.sys != s_flag[7]) {  // the system descriptor is constant in a launch
        s_sys = L.sys[item.sys];
        s_flag[7] = item.sys;
      }
      s_sub = s_sys.subs[item.p];
      s_flag[5] = item.p;
      s_flag[6] = item.ls;
    }
    __syncthreads();
  };

  if (!async) {
    // ------------------------------------------------------------ SYNC
    int fin = 0;
    for (int64_t j = 0; j < L.step_limit; ++j) {
      // one synchronous iteration: the static schedule runs this CTA's items;
      // the dynamic one takes items by ticket until the iteration's items are
      // gone (the counter is reset by the last CTA at the grid barrier), so
      // uneven subdomains and item counts that do not divide by the CTAs
      // still keep every CTA busy; either way every item is updated once
      // from x^j, so the iterates are the same bits
      for (int k = i0;; ++k) {
        int it = k;
        if (dyn) {
          if (tid == 0) {
            const unsigned long long t = atomicAdd(&L.ctl->ticket, 1ull);
            s_dyn[1] = t < (unsigned long long)L.nitems ? (int)t : -1;
          }
          __syncthreads();
          it = s_dyn[1];
          if (it < 0) break;
        } else if (k >= i1) {
          break;
        }
        load_item(it);
        if (s_done[dyn ? s_flag[7] : s_flag[6]]) continue;
        const int p = s_flag[5];
        double *xc = (j & 1) ? s_sys.xalt : s_sys.x;
        double *xn = (j & 1) ? s_sys.x : s_sys.xalt;
        double rl, ro;
        if (!update(xc, xn, rl, ro)) goto out;
        if (tid == 0) {
          SubState &ss = s_sys.sub[p];
          ss.part[j & 1] = ro;
          atomicAdd(reinterpret_cast<unsigned long long *>(&ss.updates), 1ull);
        }
      }
      if (tid == 0 && past_deadline()) set_error(L.ctl, kETIMEOUT, 4);
      if (!grid_barrier(L.ctl, fin, L.timeout_ns, s_flag)) goto out;
      fin = 0;
      if (s_flag[1] <= 0) break;  // every system decided before this barrier
      // decisions for iteration j (residual of x^j)
      for (int k = 0; k < nls; ++k) {
        if (s_done[k]) continue;
        // every CTA takes the same decision from the same bits; one (the
        // lead) writes the system's state
        const int sys = dyn ? k : L.cta_sys[2 * (cs0 + k)];
        const int lead = dyn ? (blockIdx.x == 0 ? 1 : 0) : L.cta_sys[2 * (cs0 + k) + 1];
        if (tid < 32) {
          const SysDesc &S = L.sys[sys];
          const double res2 = warp_sum_partials(S.sub, S.P, (int)(j & 1), true);
          if (tid == 0) {
            const int64_t kk = s_iter0[k] + j;
            const bool conv = res2 < S.tol2 * S.st->b2 || res2 == 0.0;
            int done = 0;
            if (conv) {
              done = 1;
              if (lead) {
                S.st->iters = kk;
                S.st->res2 = res2;
                S.st->status = kOK;
                S.st->result_alt = (int)(j & 1);
                S.st->done = 1;
              }
            } else if (kk + 1 >= L.max_updates || j + 1 == L.step_limit) {
              if (kk + 1 >= L.max_updates) done = 1;
              if (lead) {
                S.st->iters = kk + 1;
                S.st->res2 = res2;
                S.st->status = done ? kENOCONV : kOK;
                S.st->result_alt = (int)((j + 1) & 1);
                S.st->done = done;
              }
            }
            if (done) {
              s_done[k] = 1;
              if (lead) fin++;
            }
          }
        }
      }
      __syncthreads();
    }
  } else {
    // ----------------------------------------------------------- ASYNC
    // One visit of item `it`: decide and perform its next action (update,
    // park, post-termination check). Returns -1 on abort, 0 when the item had
    // nothing to do, 1 after doing something; not_done is set while the
    // item's system has not finished.
    auto async_item = [&](int it, int &not_done) -> int {
      load_item(it);
      const int p = s_flag[5];
      SubState &ss = s_sys.sub[p];
      SysState *st = s_sys.st;
      if (tid == 0) {
        const uint32_t wd = ld_acquire_u32(&st->word);
        int action = 0;  // 0 none, 1 update, 2 park, 3 check
        const int phase = (int)(wd & 3u);
        const int epoch = (int)(wd >> 2);
        if (ld_relaxed_s32(&L.ctl->abort)) action = -1;
        else if (phase != kDone) {
          s_flag[3] = 0;
          if (phase == kRun) {
            // decentralized detection: the global flag, raised here or seen
            // on a neighbour, stops this subdomain (it parks)
            bool flag = false;
            if (decentral) {
              flag = ld_relaxed_s32(&ss.gconv_epoch) == epoch;
              if (!flag) {
                const int32_t *nb = s_sys.nbr + s_sub.nbr_off;
                for (int q = 0; q < s_sub.n_nbr && !flag; ++q)
                  flag = ld_acquire_s32(&s_sys.sub[nb[q]].gconv_epoch) == epoch;
                if (flag) st_release_s32(&ss.gconv_epoch, epoch);
              }
            }
            if (flag) {
              if (ss.park_epoch != epoch) action = 2;
            } else if (ss.updates >= L.max_updates) {
              st->status = kENOCONV;
              if (atomicCAS(&st->word, wd, ((uint32_t)epoch << 2) | kDone) == wd)
                atomicSub(&L.ctl->remaining, 1);
            } else if (ss.step_updates < L.step_limit) {
              action = 1;
              if (L.fresh && ss.updates > 0 && s_sub.n_nbr > 0) {
                // wait for new neighbour data instead of repeating the solve
                // on the same interface values
                uint64_t seen = 0;
                const int32_t *nb = s_sys.nbr + s_sub.nbr_off;
                for (int q = 0; q < s_sub.n_nbr; ++q)
                  seen += ld_relaxed_u32(&s_sys.sub[nb[q]].version);
                if (seen == ss.nbr_seen) action = 0;
              }
            }
          } else if (phase == kDrain) {
            if (ss.park_epoch != epoch) action = 2;
          } else {
            if (ss.check_epoch != epoch) action = 3;
          }
        }
        s_flag[0] = action;
        s_flag[1] = (int)wd;
        s_flag[2] = (phase != kDone) ? 1 : 0;
      }
      __syncthreads();
      const int action = s_flag[0];
      const uint32_t wd = (uint32_t)s_flag[1];
      if (action < 0) return -1;
      if (s_flag[2]) not_done = 1;
      if (action == 0) return 0;
      const int epoch = (int)(wd >> 2);
      if (action == 1) {
        // acquire the neighbours' published versions before reading x: the
        // lanes of warp 0 take one neighbour each, so the acquires are in
        // flight together; the barrier then orders every thread's reads of
        // x after them
        if (tid < 32) {
          uint64_t seen = 0;
          const int32_t *nb = s_sys.nbr + s_sub.nbr_off;
          for (int q = tid; q < s_sub.n_nbr; q += 32) {
            const uint32_t v = ld_acquire_u32(&s_sys.sub[nb[q]].version);
            seen += v;
            if (q < 32) s_seq[q] = v;
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) seen += __shfl_xor_sync(0xffffffffu, seen, o);
          if (tid == 0) {
            if (ss.updates > 0 && seen == ss.nbr_seen) ss.stale += 1;
            ss.nbr_seen = seen;
          }
        }
        __syncthreads();
        double rl, ro;
        if (!update(s_sys.x, s_sys.x, rl, ro)) return -1;
        if (tid == 0) {
          // every thread fenced its owned-row stores before update()'s
          // final barrier; the release store publishes them
          ss.updates += 1;
          ss.step_updates += 1;
          st_release_u32(&ss.version, (uint32_t)(2 * ss.updates));
          // local criterion (Eq. 2) on the residual gathered before the update
          const bool conv = rl < s_sys.tol2 * ss.bloc2 || rl == 0.0;
          if (decentral) {
            // leader election on a spanning tree of the subdomain graph: a
            // locally converged subdomain that has received the convergence
            // report of all its tree neighbours but one sends its own report
            // to that one; one that has received all of them is a leader and
            // raises the global flag, which then floods to every subdomain.
            // A subdomain that loses local convergence withdraws the report
            // it sent. Reports are tagged with the epoch, so a restart voids
            // them.
            const int32_t *tn = s_sys.tnbr + s_sub.tnbr_off;
            const int nt = s_sub.n_tnbr;
            const int p = s_flag[5];
            int got = 0, missing = -1;
            for (int q = 0; q < nt; ++q) {
              const unsigned long long r = ld_acquire_u64(&s_sys.sub[tn[q]].report);
              if ((int)(r >> 32) == epoch && (int)(uint32_t)r == p) ++got;
              else missing = tn[q];
            }
            const unsigned long long mine = ld_relaxed_u64(&ss.report);
            const bool sent = (int)(mine >> 32) == epoch;
            if (conv) {
              if (got == nt) {
                st_release_s32(&ss.gconv_epoch, epoch);
              } else if (got == nt - 1 && !sent) {
                st_release_u64(&ss.report,
                               ((unsigned long long)(uint32_t)epoch << 32) | (uint32_t)missing);
              }
            } else if (sent) {
              st_release_u64(&ss.report, 0xffffffff00000000ull);
            }
          } else if (conv && ss.conv_epoch != epoch) {
            ss.conv_epoch = epoch;
            const int nc = atomicAdd(&st->nconv, 1) + 1;
            if (nc == s_sys.P) atomicCAS(&st->word, ((uint32_t)epoch << 2) | kRun,
                                         ((uint32_t)epoch << 2) | kDrain);
          } else if (!conv && ss.conv_epoch == epoch) {
            ss.conv_epoch = -1;
            atomicSub(&st->nconv, 1);
          }
        }
      } else if (action == 2) {
        if (tid == 0) {
          ss.park_epoch = epoch;
          __threadfence();
          const int np = atomicAdd(&st->nparked, 1) + 1;
          if (np == s_sys.P) {
            __threadfence();
            st_release_u32(&st->word, ((uint32_t)epoch << 2) | kCheck);
          }
        }
      } else {
        // post-termination check: owned residual of the (now frozen) x
        const SysDesc &S = s_sys;
        const SubDesc &D = s_sub;
        const int K = S.K;
        const int64_t eb = D.row_off * K;
        double o = 0.0, dmy = 0.0;
        for (int i = tid; i < D.n; i += NT) {
          if (S.ownf[D.row_off + i] != 1) continue;
          double r = S.b[S.gidx[D.row_off + i]];
          for (int k = 0; k < K; ++k) {
            const int64_t e = eb + (int64_t)k * D.npad + i;
            r -= S.rval[e] * ld_relaxed_f64(S.x + S.rcol[e]);
          }
          o += r * r;
        }
        block_sum2<NT>(o, dmy, s_red);
        if (tid < 32) {
          int last = 0;
          if (tid == 0) {
            st_relaxed_f64(&ss.part[0], o);
            ss.check_epoch = epoch;
            __threadfence();
            last = (atomicAdd(&st->nchecked, 1) + 1 == S.P) ? 1 : 0;
            if (last) __threadfence();
          }
          last = __shfl_sync(0xffffffffu, last, 0);
          if (last) {
            const double res2 = warp_sum_partials(S.sub, S.P, 0, true);
            if (tid == 0) {
              st->res2 = res2;
              uint32_t nw;
              if (res2 < S.tol2 * st->b2 || res2 == 0.0) {
                st->status = kOK;
                nw = ((uint32_t)epoch << 2) | kDone;
              } else if (ld_relaxed_s32(&st->restarts) >= L.max_restarts) {
                st->status = kENOCONV;
                nw = ((uint32_t)epoch << 2) | kDone;
              } else {
                st->restarts += 1;
                st->nconv = 0;
                st->nparked = 0;
                st->nchecked = 0;
                nw = ((uint32_t)(epoch + 1) << 2) | kRun;
              }
              __threadfence();
              st_release_u32(&st->word, nw);
              if ((nw & 3u) == (uint32_t)kDone) atomicSub(&L.ctl->remaining, 1);
            }
          }
        }
        __syncthreads();
      }
      return 1;
    };
    if (!dyn) {
      // static schedule: this CTA's own subdomains, in turn. The per-launch
      // update budget starts from zero
      if (tid == 0)
        for (int it = i0; it < i1; ++it) {
          const Item item = L.items[it];
          L.sys[item.sys].sub[item.p].step_updates = 0;
        }
      __syncthreads();
      uint64_t t_idle = gtimer();
      for (;;) {
        int any_work = 0, all_done = 1;
        for (int it = i0; it < i1; ++it) {
          int not_done = 0;
          const int r = async_item(it, not_done);
          if (r < 0) goto out;
          if (not_done) all_done = 0;
          if (r > 0) any_work = 1;
        }
        if (all_done) break;
        if (tid == 0 && past_deadline()) set_error(L.ctl, kETIMEOUT, 4);
        if (any_work) {
          t_idle = gtimer();
        } else {
          if (!L.persist) break;
          // thread 0 decides, so that every thread leaves together
          if (tid == 0) s_dyn[0] = (int64_t)(gtimer() - t_idle) > L.timeout_ns ? 1 : 0;
          __syncthreads();
          if (s_dyn[0]) {
            if (tid == 0) set_error(L.ctl, kETIMEOUT, 3);
            break;
          }
          __nanosleep(500);
        }
      }
    } else {
      // dynamic schedule (one persistent launch over every SM): CTAs take
      // tickets t = 0, 1, 2, ... from one counter and visit item t mod
      // nitems, so every subdomain is visited once per round of tickets
      // whichever CTA is free (equal update rates without equal subdomain
      // counts per CTA). A per-subdomain lock taken with an acquire CAS and
      // released with a release store gives one CTA at a time the
      // subdomain's state; a ticket whose subdomain is busy is skipped.
      // CTAs stop when every system of the launch has finished.
      uint64_t t_idle = gtimer();  // thread 0's: last time a ticket found work
      int misses = 0;              // thread 0's: tickets without work since then
      for (;;) {
        __syncthreads();  // every thread has read the previous ticket
        if (tid == 0) {
          int it = -1, stop = 0;
          if (ld_relaxed_s32(&L.ctl->abort)) {
            stop = 1;
          } else if (ld_acquire_s32(&L.ctl->remaining) <= 0) {
            stop = 2;
          } else if (misses >= L.nitems) {
            // a whole round of tickets found nothing to do: back off, and
            // give up once the idle limit has passed
            misses = 0;
            if ((int64_t)(gtimer() - t_idle) > L.timeout_ns) {
              set_error(L.ctl, kETIMEOUT, 3);
              stop = 3;
            } else {
              __nanosleep(500);
            }
          }
          if (!stop) {
            const unsigned long long t = atomicAdd(&L.ctl->ticket, 1ull);
            it = (int)(t % (unsigned long long)L.nitems);
            const Item item = L.items[it];
            if (atom_cas_acquire_u32(&L.sys[item.sys].sub[item.p].busy, 0u, 1u) != 0u) it = -1;
          }
          s_dyn[0] = stop;
          s_dyn[1] = it;
        }
        __syncthreads();
        const int stop = s_dyn[0], it = s_dyn[1];
        if (stop) break;
        int r = 0;
        if (it >= 0) {
          int not_done = 0;
          r = async_item(it, not_done);
          if (tid == 0) {
            const Item item = L.items[it];
            __threadfence();
            st_release_u32(&L.sys[item.sys].sub[item.p].busy, 0u);
          }
          if (r < 0) goto out;
        }
        if (tid == 0) {
          if (r > 0) {
            t_idle = gtimer();
            misses = 0;
          } else {
            ++misses;
          }
          if (past_deadline()) set_error(L.ctl, kETIMEOUT, 4);
        }
      }
    }
  }
out:
  return;
}

// --------------------------------------------------------------------------
// host-side launchers
// --------------------------------------------------------------------------

// The dynamic shared-memory limit of a kernel is process-wide state. Every
// caller sets it to the device's opt-in maximum (the same value each time), so
// host threads setting it concurrently cannot lower it under each other's
// launches; each launch passes its actual size.
static cudaError_t allow_max_smem(const void *fn) {
  int dev = 0, maxb = 0;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxb, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);  // the opt-in limit covers static + dynamic
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             maxb - (int)fa.sharedSizeBytes);
  return e;
}

template <int KIND, typename T, int NT>
static cudaError_t launch_main_t(const Launch &L, int grid, size_t smem, cudaStream_t stream) {
  auto fn = ras_main_kernel<KIND, T, NT>;
  cudaError_t e = allow_max_smem((const void *)fn);
  if (e != cudaSuccess) return e;
  Launch Lc = L;
  void *args[] = {&Lc};
  return cudaLaunchCooperativeKernel((void *)fn, dim3(grid), dim3(NT), args, smem, stream);
}

template <int KIND, typename T, int NT>
static int occupancy_t(size_t smem) {
  auto fn = ras_main_kernel<KIND, T, NT>;
  if (allow_max_smem((const void *)fn) != cudaSuccess) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, NT, smem) != cudaSuccess) return 0;
  return nb;
}

#define RAS_DISPATCH(KIND_, PREC_, NT_, CALL)                                              \
  do {                                                                                     \
    if (KIND_ == kBand) {                                                                  \
      if (PREC_ == kF64) { if (NT_ == 256) { CALL(kBand, double, 256); } else { CALL(kBand, double, 128); } } \
      else if (PREC_ == kF32) { if (NT_ == 256) { CALL(kBand, float, 256); } else { CALL(kBand, float, 128); } } \
      else { if (NT_ == 256) { CALL(kBand, __nv_bfloat16, 256); } else { CALL(kBand, __nv_bfloat16, 128); } } \
    } else if (KIND_ == kCGS) {                                                            \
      CALL(kCGS, float, 512);                                                              \
    } else if (KIND_ == kCG) {                                                             \
      if (PREC_ == kF64) { if (NT_ == 512) { CALL(kCG, double, 512); } else { CALL(kCG, double, 256); } } \
      else { if (NT_ == 512) { CALL(kCG, float, 512); } else { CALL(kCG, float, 256); } }  \
    } else if (KIND_ == kGMRES) {                                                          \
      if (PREC_ == kF64) { if (NT_ == 512) { CALL(kGMRES, double, 512); } else { CALL(kGMRES, double, 256); } } \
      else { if (NT_ == 512) { CALL(kGMRES, float, 512); } else { CALL(kGMRES, float, 256); } } \
    } else {                                                                               \
      if (PREC_ == kF64) { if (NT_ == 512) { CALL(kILU, double, 512); } else { CALL(kILU, double, 256); } } \
      else { if (NT_ == 512) { CALL(kILU, float, 512); } else { CALL(kILU, float, 256); } } \
    }                                                                                      \
  } while (0)

size_t main_smem_bytes(int kind, int prec, int nt, int Wmax, int npad_max, int kmax, int nstages) {
  size_t r = 0;
#define RAS_SMEM(K_, T_, NT_) r = Smem<K_, T_, NT_>::bytes(Wmax, npad_max, kmax, nstages)
  RAS_DISPATCH(kind, prec, nt, RAS_SMEM);
#undef RAS_SMEM
  return r;
}

int main_threads(int kind, int prec, int nt_pref) {
  if (kind == kCGS) return 512;
  // banded: BF16 records are half the bytes, so the chain is step-latency
  // bound; 128-thread CTAs fit three to an SM and run more chains at once
  // (config 4: 0.81 against 0.85 ms per synchronous iteration)
  if (kind == kBand) return nt_pref == 128 || (nt_pref == 0 && prec == kBF16) ? 128 : 256;
  return nt_pref == 512 ? 512 : 256;
}

int main_occupancy(int kind, int prec, int nt, size_t smem) {
  int r = 0;
#define RAS_OCC(K_, T_, NT_) r = occupancy_t<K_, T_, NT_>(smem)
  RAS_DISPATCH(kind, prec, nt, RAS_OCC);
#undef RAS_OCC
  return r;
}

cudaError_t launch_main(int kind, int prec, int nt, const Launch &L, int grid, size_t smem,
                        cudaStream_t stream) {
  cudaError_t e = cudaErrorInvalidValue;
#define RAS_LAUNCH(K_, T_, NT_) e = launch_main_t<K_, T_, NT_>(L, grid, smem, stream)
  RAS_DISPATCH(kind, prec, nt, RAS_LAUNCH);
#undef RAS_LAUNCH
  return e;
}

cudaError_t launch_init(const Launch &L, int nitems, cudaStream_t stream) {
  ras_init_kernel<<<nitems, 128, 0, stream>>>(L);
  ras_sysnorm_kernel<<<L.nsys, 32, 0, stream>>>(L, 0);
  return cudaGetLastError();
}

cudaError_t launch_residual(const Launch &L, int nitems, cudaStream_t stream) {
  ras_residual_kernel<<<nitems, 128, 0, stream>>>(L);
  ras_sysnorm_kernel<<<L.nsys, 32, 0, stream>>>(L, 1);
  return cudaGetLastError();
}

__global__ void fill_kernel(double *x, double v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

cudaError_t launch_fill(double *x, double v, int64_t n, cudaStream_t stream) {
  fill_kernel<<<256, 256, 0, stream>>>(x, v, n);
  return cudaGetLastError();
}

cudaError_t launch_copyback(const Launch &L, int nitems, cudaStream_t stream) {
  ras_copyback_kernel<<<nitems, 128, 0, stream>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_band_chol(const BandJob *jobs, int njobs, int max_w, double *band,
                             GridCtl *ctl, cudaStream_t stream) {
  const size_t smem = (size_t)(max_w + 1) * (max_w + 1) * sizeof(double);
  cudaError_t e = allow_max_smem((const void *)band_chol_kernel);
  if (e != cudaSuccess) return e;
  band_chol_kernel<<<njobs, 256, smem, stream>>>(jobs, band, ctl);
  return cudaGetLastError();
}

cudaError_t launch_band_lu(const BandJob *jobs, int njobs, int max_w, double *band, GridCtl *ctl,
                           cudaStream_t stream) {
  const size_t smem = (size_t)(max_w + 1) * (2 * max_w + 1) * sizeof(double);
  cudaError_t e = allow_max_smem((const void *)band_lu_kernel);
  if (e != cudaSuccess) return e;
  band_lu_kernel<<<njobs, 256, smem, stream>>>(jobs, band, ctl);
  return cudaGetLastError();
}

template <bool LU>
static void layout_t(int prec, const LayoutJob *jobs, int njobs, const double *band, void *fac,
                     cudaStream_t stream) {
  if (prec == kF64)
    band_layout_kernel<double, LU><<<njobs, 32, 0, stream>>>(jobs, band, (double *)fac);
  else if (prec == kF32)
    band_layout_kernel<float, LU><<<njobs, 32, 0, stream>>>(jobs, band, (float *)fac);
  else
    band_layout_kernel<__nv_bfloat16, LU><<<njobs, 32, 0, stream>>>(jobs, band,
                                                                    (__nv_bfloat16 *)fac);
}

cudaError_t launch_band_layout(int prec, bool lu, const LayoutJob *jobs, int njobs,
                               const double *band, void *fac, cudaStream_t stream) {
  if (lu) layout_t<true>(prec, jobs, njobs, band, fac, stream);
  else layout_t<false>(prec, jobs, njobs, band, fac, stream);
  return cudaGetLastError();
}

}  // namespace ras
