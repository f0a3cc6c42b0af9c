// Host-callable launchers for the device kernels (implemented in ras_kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "ras_internal.h"

namespace ras {

// One banded Cholesky factorisation job (one subdomain).
struct BandJob {
  int32_t n;         // rows
  int32_t w;         // true half-bandwidth
  int64_t band_off;  // offset of the row-major band (ld = w+1) in the FP64 scratch
};

// One 32-row block of one subdomain for the slab layout.
struct LayoutJob {
  int32_t n, w, W, K, nb, pad_;
  int64_t band_off;  // FP64 band of the subdomain
  int64_t fac_off;   // first slab of the subdomain (entries)
};

// Per-lane row stride (elements) of a band slab of half-width W for elements
// of `esize` bytes: >= W+1, a whole number of 16-byte vectors, and padded so
// that 8 consecutive lanes' 16-byte loads fall in distinct bank groups
// (FP64: S = 2 mod 4, FP32: S = 4 mod 8, BF16: S = 8 mod 16).
__host__ __device__ inline int slab_stride(int W, int esize) {
  const int v = 16 / esize;  // elements per 16-byte vector
  int s = (W + 1 + v - 1) / v * v;
  if (((s / v) & 1) == 0) s += v;
  return s;
}

size_t main_smem_bytes(int kind, int prec, int nt, int Wmax, int npad_max, int kmax, int nstages);
int main_threads(int kind, int nt_pref);
int main_occupancy(int kind, int prec, int nt, size_t smem);
cudaError_t launch_main(int kind, int prec, int nt, const Launch &L, int grid, size_t smem,
                        cudaStream_t stream);
cudaError_t launch_init(const Launch &L, int nitems, cudaStream_t stream);
cudaError_t launch_residual(const Launch &L, int nitems, cudaStream_t stream);
cudaError_t launch_copyback(const Launch &L, int nitems, cudaStream_t stream);
cudaError_t launch_band_chol(const BandJob *jobs, int njobs, int max_w, double *band, GridCtl *ctl,
                             cudaStream_t stream);
cudaError_t launch_band_layout(int prec, const LayoutJob *jobs, int njobs, const double *band,
                               void *fac, cudaStream_t stream);

}  // namespace ras
