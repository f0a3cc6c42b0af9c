// Host-callable launchers for the device kernels (implemented in ras_kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "ras_internal.h"

namespace ras {

// One banded factorisation job (one subdomain).
struct BandJob {
  int32_t n;         // rows
  int32_t w;         // true half-bandwidth
  int64_t band_off;  // offset of the row-major band in the FP64 scratch
                     // (ld = w+1, lower half, for Cholesky; ld = 2w+1 for LU)
};

// One 32-row block of one subdomain for the record layout.
struct LayoutJob {
  int32_t n, w, W, K, nb, pad_;
  int64_t band_off;  // FP64 band of the subdomain
  int64_t fac_off;   // first record of the subdomain (entries)
};

size_t main_smem_bytes(int kind, int prec, int nt, int Wmax, int npad_max, int kmax, int nstages);
int main_threads(int kind, int prec, int nt_pref);
int main_occupancy(int kind, int prec, int nt, size_t smem);
cudaError_t launch_main(int kind, int prec, int nt, const Launch &L, int grid, size_t smem,
                        cudaStream_t stream);
cudaError_t launch_init(const Launch &L, int nitems, cudaStream_t stream);
cudaError_t launch_residual(const Launch &L, int nitems, cudaStream_t stream);
cudaError_t launch_copyback(const Launch &L, int nitems, cudaStream_t stream);
cudaError_t launch_fill(double *x, double v, int64_t n, cudaStream_t stream);
cudaError_t launch_band_chol(const BandJob *jobs, int njobs, int max_w, double *band, GridCtl *ctl,
                             cudaStream_t stream);
cudaError_t launch_band_lu(const BandJob *jobs, int njobs, int max_w, double *band, GridCtl *ctl,
                           cudaStream_t stream);
// lu: the bands hold LU factors (ld = 2w+1) instead of a Cholesky factor
cudaError_t launch_band_layout(int prec, bool lu, const LayoutJob *jobs, int njobs,
                               const double *band, void *fac, cudaStream_t stream);

}  // namespace ras
