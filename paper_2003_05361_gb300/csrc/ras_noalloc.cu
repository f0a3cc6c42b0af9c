// ras_relres_noalloc: the relative residual ||b - A x|| / ||b|| without any
// device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured (allocation is not a capturable operation), programs whose
// device memory is owned by a fixed pool or a custom allocator that forbids
// raw cudaMalloc, and real-time loops that must not allocate after start-up.
// ras_relres needs a context built by ras_setup, which allocates; this entry
// point instead takes the matrix and vectors the caller already holds on the
// device and keeps its only scratch - one pair of partial sums per chunk of
// kChunkRows rows - in the file-scope array below.
//
// The array is part of the loaded library: every GPU that loads it holds
// 2 * kMaxChunks doubles (1 MiB) until the process exits. Every call shares
// it and it keeps the last call's contents; each call writes every partial it
// later reads, so nothing has to be cleared, but calls whose work overlaps on
// the GPU (two streams, or two host threads) race on it and must be ordered by
// the caller.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/ras.h"

namespace {

constexpr int kChunkRows = 1024;    // rows per partial sum
constexpr int kMaxChunks = 65536;   // => n <= 67,108,864 rows
constexpr int kThreads = 256;

static __device__ __align__(256) double g_relres_scratch[2 * kMaxChunks];

// Deterministic block reduction of two values (same tree on every call).
__device__ __forceinline__ void block_sum2_det(double &a, double &b) {
  __shared__ double ra[kThreads / 32], rb[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    ra[threadIdx.x >> 5] = a;
    rb[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  double sa = ra[0], sb = rb[0];
#pragma unroll
  for (int w = 1; w < kThreads / 32; ++w) {
    sa += ra[w];
    sb += rb[w];
  }
  a = sa;
  b = sb;
}

// Block c: partial sums of r_i^2 and b_i^2 over rows [c*kChunkRows, ...).
__global__ void __launch_bounds__(kThreads)
    relres_partials_kernel(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const double *__restrict__ val, const double *__restrict__ b,
                           const double *__restrict__ x, double *__restrict__ scratch) {
  const int r0 = blockIdx.x * kChunkRows;
  const int r1 = min(n, r0 + kChunkRows);
  double rr = 0.0, bb = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += kThreads) {
    double r = b[i];
    for (int k = rp[i]; k < rp[i + 1]; ++k) r -= val[k] * x[ci[k]];
    rr += r * r;
    bb += b[i] * b[i];
  }
  block_sum2_det(rr, bb);
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x] = rr;
    scratch[2 * blockIdx.x + 1] = bb;
  }
}

// One block: fixed-order sum of the chunk partials, then the ratio.
__global__ void __launch_bounds__(kThreads)
    relres_final_kernel(int nchunks, const double *__restrict__ scratch, double *__restrict__ out) {
  double rr = 0.0, bb = 0.0;
  for (int c = threadIdx.x; c < nchunks; c += kThreads) {
    rr += scratch[2 * c];
    bb += scratch[2 * c + 1];
  }
  block_sum2_det(rr, bb);
  if (threadIdx.x == 0) *out = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
}

// Device address of g_relres_scratch for each device, looked up with that
// device current (the host-side name of the array is only a stand-in and
// must never be passed to a kernel). The first call on a device does the
// look-up; later calls that are not being captured into a CUDA graph look it
// up again (a cheap table query once the module is loaded), so the address
// stays right even after cudaDeviceReset reloads the module; calls made
// during a capture use the address cached by an earlier call.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_addr[kMaxDevices] = {};

ras_status scratch_for_current_device(cudaStream_t st, double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RAS_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return RAS_ENOTSUP;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    (void)cudaGetLastError();  // the query itself is not an error of this call
    cs = cudaStreamCaptureStatusActive;  // treat an unanswerable query as a capture
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev] || cs == cudaStreamCaptureStatusNone) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_relres_scratch) != cudaSuccess || !p) return RAS_ECUDA;
    g_scratch_addr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[dev];
  return RAS_OK;
}

}  // namespace

extern "C" ras_status ras_relres_noalloc(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                                         const double *val, const double *b, const double *x,
                                         double *relres, void *cuda_stream) {
  if (n <= 0 || !row_ptr || !col_idx || !val || !b || !x || !relres) return RAS_EINVAL;
  if ((int64_t)n > (int64_t)kChunkRows * kMaxChunks) return RAS_EINVAL;  // beyond the scratch
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  double *scratch = nullptr;
  ras_status s = scratch_for_current_device(st, &scratch);
  if (s != RAS_OK) return s;
  const int nchunks = (n + kChunkRows - 1) / kChunkRows;
  relres_partials_kernel<<<nchunks, kThreads, 0, st>>>(n, row_ptr, col_idx, val, b, x, scratch);
  relres_final_kernel<<<1, kThreads, 0, st>>>(nchunks, scratch, relres);
  return cudaGetLastError() == cudaSuccess ? RAS_OK : RAS_ECUDA;
}
