// rr_apply_noalloc: the operator A v = X^T (X v) + lambda v without any device
// allocation, for callers that must not allocate (see include/rr.h).
//
// The intermediate u = X v lives in a file-scope device array of fixed size.
// In host code the name of that array is only a host-side stand-in, so its
// device address is looked up once per device (cudaGetSymbolAddress, with the
// device current) and passed to the kernels. Every call overwrites u[0, N)
// before reading it, so nothing has to be cleared between calls. An index
// outside its range is skipped rather than read, so a bad index gives a wrong
// result but never an access outside the vectors or the array.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int64_t kNoAllocMaxRows = int64_t(1) << 22;   // 4,194,304 rows = 32 MiB of FP64
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_u_scratch[kNoAllocMaxRows];

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};

// u[r] = sum of v over the columns of row r (one warp per row).
__global__ void k_na_rows(int64_t N, int64_t F, const int64_t *__restrict__ row_ptr,
                          const int32_t *__restrict__ col_idx, const double *__restrict__ v,
                          double *__restrict__ u) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < N; r += nwarps) {
    double s = 0.0;
    for (int64_t p = row_ptr[r] + lane; p < row_ptr[r + 1]; p += 32) {
      const int32_t c = col_idx[p];
      if (c >= 0 && c < F) s += v[c];
    }
    s = rr::warp_sum(s);
    if (lane == 0) u[r] = s;
  }
}

// out[i] = sum of u over the rows of column i + lambda v[i] (one warp per column).
__global__ void k_na_cols(int64_t N, int64_t F, const int64_t *__restrict__ col_ptr,
                          const int32_t *__restrict__ row_idx, const double *__restrict__ u,
                          double lambda, const double *__restrict__ v, double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < F; i += nwarps) {
    double s = 0.0;
    for (int64_t p = col_ptr[i] + lane; p < col_ptr[i + 1]; p += 32) {
      const int32_t r = row_idx[p];
      if (r >= 0 && r < N) s += u[r];
    }
    s = rr::warp_sum(s);
    if (lane == 0) out[i] = s + lambda * v[i];
  }
}

// Device address of g_u_scratch on the current device (looked up once per device).
rr_status scratch_address(double **out) {
  int dev = -1;
  RR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    rr_set_error("rr_apply_noalloc: device ordinal %d out of range", dev);
    return RR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    RR_CUDA(cudaGetSymbolAddress(&p, g_u_scratch));
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  return RR_OK;
}

}  // namespace

extern "C" rr_status rr_apply_noalloc(int64_t n_rows, int64_t n_cols, const int64_t *row_ptr,
                                      const int32_t *col_idx, const int64_t *col_ptr,
                                      const int32_t *row_idx, double lambda, const double *v,
                                      double *out, void *stream) {
  if (n_rows < 1 || n_cols < 1 || !row_ptr || !col_idx || !col_ptr || !row_idx || !v || !out ||
      v == out) {
    rr_set_error("rr_apply_noalloc: bad sizes or NULL pointers");
    return RR_INVALID_ARG;
  }
  if (n_rows > kNoAllocMaxRows) {
    rr_set_error("rr_apply_noalloc: %lld rows exceed the fixed scratch of %lld rows",
                 (long long)n_rows, (long long)kNoAllocMaxRows);
    return RR_UNSUPPORTED;
  }
  double *u = nullptr;
  RR_TRY(scratch_address(&u));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  RR_LAUNCH(k_na_rows, rr::grid_for(n_rows, rr::kWarps), rr::kThreads, 0, st, n_rows, n_cols,
            row_ptr, col_idx, v, u);
  RR_LAUNCH(k_na_cols, rr::grid_for(n_cols, rr::kWarps), rr::kThreads, 0, st, n_rows, n_cols,
            col_ptr, row_idx, u, lambda, v, out);
  return RR_OK;
}
