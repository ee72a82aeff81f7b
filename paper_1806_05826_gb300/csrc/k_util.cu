// Setup utilities: prefix sums, CSR validation and the CSR -> CSC transpose
// (the transposed copy X^T u needs, with rows ascending inside every column).
#include "common.cuh"
#include "kernels.h"

namespace rr {

namespace {

constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;

// Exclusive scan of one value per thread across the block; *total gets the sum.
__device__ int64_t block_exclusive_scan(int64_t v, int64_t *smem /*kWarps+1*/, int64_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  __syncthreads();
  if (lane == 31) smem[warp] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int w = 0; w < kWarps; ++w) {
      int64_t t = smem[w];
      smem[w] = run;
      run += t;
    }
    smem[kWarps] = run;
  }
  __syncthreads();
  *total = smem[kWarps];
  return smem[warp] + inc - v;
}

__global__ void k_scan_tiles(const int64_t *__restrict__ in, int64_t n, int64_t *__restrict__ sums) {
  __shared__ int64_t sm[kWarps + 1];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += in[base + i];
  int64_t total;
  block_exclusive_scan(s, sm, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Single block: in-place exclusive scan of the tile sums.
__global__ void k_scan_sums(int64_t *sums, int64_t ntiles) {
  __shared__ int64_t sm[kWarps + 1];
  int64_t carry = 0;
  for (int64_t b = 0; b < ntiles; b += kThreads) {
    int64_t i = b + threadIdx.x;
    int64_t v = i < ntiles ? sums[i] : 0;
    int64_t total;
    int64_t ex = block_exclusive_scan(v, sm, &total);
    if (i < ntiles) sums[i] = carry + ex;
    carry += total;
    __syncthreads();
  }
}

__global__ void k_scan_apply(const int64_t *__restrict__ in, int64_t n,
                             const int64_t *__restrict__ offs, int64_t *__restrict__ out) {
  __shared__ int64_t sm[kWarps + 1];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t vals[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    vals[i] = (base + i < n) ? in[base + i] : 0;
    s += vals[i];
  }
  int64_t total;
  int64_t run = offs[blockIdx.x] + block_exclusive_scan(s, sm, &total);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    run += vals[i];
    if (base + i < n) out[base + i + 1] = run;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
}

__global__ void k_validate_csr(int64_t n_rows, int64_t n_cols, int64_t nnz,
                               const int64_t *__restrict__ row_ptr,
                               const int32_t *__restrict__ col_idx, int32_t *err) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < n_rows; r += nwarps) {
    int64_t b = row_ptr[r], e = row_ptr[r + 1];
    // a row's bounds must lie in [0, nnz] before its indices are read
    bool bad = e < b || b < 0 || e > nnz;
    if (!bad) {
      for (int64_t p = b + lane; p < e; p += 32) {
        int32_t c = col_idx[p];
        if (c < 0 || c >= n_cols) bad = true;
        if (p > b && col_idx[p - 1] >= c) bad = true;
      }
    }
    if (__any_sync(0xffffffffu, bad)) {
      if (lane == 0) set_dev_error(err, DEV_BAD_INDEX);
      return;
    }
  }
}

__global__ void k_count_cols(int64_t nnz, const int32_t *__restrict__ col_idx,
                             unsigned long long *__restrict__ counts) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&counts[col_idx[e]], 1ULL);
}

// Unordered scatter of row ids into their columns (order fixed by the next kernel).
__global__ void k_scatter_rows(int64_t n_rows, const int64_t *__restrict__ row_ptr,
                               const int32_t *__restrict__ col_idx,
                               unsigned long long *__restrict__ cursor, int32_t *__restrict__ tmp) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < n_rows; r += nwarps) {
    for (int64_t p = row_ptr[r] + lane; p < row_ptr[r + 1]; p += 32) {
      unsigned long long pos = atomicAdd(&cursor[col_idx[p]], 1ULL);
      tmp[pos] = (int32_t)r;
    }
  }
}

constexpr int kSmallSeg = kThreads;         // sorted by ranks in shared memory
constexpr int kBitmapWords = 8192;          // 262,144 rows per bitmap pass

// Sorts every column segment of tmp (distinct row ids) into out, ascending.
// Short segments: rank of each element by comparison with all others.
// Long segments: a shared-memory bitmap of the row range, then a block scan
// of per-thread popcounts gives every row its output position.
__global__ void __launch_bounds__(kThreads) k_sort_segments(int64_t n_cols, int64_t n_rows,
                                                            const int64_t *__restrict__ col_ptr,
                                                            const int32_t *__restrict__ tmp,
                                                            int32_t *__restrict__ out) {
  extern __shared__ uint32_t bitmap[];           // kBitmapWords
  __shared__ int32_t vals[kSmallSeg];
  __shared__ int64_t sm[kWarps + 1];
  constexpr int kWordsPerThread = kBitmapWords / kThreads;
  for (int64_t j = blockIdx.x; j < n_cols; j += gridDim.x) {
    const int64_t b = col_ptr[j], m = col_ptr[j + 1] - b;
    if (m == 0) continue;
    if (m <= kSmallSeg) {
      if (threadIdx.x < m) vals[threadIdx.x] = tmp[b + threadIdx.x];
      __syncthreads();
      if (threadIdx.x < m) {
        int32_t v = vals[threadIdx.x];
        int rank = 0;
        for (int u = 0; u < m; ++u) rank += vals[u] < v;
        out[b + rank] = v;
      }
      __syncthreads();
      continue;
    }
    int64_t written = 0;
    for (int64_t base = 0; base < n_rows; base += 32LL * kBitmapWords) {
      for (int w = threadIdx.x; w < kBitmapWords; w += kThreads) bitmap[w] = 0u;
      __syncthreads();
      for (int64_t p = threadIdx.x; p < m; p += kThreads) {
        int64_t rr = (int64_t)tmp[b + p] - base;
        if (rr >= 0 && rr < 32LL * kBitmapWords) atomicOr(&bitmap[rr >> 5], 1u << (rr & 31));
      }
      __syncthreads();
      const int w0 = threadIdx.x * kWordsPerThread;
      int64_t cnt = 0;
      for (int w = 0; w < kWordsPerThread; ++w) cnt += __popc(bitmap[w0 + w]);
      int64_t total;
      int64_t pos = b + written + block_exclusive_scan(cnt, sm, &total);
      for (int w = 0; w < kWordsPerThread; ++w) {
        uint32_t bits = bitmap[w0 + w];
        while (bits) {
          int bit = __ffs(bits) - 1;
          bits &= bits - 1;
          out[pos++] = (int32_t)(base + (int64_t)(w0 + w) * 32 + bit);
        }
      }
      written += total;
      __syncthreads();
    }
  }
}

__global__ void k_iota(int64_t *out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = i;
}

__global__ void k_fill(double *out, double v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = v;
}

}  // namespace

int64_t scan_scratch_len(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

rr_status scan_exclusive(const int64_t *in, int64_t *out, int64_t n, int64_t *scratch,
                         cudaStream_t st) {
  if (n <= 0) {
    RR_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
    return RR_OK;
  }
  const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
  RR_LAUNCH(k_scan_tiles, (unsigned)ntiles, kThreads, 0, st, in, n, scratch);
  RR_LAUNCH(k_scan_sums, 1, kThreads, 0, st, scratch, ntiles);
  RR_LAUNCH(k_scan_apply, (unsigned)ntiles, kThreads, 0, st, in, n, scratch, out);
  return RR_OK;
}

rr_status validate_csr(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t *row_ptr,
                       const int32_t *col_idx, int32_t *err, cudaStream_t st) {
  if (n_rows == 0) return RR_OK;
  RR_LAUNCH(k_validate_csr, grid_for(n_rows, kWarps), kThreads, 0, st, n_rows, n_cols, nnz, row_ptr,
            col_idx, err);
  return RR_OK;
}

rr_status transpose_pattern(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t *row_ptr,
                            const int32_t *col_idx, int64_t *col_ptr, int32_t *row_idx,
                            int64_t *counts, int64_t *cursor, int32_t *tmp,
                            int64_t *scan_scratch, cudaStream_t st) {
  RR_CUDA(cudaMemsetAsync(counts, 0, sizeof(int64_t) * n_cols, st));
  if (nnz > 0)
    RR_LAUNCH(k_count_cols, grid_for(nnz, kThreads), kThreads, 0, st, nnz, col_idx,
              (unsigned long long *)counts);
  RR_TRY(scan_exclusive(counts, col_ptr, n_cols, scan_scratch, st));
  if (nnz == 0) return RR_OK;
  RR_CUDA(cudaMemcpyAsync(cursor, col_ptr, sizeof(int64_t) * n_cols, cudaMemcpyDeviceToDevice, st));
  RR_LAUNCH(k_scatter_rows, grid_for(n_rows, kWarps), kThreads, 0, st, n_rows, row_ptr, col_idx,
            (unsigned long long *)cursor, tmp);
  const size_t smem = sizeof(uint32_t) * kBitmapWords;
  static bool attr_set = false;
  if (!attr_set) {
    RR_CUDA(cudaFuncSetAttribute(k_sort_segments, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    attr_set = true;
  }
  RR_LAUNCH(k_sort_segments, (unsigned)std::min<int64_t>(n_cols, kSMs * 6), kThreads, smem, st,
            n_cols, n_rows, col_ptr, tmp, row_idx);
  return RR_OK;
}

rr_status iota_i64(int64_t *out, int64_t n, cudaStream_t st) {
  if (n > 0) RR_LAUNCH(k_iota, grid_for(n, kThreads), kThreads, 0, st, out, n);
  return RR_OK;
}

rr_status fill_f64(double *out, double v, int64_t n, cudaStream_t st) {
  if (n > 0) RR_LAUNCH(k_fill, grid_for(n, kThreads), kThreads, 0, st, out, v, n);
  return RR_OK;
}

}  // namespace rr
