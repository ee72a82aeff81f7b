// Internal helpers shared by the library's CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <algorithm>

#include "rr.h"

// ---------------------------------------------------------------- host side

void rr_set_error(const char *fmt, ...);
extern thread_local int64_t rr_launch_counter;

#define RR_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      rr_set_error("%s:%d: %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return RR_CUDA_ERROR;                                                        \
    }                                                                              \
  } while (0)

#define RR_TRY(call)                     \
  do {                                   \
    rr_status s_ = (call);               \
    if (s_ != RR_OK) return s_;          \
  } while (0)

// A named NVTX range over a scope (for nsys and ncu's NVTX filters; a no-op
// without a tool attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// The setup's phases as consecutive NVTX ranges: next(name) closes the open
// one and opens the next; the last one closes with the object.
struct NvtxPhases {
  bool open = false;
  void next(const char *name) {
    if (open) nvtxRangePop();
    nvtxRangePushA(name);
    open = true;
  }
  ~NvtxPhases() {
    if (open) nvtxRangePop();
  }
};

// Every kernel launch goes through this so launches can be counted.
#define RR_LAUNCH(kernel, grid, block, smem, stream, ...)                          \
  do {                                                                             \
    kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                    \
    ++rr_launch_counter;                                                           \
    cudaError_t e_ = cudaGetLastError();                                           \
    if (e_ != cudaSuccess) {                                                       \
      rr_set_error("%s:%d: launch %s: %s", __FILE__, __LINE__, #kernel,            \
                   cudaGetErrorString(e_));                                        \
      return RR_CUDA_ERROR;                                                        \
    }                                                                              \
  } while (0)

// Launch with programmatic dependent launch: the kernel may be scheduled while
// its predecessor on the stream finishes; it must call rr::pdl_wait() before it
// reads anything (every kernel launched this way does so first).
#define RR_LAUNCH_PDL(kernel_, grid_, block_, smem_, stream_, ...)                 \
  do {                                                                             \
    cudaLaunchConfig_t cfg_{};                                                     \
    cfg_.gridDim = dim3(grid_);                                                    \
    cfg_.blockDim = dim3(block_);                                                  \
    cfg_.dynamicSmemBytes = (smem_);                                               \
    cfg_.stream = (stream_);                                                       \
    cudaLaunchAttribute at_[1];                                                    \
    at_[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;                \
    at_[0].val.programmaticStreamSerializationAllowed = 1;                         \
    cfg_.attrs = at_;                                                              \
    cfg_.numAttrs = 1;                                                             \
    cudaError_t e_ = cudaLaunchKernelEx(&cfg_, kernel_, __VA_ARGS__);              \
    ++rr_launch_counter;                                                           \
    if (e_ != cudaSuccess) {                                                       \
      rr_set_error("%s:%d: launch %s: %s", __FILE__, __LINE__, #kernel_,           \
                   cudaGetErrorString(e_));                                        \
      return RR_CUDA_ERROR;                                                        \
    }                                                                              \
  } while (0)

namespace rr {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kSMs = 152;                    // GB300: 2 dies x 76 SMs
constexpr int kMaxGrid = kSMs * 8;           // resident-CTA-sized grids for grid-stride loops

inline int grid_for(int64_t work_items, int per_block) {
  int64_t g = (work_items + per_block - 1) / per_block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, kMaxGrid));
}

// Error word in device memory: kernels record the first failure and return;
// the host reads it after the stream synchronises. Never __trap().
enum DevError : int32_t {
  DEV_OK = 0,
  DEV_BAD_INDEX = 1,      // CSR index out of range / not increasing
  DEV_NOT_SPD = 2,        // Cholesky pivot <= 0
  DEV_COUNT_OVERFLOW = 3, // a per-row cluster count above the FP16-exact range
  DEV_NONFINITE = 4,
  DEV_TIMEOUT = 5,        // a bounded wait on an mbarrier expired
};

}  // namespace rr

// ---------------------------------------------------------------- device side

#ifdef __CUDACC__
namespace rr {

// Waits until the grids this kernel depends on have completed and their
// memory is visible (a no-op unless launched with RR_LAUNCH_PDL).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void set_dev_error(int32_t *err, int32_t code) {
  atomicCAS(err, 0, code);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int64_t warp_sum_i64(int64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of a block's per-thread values in a fixed order (same result on every run).
// Every thread of the block must call it; the result is returned to all threads.
__device__ __forceinline__ double block_sum(double v, double *smem /*>= kWarps+1*/) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += smem[i];
    smem[kWarps] = s;
  }
  __syncthreads();
  return smem[kWarps];
}

// Fixed-order sum of n per-block partial values, computed identically by every
// block that calls it (so consumers need no separate finishing kernel).
__device__ __forceinline__ double sum_partials(const double *parts, int n, double *smem) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += parts[i];
  return block_sum(v, smem);
}

}  // namespace rr
#endif
