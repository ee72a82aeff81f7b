// Coarse Gram G = C^T C on the 5th-generation tensor cores (tcgen05), the one
// dense contraction of the method (Section 3.2: X_c^T X_c with X_c = X P; the
// integer counts C = X * onehot(labels) carry it, G = D_s^-1 X_c^T X_c D_s^-1).
//
// Operands: Ct (k_pad x n_pad, FP16, rows = clusters, K = samples contiguous)
// serves as both A and B (K-major). TMA brings 128 x 64 tiles with the 128-byte
// swizzle into a 4-stage shared-memory ring; one thread issues
// tcgen05.mma.kind::f16 (M = N = 128, K = 16) into a 128-column FP32
// accumulator in tensor memory; four warps read it back with tcgen05.ld.
//
// Exactness: counts are integers <= 2048 (exact in FP16), products <= 2^22;
// the K range of one CTA is limited so that every FP32 partial sum stays
// below 2^24 (exact), and the chunks are added into G in FP64 (exact below
// 2^53, so the order of the atomic additions does not matter).
//
// Every wait on an mbarrier is bounded: on expiry the CTA records
// DEV_TIMEOUT, waits (bounded) for its own copies still in flight, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace rr {

namespace {
using namespace tc;

constexpr int kTM = 128, kTN = 128, kTK = 64;   // tile: rows x cols x K per stage
constexpr int kStages = 4;
constexpr int kStageBytes = (kTM + kTN) * kTK * 2;   // A and B tiles, FP16
constexpr int kTmemCols = 128;
constexpr int kGramThreads = 128;

// Instruction descriptor, kind::f16: FP32 accumulator, FP16 A and B, both
// K-major, N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kTN >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);

// One CTA: the lower tile (ti >= tj) blockIdx.x % n_tiles over the K chunk
// blockIdx.x / n_tiles.
__global__ void __launch_bounds__(kGramThreads, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap tmap, int32_t k, int32_t n_tiles_lower,
              int64_t n_pad, int64_t k_chunk, double *__restrict__ G, int32_t *err,
              uint32_t wait_limit) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte alignment of the tile ring (the 128-byte swizzle repeats every 1024 bytes)
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *ring = smem;
  uint64_t *full = (uint64_t *)(smem + kStages * kStageBytes);
  uint64_t *empty = full + kStages;
  uint64_t *done = empty + kStages;
  uint32_t *tmem_slot = (uint32_t *)(done + 1);
  int32_t *abort_flag = (int32_t *)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tile = blockIdx.x % n_tiles_lower;
  const int64_t chunk = blockIdx.x / n_tiles_lower;
  int ti = (int)((sqrt(8.0 * (double)tile + 1.0) - 1.0) * 0.5);
  while ((int64_t)(ti + 1) * (ti + 2) / 2 <= tile) ++ti;
  while ((int64_t)ti * (ti + 1) / 2 > tile) --ti;
  const int tj = (int)(tile - (int64_t)ti * (ti + 1) / 2);
  const int S0 = ti * kTM, T0 = tj * kTN;
  const int64_t kbeg = chunk * k_chunk;
  const int64_t kend = min(n_pad, kbeg + k_chunk);
  const int nk = (int)((kend - kbeg) / kTK);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: TMA loads of the A (rows S0..) and B (rows T0..) tiles
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages;
      if (kb >= kStages &&
          !mbar_wait(&empty[s], ((kb / kStages) + 1) & 1, abort_flag, wait_limit)) {
        set_dev_error(err, DEV_TIMEOUT);
        atomicExch(abort_flag, 1);
        break;
      }
      if (*(volatile int32_t *)abort_flag) break;
      uint8_t *a = ring + s * kStageBytes;
      uint8_t *b = a + kTM * kTK * 2;
      mbar_expect_tx(&full[s], kStageBytes);
      const int32_t x = (int32_t)(kbeg + (int64_t)kb * kTK);
      tma_load_2d(a, &tmap, &full[s], x, S0);
      tma_load_2d(b, &tmap, &full[s], x, T0);
      issued = kb + 1;
    }
    // copies of the last stages may still be in flight if the consumer
    // stopped: wait for them (bounded) before the CTA can exit
    const int32_t never = 0;   // the copies themselves must land: ignore the abort flag
    for (int kb = max(0, issued - kStages); kb < issued; ++kb)
      (void)mbar_wait(&full[kb % kStages], (kb / kStages) & 1, &never);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    bool ok = true;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages;
      if (!mbar_wait(&full[s], (kb / kStages) & 1, abort_flag, wait_limit) ||
          *(volatile int32_t *)abort_flag) {
        set_dev_error(err, DEV_TIMEOUT);
        atomicExch(abort_flag, 1);
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t a = smem_u32(ring + s * kStageBytes);
      const uint32_t b = a + kTM * kTK * 2;
#pragma unroll
      for (int kk = 0; kk < kTK / 16; ++kk) {
        umma_f16(tmem, smem_desc_sw128(a + kk * 32), smem_desc_sw128(b + kk * 32), kIdesc,
                 (kb > 0 || kk > 0) ? 1u : 0u);
      }
      umma_commit(&empty[s]);   // the stage is free once these MMAs have read it
    }
    if (ok) umma_commit(done);
  }
  __syncthreads();

  // epilogue: all four warps; warp w owns accumulator rows 32w..32w+31
  bool have = !*(volatile int32_t *)abort_flag && nk > 0;
  if (have && !mbar_wait(done, 0, abort_flag, wait_limit)) {
    set_dev_error(err, DEV_TIMEOUT);
    have = false;
  }
  tc_fence_after();
  if (have) {
    const int row = S0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < kTN; c0 += 32) {
      float v[32];
      tmem_ld_32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row < k) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = T0 + c0 + j;
          if (col < k && col <= row && v[j] != 0.0f) {
            atomicAdd(&G[(int64_t)row * k + col], (double)v[j]);
            if (col != row) atomicAdd(&G[(int64_t)col * k + row], (double)v[j]);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

}  // namespace

int64_t gram_tc_chunk(int32_t max_count) {
  // largest multiple of the K tile with chunk * max_count^2 < 2^24
  if (max_count <= 0) max_count = 1;
  const int64_t c = ((int64_t)1 << 24) / ((int64_t)max_count * max_count);
  return (c / kTK) * kTK;
}

rr_status gram_tensor_cores(int32_t k, int32_t k_pad, int64_t n_pad, const void *Ct,
                            int32_t max_count, double *G, int32_t *err, cudaStream_t st,
                            int32_t wait_limit) {
  const int64_t chunk = gram_tc_chunk(max_count);
  // the pipeline's waits (the drain of copies in flight keeps the default)
  const uint32_t limit = wait_limit == 0 ? tc::kSpinLimit : wait_limit < 0 ? 0u : (uint32_t)wait_limit;
  if (chunk < kTK || k_pad % kTM != 0 || n_pad % kTK != 0) {
    rr_set_error("tensor-core Gram: counts too large for exact FP32 chunks");
    return RR_UNSUPPORTED;
  }
  PFN_cuTensorMapEncodeTiled_v12000 enc = tc::encode_fn();
  if (!enc) {
    rr_set_error("cuTensorMapEncodeTiled is not available");
    return RR_CUDA_ERROR;
  }
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)n_pad, (cuuint64_t)k_pad};
  const cuuint64_t strides[1] = {(cuuint64_t)n_pad * 2};
  const cuuint32_t box[2] = {kTK, kTM};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(Ct), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) {
    rr_set_error("cuTensorMapEncodeTiled failed (%d)", (int)cr);
    return RR_CUDA_ERROR;
  }
  const int32_t nt = k_pad / kTM;
  const int32_t n_lower = nt * (nt + 1) / 2;
  const int64_t n_chunks = (n_pad + chunk - 1) / chunk;
  const size_t smem = (size_t)kStages * kStageBytes + 1024 + 256;
  static bool attr = false;
  if (!attr) {
    RR_CUDA(cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  RR_CUDA(cudaMemsetAsync(G, 0, sizeof(double) * (size_t)k * k, st));
  RR_LAUNCH(k_gram_tc, (unsigned)(n_lower * n_chunks), kGramThreads, smem, st, map, k, n_lower,
            n_pad, chunk, G, err, limit);
  return RR_OK;
}

}  // namespace rr
