// The learned coarse correction's network. The paper has no learned part:
// this network takes the place of the coarse solve e_c = A_c^-1 r_c in the
// two-level cycle of Section 3.1 when the cycle runs inside the flexible CG of
// Algorithm 3 (which tolerates a preconditioner that changes from step to
// step). It is a three-layer ReLU network from the normalised restricted
// residual x = r_c / ||r_c|| (length k) to a coarse correction,
//   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), o = W3 h2 + b3,
//   e_c = ||r_c|| o   (positively homogeneous in r_c),
// trained on the squared error 0.5/B sum_b ||o_b - t_b||^2 with Adam
// (Kingma & Ba, ICLR 2015) on FP32 master weights.
//
// Training products run on the tensor cores: one tcgen05 kernel computes
// D = A B^T for BF16 operands stored K-major (row-major with K contiguous),
// 128 x 128 output tiles, FP32 accumulation in tensor memory, with the bias,
// ReLU and BF16 conversion of the next layer's input fused into the
// epilogue. Every product of the forward and backward passes is put in that
// form by keeping transposed BF16 copies (X^T, h^T, dL/da^T, W2^T, W3^T).
// Inference inside the solver is three warp-per-row mat-vecs on the BF16
// weights with FP32 accumulation (2.6 MB of weights, L2-resident).
//
// Parameter layout on the device (FP32, padded): W1 [H x kp], b1 [H],
// W2 [H x H], b2 [H], W3 [kp x H], b3 [kp] with kp = k rounded up to 128 and
// zero padding (padding stays zero: its gradients are zero).
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "handle.h"
#include "kernels.h"
#include "tc_common.cuh"

struct rr_mlp {
  int32_t k = 0, H = 0, kp = 0, max_batch = 0, Bp_max = 0;
  int64_t n_params = 0;   // padded layout
  int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
  float *P = nullptr, *G = nullptr, *Mo = nullptr, *Vo = nullptr;
  int64_t adam_t = 0;
  __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W3b = nullptr, *W2T = nullptr, *W3T = nullptr;
  __nv_bfloat16 *Xb = nullptr, *XT = nullptr, *h1b = nullptr, *h1T = nullptr, *h2b = nullptr,
                *h2T = nullptr, *dob = nullptr, *doT = nullptr, *da2b = nullptr, *da2T = nullptr,
                *da1T = nullptr;
  float *a1 = nullptr, *a2 = nullptr, *o = nullptr, *dh = nullptr, *Tn = nullptr,
        *rowloss = nullptr, *loss = nullptr;
  int64_t *bidx = nullptr;
  float *xin = nullptr, *g1 = nullptr, *g2 = nullptr;
  double *nrm = nullptr;
  // the loss metric W (rr_mlp_set_metric): BF16 [kp x kp] zero padded, and
  // the FP32 output differences of a batch [Bp x kp]; null: the plain loss
  __nv_bfloat16 *Wm = nullptr;
  float *dm = nullptr;
  bool metric = false;
  int32_t *err = nullptr;
  cudaStream_t st = nullptr;
  DevArena mem;
};

namespace rr {

namespace {
using namespace tc;

constexpr int kGM = 128, kGN = 128, kGK = 64, kGStages = 4;
constexpr int kGStageBytes = (kGM + kGN) * kGK * 2;
constexpr int kGThreads = 128;
constexpr int kGTmemCols = 128;
// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// (bits 7-9 = 1) and B (bits 10-12 = 1), both K-major, N = 128, M = 128.
constexpr uint32_t kIdescBF16 = (1u << 4) | (1u << 7) | (1u << 10) |
                                ((uint32_t)(kGN >> 3) << 17) | ((uint32_t)(kGM >> 4) << 24);

struct GemmEpi {
  const float *bias;        // [N] added to every row, or null
  float *out_f32;           // [M x ldo] the sum (pre-activation), or null
  __nv_bfloat16 *out_bf16;  // [M x ldo] relu(sum) if relu, else sum; or null
  int32_t relu;
  int32_t ldo;
};

// D (M x N) = A (M x K) B (N x K)^T for one 128 x 128 tile (blockIdx.x: N
// tile, blockIdx.y: M tile). Warp 0 lane 0 issues the TMA loads of a 4-stage
// ring, warp 1 lane 0 the MMAs, all four warps read the accumulator back
// (warp w: tile rows 32w..32w+31). Waits are bounded as in the coarse Gram.
__global__ void __launch_bounds__(kGThreads, 1)
    k_gemm_nt(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
              int32_t K, GemmEpi ep, int32_t *err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *ring = smem;
  uint64_t *full = (uint64_t *)(smem + kGStages * kGStageBytes);
  uint64_t *empty = full + kGStages;
  uint64_t *done = empty + kGStages;
  uint32_t *tmem_slot = (uint32_t *)(done + 1);
  int32_t *abort_flag = (int32_t *)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int M0 = blockIdx.y * kGM, N0 = blockIdx.x * kGN;
  const int nk = K / kGK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kGStages; ++s) {
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
                 "r"(kGTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kGStages;
      if (kb >= kGStages && !mbar_wait(&empty[s], ((kb / kGStages) + 1) & 1, abort_flag)) {
        set_dev_error(err, DEV_TIMEOUT);
        atomicExch(abort_flag, 1);
        break;
      }
      if (*(volatile int32_t *)abort_flag) break;
      uint8_t *a = ring + s * kGStageBytes;
      uint8_t *b = a + kGM * kGK * 2;
      mbar_expect_tx(&full[s], kGStageBytes);
      tma_load_2d(a, &ta, &full[s], kb * kGK, M0);
      tma_load_2d(b, &tb, &full[s], kb * kGK, N0);
      issued = kb + 1;
    }
    const int32_t never = 0;   // the issued copies must land before the CTA exits
    for (int kb = max(0, issued - kGStages); kb < issued; ++kb)
      (void)mbar_wait(&full[kb % kGStages], (kb / kGStages) & 1, &never);
  } else if (warp == 1 && lane == 0) {
    bool ok = true;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kGStages;
      if (!mbar_wait(&full[s], (kb / kGStages) & 1, abort_flag) || *(volatile int32_t *)abort_flag) {
        set_dev_error(err, DEV_TIMEOUT);
        atomicExch(abort_flag, 1);
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t a = smem_u32(ring + s * kGStageBytes);
      const uint32_t b = a + kGM * kGK * 2;
#pragma unroll
      for (int kk = 0; kk < kGK / 16; ++kk)
        umma_f16(tmem, smem_desc_sw128(a + kk * 32), smem_desc_sw128(b + kk * 32), kIdescBF16,
                 (kb > 0 || kk > 0) ? 1u : 0u);
      umma_commit(&empty[s]);
    }
    if (ok) umma_commit(done);
  }
  __syncthreads();

  bool have = !*(volatile int32_t *)abort_flag && nk > 0;
  if (have && !mbar_wait(done, 0, abort_flag)) {
    set_dev_error(err, DEV_TIMEOUT);
    have = false;
  }
  tc_fence_after();
  if (have) {
    const int64_t m = M0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < kGN; c0 += 32) {
      float v[32];
      tmem_ld_32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      const int n0 = N0 + c0;
      if (ep.bias) {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] += ep.bias[n0 + j];
      }
      if (ep.out_f32) {
        float4 *o4 = reinterpret_cast<float4 *>(ep.out_f32 + m * ep.ldo + n0);
#pragma unroll
        for (int j = 0; j < 8; ++j) o4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
      }
      if (ep.out_bf16) {
        __nv_bfloat162 *ob = reinterpret_cast<__nv_bfloat162 *>(ep.out_bf16 + m * ep.ldo + n0);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float x0 = v[2 * j], x1 = v[2 * j + 1];
          if (ep.relu) {
            x0 = fmaxf(x0, 0.0f);
            x1 = fmaxf(x1, 0.0f);
          }
          ob[j] = __floats2bfloat162_rn(x0, x1);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kGTmemCols)
                 : "memory");
  }
}

// ---------------------------------------------------------------- elementwise

__global__ void k_mlp_refresh(int32_t H, int32_t kp, const float *__restrict__ P, int64_t oW1,
                              int64_t oW2, int64_t oW3, __nv_bfloat16 *__restrict__ W1b,
                              __nv_bfloat16 *__restrict__ W2b, __nv_bfloat16 *__restrict__ W3b,
                              __nv_bfloat16 *__restrict__ W2T, __nv_bfloat16 *__restrict__ W3T) {
  const int64_t n1 = (int64_t)H * kp, n2 = (int64_t)H * H;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n1; e += stride) {
    W1b[e] = __float2bfloat16(P[oW1 + e]);
    W3b[e] = __float2bfloat16(P[oW3 + e]);                    // [kp x H]
    const int64_t i = e / H, h = e % H;                        // W3[i][h] -> W3T[h][i]
    W3T[h * kp + i] = __float2bfloat16(P[oW3 + e]);
  }
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n2; e += stride) {
    W2b[e] = __float2bfloat16(P[oW2 + e]);
    const int64_t i = e / H, h = e % H;
    W2T[h * H + i] = __float2bfloat16(P[oW2 + e]);
  }
}

// One block per batch row b < Bp: x and t rows from the pair arrays (row
// idx[b], or b when idx is null), divided by ||x|| when `normalize` (the
// homogeneous scaling of the learned map); BF16 x row and its transposed
// column, FP32 target row; zero rows and columns as padding.
__global__ void k_mlp_pack(int32_t B, int32_t Bp, int32_t k, int32_t kp, const int64_t *idx,
                           const float *__restrict__ X, const float *__restrict__ T,
                           int32_t normalize, __nv_bfloat16 *__restrict__ Xb,
                           __nv_bfloat16 *__restrict__ XT, float *__restrict__ Tn) {
  __shared__ float red[32];
  __shared__ float scale;
  const int b = blockIdx.x;
  const int64_t row = b < B ? (idx ? idx[b] : b) : -1;
  float s = 1.0f;
  if (normalize && row >= 0) {
    float acc = 0.0f;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
      const float v = X[row * k + i];
      acc += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.0f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      scale = t > 0.0f ? 1.0f / sqrtf(t) : 0.0f;
    }
    __syncthreads();
    s = scale;
  }
  for (int i = threadIdx.x; i < kp; i += blockDim.x) {
    const bool in = row >= 0 && i < k;
    const float x = in ? X[row * k + i] * s : 0.0f;
    const float t = in && T ? T[row * k + i] * s : 0.0f;
    Xb[(int64_t)b * kp + i] = __float2bfloat16(x);
    XT[(int64_t)i * Bp + b] = __float2bfloat16(x);
    if (Tn) Tn[(int64_t)b * kp + i] = t;
  }
}

// do = (o - t) / B for the B real rows (zero elsewhere), in place in o; BF16
// copies dob and doT; per-row squared errors.
__global__ void k_mlp_dout(int32_t B, int32_t Bp, int32_t k, int32_t kp, float *__restrict__ o,
                           const float *__restrict__ Tn, __nv_bfloat16 *__restrict__ dob,
                           __nv_bfloat16 *__restrict__ doT, float *__restrict__ rowloss) {
  __shared__ float red[32];
  const int b = blockIdx.x;
  float acc = 0.0f;
  for (int i = threadIdx.x; i < kp; i += blockDim.x) {
    const int64_t e = (int64_t)b * kp + i;
    float d = 0.0f;
    if (b < B && i < k) {
      const float diff = o[e] - Tn[e];
      acc += diff * diff;
      d = diff / (float)B;
    }
    o[e] = d;
    dob[e] = __float2bfloat16(d);
    doT[(int64_t)i * Bp + b] = __float2bfloat16(d);
  }
  for (int w = 16; w > 0; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    rowloss[b] = t;
  }
}

// With a metric W, pass 1: d = o - t for the B real rows (zero elsewhere) in
// FP32 (dm) and BF16 (dob), the left operand of d W^T = d W (W symmetric).
__global__ void k_mlp_diff(int32_t B, int32_t k, int32_t kp, const float *__restrict__ o,
                           const float *__restrict__ Tn, float *__restrict__ dm,
                           __nv_bfloat16 *__restrict__ dob) {
  const int b = blockIdx.x;
  for (int i = threadIdx.x; i < kp; i += blockDim.x) {
    const int64_t e = (int64_t)b * kp + i;
    const float d = (b < B && i < k) ? o[e] - Tn[e] : 0.0f;
    dm[e] = d;
    dob[e] = __float2bfloat16(d);
  }
}

// Pass 2, after g = d W (FP32, in o): do = g / B in place and its BF16
// copies; per-row d^T W d = sum_i d_i g_i.
__global__ void k_mlp_dout_w(int32_t B, int32_t Bp, int32_t kp, float *__restrict__ o,
                             const float *__restrict__ dm, __nv_bfloat16 *__restrict__ dob,
                             __nv_bfloat16 *__restrict__ doT, float *__restrict__ rowloss) {
  __shared__ float red[32];
  const int b = blockIdx.x;
  float acc = 0.0f;
  for (int i = threadIdx.x; i < kp; i += blockDim.x) {
    const int64_t e = (int64_t)b * kp + i;
    const float g = b < B ? o[e] : 0.0f;
    acc += dm[e] * g;
    const float d = g / (float)B;
    o[e] = d;
    dob[e] = __float2bfloat16(d);
    doT[(int64_t)i * Bp + b] = __float2bfloat16(d);
  }
  for (int w = 16; w > 0; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    rowloss[b] = t;
  }
}

// da = dh * (a > 0) in place; optional BF16 copy and BF16 transposed copy.
__global__ void k_mlp_relu_back(int32_t Bp, int32_t H, float *__restrict__ dh,
                                const float *__restrict__ a, __nv_bfloat16 *__restrict__ dab,
                                __nv_bfloat16 *__restrict__ daT) {
  const int64_t n = (int64_t)Bp * H;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float d = a[e] > 0.0f ? dh[e] : 0.0f;
    dh[e] = d;
    const __nv_bfloat16 db = __float2bfloat16(d);
    if (dab) dab[e] = db;
    const int64_t b = e / H, h = e % H;
    daT[h * Bp + b] = db;
  }
}

// dst (C x R) = src (R x C)^T, BF16.
__global__ void k_transpose_bf16(int32_t R, int32_t C, const __nv_bfloat16 *__restrict__ src,
                                 __nv_bfloat16 *__restrict__ dst) {
  __shared__ __nv_bfloat16 t[32][34];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int r = r0 + y, c = c0 + threadIdx.x;
    if (r < R && c < C) t[y][threadIdx.x] = src[(int64_t)r * C + c];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = c0 + y, r = r0 + threadIdx.x;
    if (r < R && c < C) dst[(int64_t)c * R + r] = t[threadIdx.x][y];
  }
}

// g[n] = sum over the Bp rows of d[b, n] (fixed order).
__global__ void k_colsum(int32_t Bp, int32_t N, const float *__restrict__ d, float *__restrict__ g) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int b = 0; b < Bp; ++b) s += d[(int64_t)b * N + n];
    g[n] = s;
  }
}

__global__ void k_loss_sum(int32_t B, const float *__restrict__ rowloss, float *loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < B; ++b) s += rowloss[b];
    *loss = (float)(0.5 * s / B);
  }
}

// Adam on the FP32 master weights: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr (m / c1) / (sqrt(v / c2) + eps) with the bias corrections c1 = 1 - b1^t, c2 = 1 - b2^t.
__global__ void k_adam(int64_t n, float *__restrict__ P, const float *__restrict__ G,
                       float *__restrict__ Mo, float *__restrict__ Vo, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float g = G[e];
    const float m = b1 * Mo[e] + (1.0f - b1) * g;
    const float v = b2 * Vo[e] + (1.0f - b2) * g * g;
    Mo[e] = m;
    Vo[e] = v;
    P[e] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  }
}

// Batch rows drawn uniformly from n pairs: SplitMix64 (Steele, Lea & Flood 2014)
// at counter base + b, mapped by the high bits: floor(u * n), u = (x >> 11) 2^-53.
__global__ void k_draw_rows(int32_t B, int64_t n, uint64_t seed, int64_t base, int64_t *idx) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    uint64_t z = seed + (uint64_t)(base + b + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    const double u = (double)(z >> 11) * 0x1.0p-53;
    int64_t r = (int64_t)(u * (double)n);
    idx[b] = r < n ? r : n - 1;
  }
}

// ---------------------------------------------------------------- inference

// x = r_c / ||r_c|| (FP32, zero padded to kp) from the restricted vector;
// nrm = ||r_c|| in FP64. One block.
__global__ void k_mlp_input(int32_t k, int32_t kp, const double *__restrict__ rc,
                            float *__restrict__ x, double *__restrict__ nrm,
                            const int32_t *__restrict__ stop) {
  pdl_wait();
  if (stop && *stop) return;
  __shared__ double sm[kWarps + 1];
  extern __shared__ double rcs[];
  double acc = 0.0;
  for (int S = threadIdx.x; S < k; S += blockDim.x) {
    const double t = rc[S];
    rcs[S] = t;
    acc += t * t;
  }
  const double n2 = block_sum(acc, sm);
  const double n = sqrt(n2);
  const double inv = n > 0.0 ? 1.0 / n : 0.0;
  for (int S = threadIdx.x; S < kp; S += blockDim.x) x[S] = S < k ? (float)(rcs[S] * inv) : 0.0f;
  if (threadIdx.x == 0) *nrm = n;
}

// y = act(W x + bias) for a [rows x cols] BF16 weight (warp per row, x staged
// in shared memory, 8 BF16 per 16-byte load). out64: y64[r] = (*scale) * y
// for r < n_out (the output layer) instead of the FP32 y.
__global__ void k_mlp_gemv(int32_t rows, int32_t cols, const __nv_bfloat16 *__restrict__ W,
                           const float *__restrict__ bias, const float *__restrict__ x,
                           int32_t relu, float *__restrict__ y, int32_t n_out,
                           const double *__restrict__ scale, double *__restrict__ y64,
                           const int32_t *__restrict__ stop) {
  pdl_wait();
  if (stop && *stop) return;
  extern __shared__ float xs[];
  for (int i = threadIdx.x; i < cols; i += blockDim.x) xs[i] = x[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < rows; r += nwarps) {
    const uint4 *wr = reinterpret_cast<const uint4 *>(W + r * cols);
    float acc = 0.0f;
    for (int c8 = lane; c8 < cols / 8; c8 += 32) {
      const uint4 q = __ldg(wr + c8);
      const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&q);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 f = __bfloat1622float2(h[j]);
        acc = fmaf(f.x, xs[c8 * 8 + 2 * j], acc);
        acc = fmaf(f.y, xs[c8 * 8 + 2 * j + 1], acc);
      }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      float v = acc + bias[r];
      if (relu) v = fmaxf(v, 0.0f);
      if (y64) {
        if (r < n_out) y64[r] = *scale * (double)v;
      } else {
        y[r] = v;
      }
    }
  }
}

// ---------------------------------------------------------------- host

PFN_cuTensorMapEncodeTiled_v12000 gemm_encoder() { return encode_fn(); }

rr_status make_map(CUtensorMap *map, const __nv_bfloat16 *base, int64_t rows, int64_t K) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = gemm_encoder();
  if (!enc) {
    rr_set_error("cuTensorMapEncodeTiled is not available");
    return RR_CUDA_ERROR;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  const cuuint32_t box[2] = {kGK, kGM};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(base),
                          dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) {
    rr_set_error("cuTensorMapEncodeTiled failed (%d)", (int)cr);
    return RR_CUDA_ERROR;
  }
  return RR_OK;
}

// D (M x N) = A (M x K) B (N x K)^T with the epilogue ep; M, N multiples of 128, K of 64.
rr_status gemm_nt(int64_t M, int64_t N, int64_t K, const __nv_bfloat16 *A, const __nv_bfloat16 *B,
                  const GemmEpi &ep, int32_t *err, cudaStream_t st) {
  if (M % kGM || N % kGN || K % kGK || K <= 0) {
    rr_set_error("gemm_nt: sizes %lld x %lld x %lld not multiples of the tile", (long long)M,
                 (long long)N, (long long)K);
    return RR_INVALID_ARG;
  }
  CUtensorMap ta, tb;
  RR_TRY(make_map(&ta, A, M, K));
  RR_TRY(make_map(&tb, B, N, K));
  const size_t smem = (size_t)kGStages * kGStageBytes + 1024 + 256;
  static bool attr = false;
  if (!attr) {
    RR_CUDA(cudaFuncSetAttribute(k_gemm_nt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  RR_LAUNCH(k_gemm_nt, dim3((unsigned)(N / kGN), (unsigned)(M / kGM)), kGThreads, smem, st, ta, tb,
            (int32_t)K, ep, err);
  return RR_OK;
}

rr_status check_err(rr_mlp *m, const char *where) {
  int32_t e = 0;
  RR_CUDA(cudaMemcpyAsync(&e, m->err, sizeof(int32_t), cudaMemcpyDeviceToHost, m->st));
  RR_CUDA(cudaStreamSynchronize(m->st));
  if (e == DEV_OK) return RR_OK;
  RR_CUDA(cudaMemsetAsync(m->err, 0, sizeof(int32_t), m->st));
  rr_set_error("%s: device error %d (a bounded wait expired)", where, e);
  return e == DEV_TIMEOUT ? RR_TIMEOUT : RR_CUDA_ERROR;
}

rr_status refresh(rr_mlp *m) {
  RR_LAUNCH(k_mlp_refresh, grid_for((int64_t)m->H * m->kp, kThreads), kThreads, 0, m->st, m->H,
            m->kp, m->P, m->oW1, m->oW2, m->oW3, m->W1b, m->W2b, m->W3b, m->W2T, m->W3T);
  return RR_OK;
}

// Forward pass of Bp rows already packed in Xb / XT: a1, h1b, a2, h2b, o.
rr_status forward(rr_mlp *m, int32_t Bp) {
  cudaStream_t st = m->st;
  RR_TRY(gemm_nt(Bp, m->H, m->kp, m->Xb, m->W1b, GemmEpi{m->P + m->ob1, m->a1, m->h1b, 1, m->H},
                 m->err, st));
  RR_TRY(gemm_nt(Bp, m->H, m->H, m->h1b, m->W2b, GemmEpi{m->P + m->ob2, m->a2, m->h2b, 1, m->H},
                 m->err, st));
  RR_TRY(gemm_nt(Bp, m->kp, m->H, m->h2b, m->W3b, GemmEpi{m->P + m->ob3, m->o, nullptr, 0, m->kp},
                 m->err, st));
  return RR_OK;
}

// Loss and gradients (into G, padded layout) of B packed rows with targets Tn.
rr_status backward(rr_mlp *m, int32_t B, int32_t Bp) {
  cudaStream_t st = m->st;
  const int32_t H = m->H, kp = m->kp;
  if (m->metric) {
    RR_LAUNCH(k_mlp_diff, Bp, kThreads, 0, st, B, m->k, kp, m->o, m->Tn, m->dm, m->dob);
    RR_TRY(gemm_nt(Bp, kp, kp, m->dob, m->Wm, GemmEpi{nullptr, m->o, nullptr, 0, kp}, m->err, st));
    RR_LAUNCH(k_mlp_dout_w, Bp, kThreads, 0, st, B, Bp, kp, m->o, m->dm, m->dob, m->doT,
              m->rowloss);
  } else {
    RR_LAUNCH(k_mlp_dout, Bp, kThreads, 0, st, B, Bp, m->k, kp, m->o, m->Tn, m->dob, m->doT,
              m->rowloss);
  }
  const dim3 tb(32, 8);
  RR_LAUNCH(k_transpose_bf16, dim3((unsigned)(H / 32), (unsigned)(Bp / 32)), tb, 0, st, Bp, H,
            m->h2b, m->h2T);
  RR_LAUNCH(k_transpose_bf16, dim3((unsigned)(H / 32), (unsigned)(Bp / 32)), tb, 0, st, Bp, H,
            m->h1b, m->h1T);
  // layer 3: gW3 = do^T h2, gb3 = column sums of do, dh2 = do W3
  RR_TRY(gemm_nt(kp, H, Bp, m->doT, m->h2T, GemmEpi{nullptr, m->G + m->oW3, nullptr, 0, H}, m->err, st));
  RR_LAUNCH(k_colsum, grid_for(kp, kThreads), kThreads, 0, st, Bp, kp, m->o, m->G + m->ob3);
  RR_TRY(gemm_nt(Bp, H, kp, m->dob, m->W3T, GemmEpi{nullptr, m->dh, nullptr, 0, H}, m->err, st));
  // layer 2
  RR_LAUNCH(k_mlp_relu_back, grid_for((int64_t)Bp * H, kThreads), kThreads, 0, st, Bp, H, m->dh,
            m->a2, m->da2b, m->da2T);
  RR_LAUNCH(k_colsum, grid_for(H, kThreads), kThreads, 0, st, Bp, H, m->dh, m->G + m->ob2);
  RR_TRY(gemm_nt(H, H, Bp, m->da2T, m->h1T, GemmEpi{nullptr, m->G + m->oW2, nullptr, 0, H}, m->err, st));
  RR_TRY(gemm_nt(Bp, H, H, m->da2b, m->W2T, GemmEpi{nullptr, m->dh, nullptr, 0, H}, m->err, st));
  // layer 1
  RR_LAUNCH(k_mlp_relu_back, grid_for((int64_t)Bp * H, kThreads), kThreads, 0, st, Bp, H, m->dh,
            m->a1, (__nv_bfloat16 *)nullptr, m->da1T);
  RR_LAUNCH(k_colsum, grid_for(H, kThreads), kThreads, 0, st, Bp, H, m->dh, m->G + m->ob1);
  RR_TRY(gemm_nt(H, kp, Bp, m->da1T, m->XT, GemmEpi{nullptr, m->G + m->oW1, nullptr, 0, kp}, m->err, st));
  RR_LAUNCH(k_loss_sum, 1, 32, 0, st, B, m->rowloss, m->loss);
  return RR_OK;
}

inline int32_t round128(int64_t a) { return (int32_t)((a + 127) / 128 * 128); }

void to_padded(const rr_mlp *m, const float *packed, std::vector<float> &pad) {
  const int32_t k = m->k, H = m->H, kp = m->kp;
  pad.assign(m->n_params, 0.0f);
  const float *q = packed;
  for (int h = 0; h < H; ++h)
    for (int i = 0; i < k; ++i) pad[m->oW1 + (int64_t)h * kp + i] = *q++;
  for (int h = 0; h < H; ++h) pad[m->ob1 + h] = *q++;
  for (int64_t e = 0; e < (int64_t)H * H; ++e) pad[m->oW2 + e] = *q++;
  for (int h = 0; h < H; ++h) pad[m->ob2 + h] = *q++;
  for (int i = 0; i < k; ++i)
    for (int h = 0; h < H; ++h) pad[m->oW3 + (int64_t)i * H + h] = *q++;
  for (int i = 0; i < k; ++i) pad[m->ob3 + i] = *q++;
}

void to_packed(const rr_mlp *m, const std::vector<float> &pad, float *packed) {
  const int32_t k = m->k, H = m->H, kp = m->kp;
  float *q = packed;
  for (int h = 0; h < H; ++h)
    for (int i = 0; i < k; ++i) *q++ = pad[m->oW1 + (int64_t)h * kp + i];
  for (int h = 0; h < H; ++h) *q++ = pad[m->ob1 + h];
  for (int64_t e = 0; e < (int64_t)H * H; ++e) *q++ = pad[m->oW2 + e];
  for (int h = 0; h < H; ++h) *q++ = pad[m->ob2 + h];
  for (int i = 0; i < k; ++i)
    for (int h = 0; h < H; ++h) *q++ = pad[m->oW3 + (int64_t)i * H + h];
  for (int i = 0; i < k; ++i) *q++ = pad[m->ob3 + i];
}

rr_status pack_rows(rr_mlp *m, int32_t B, const int64_t *idx, const float *X, const float *T,
                    int32_t normalize) {
  const int32_t Bp = round128(B);
  RR_LAUNCH(k_mlp_pack, Bp, kThreads, 0, m->st, B, Bp, m->k, m->kp, idx, X, T, normalize, m->Xb,
            m->XT, m->Tn);
  return RR_OK;
}

}  // namespace

// The learned correction inside the solver: e_c = ||r_c|| net(r_c / ||r_c||)
// from the restriction's item sums (see k_pcg.cu), all kernels returning at
// once when *stop is set.
rr_status mlp_coarse(const rr_mlp *m, const RestrictPlan &plan, const double *s, double *ec,
                     const int32_t *stop, cudaStream_t st) {
  const int32_t k = m->k, kp = m->kp, H = m->H;
  (void)s;
  RR_LAUNCH_PDL(k_mlp_input, 1, kThreads, sizeof(double) * k, st, k, kp, (const double *)plan.rc,
                m->xin, m->nrm, stop);
  const int g1 = (H + kWarps - 1) / kWarps;
  RR_LAUNCH_PDL(k_mlp_gemv, g1, kThreads, sizeof(float) * kp, st, H, kp, m->W1b, m->P + m->ob1, m->xin,
            1, m->g1, 0, (const double *)nullptr, (double *)nullptr, stop);
  RR_LAUNCH_PDL(k_mlp_gemv, g1, kThreads, sizeof(float) * H, st, H, H, m->W2b, m->P + m->ob2, m->g1, 1,
            m->g2, 0, (const double *)nullptr, (double *)nullptr, stop);
  const int g3 = (kp + kWarps - 1) / kWarps;
  RR_LAUNCH_PDL(k_mlp_gemv, g3, kThreads, sizeof(float) * H, st, kp, H, m->W3b, m->P + m->ob3, m->g2, 0,
            (float *)nullptr, k, m->nrm, ec, stop);
  return RR_OK;
}

int32_t mlp_k(const rr_mlp *m) { return m->k; }

}  // namespace rr

using namespace rr;

extern "C" {

rr_status rr_mlp_create(int32_t k, int32_t hidden, int32_t max_batch, const float *params_host,
                        void *stream, rr_mlp **out) {
  if (!out || !params_host || k < 1 || hidden < 128 || hidden % 128 || max_batch < 1 ||
      max_batch > (1 << 16)) {
    rr_set_error("rr_mlp_create: need k >= 1, hidden a positive multiple of 128, "
                 "1 <= max_batch <= 65536 and params");
    return RR_INVALID_ARG;
  }
  *out = nullptr;
  rr_mlp *m = new rr_mlp();
  m->k = k;
  m->H = hidden;
  m->kp = round128(k);
  m->max_batch = max_batch;
  m->Bp_max = round128(max_batch);
  m->st = static_cast<cudaStream_t>(stream);
  const int64_t H = hidden, kp = m->kp, Bp = m->Bp_max;
  m->oW1 = 0;
  m->ob1 = m->oW1 + H * kp;
  m->oW2 = m->ob1 + H;
  m->ob2 = m->oW2 + H * H;
  m->oW3 = m->ob2 + H;
  m->ob3 = m->oW3 + kp * H;
  m->n_params = m->ob3 + kp;
  auto fail = [&](rr_status s) {
    rr_mlp_free(m);
    return s;
  };
  rr_status s = RR_OK;
#define MLP_ALLOC(ptr, n)                   \
  if ((s = m->mem.alloc(&(ptr), (n))) != RR_OK) return fail(s);
  MLP_ALLOC(m->P, m->n_params);
  MLP_ALLOC(m->G, m->n_params);
  MLP_ALLOC(m->Mo, m->n_params);
  MLP_ALLOC(m->Vo, m->n_params);
  MLP_ALLOC(m->W1b, H * kp);
  MLP_ALLOC(m->W2b, H * H);
  MLP_ALLOC(m->W3b, kp * H);
  MLP_ALLOC(m->W2T, H * H);
  MLP_ALLOC(m->W3T, H * kp);
  MLP_ALLOC(m->Xb, Bp * kp);
  MLP_ALLOC(m->XT, kp * Bp);
  MLP_ALLOC(m->h1b, Bp * H);
  MLP_ALLOC(m->h1T, H * Bp);
  MLP_ALLOC(m->h2b, Bp * H);
  MLP_ALLOC(m->h2T, H * Bp);
  MLP_ALLOC(m->dob, Bp * kp);
  MLP_ALLOC(m->doT, kp * Bp);
  MLP_ALLOC(m->da2b, Bp * H);
  MLP_ALLOC(m->da2T, H * Bp);
  MLP_ALLOC(m->da1T, H * Bp);
  MLP_ALLOC(m->a1, Bp * H);
  MLP_ALLOC(m->a2, Bp * H);
  MLP_ALLOC(m->o, Bp * kp);
  MLP_ALLOC(m->dh, Bp * H);
  MLP_ALLOC(m->Tn, Bp * kp);
  MLP_ALLOC(m->rowloss, Bp);
  MLP_ALLOC(m->loss, 1);
  MLP_ALLOC(m->bidx, Bp);
  MLP_ALLOC(m->xin, kp);
  MLP_ALLOC(m->g1, H);
  MLP_ALLOC(m->g2, H);
  MLP_ALLOC(m->nrm, 1);
  MLP_ALLOC(m->err, 1);
#undef MLP_ALLOC
  if (cudaMemsetAsync(m->Mo, 0, sizeof(float) * m->n_params, m->st) != cudaSuccess ||
      cudaMemsetAsync(m->Vo, 0, sizeof(float) * m->n_params, m->st) != cudaSuccess ||
      cudaMemsetAsync(m->err, 0, sizeof(int32_t), m->st) != cudaSuccess) {
    rr_set_error("rr_mlp_create: memset failed");
    return fail(RR_CUDA_ERROR);
  }
  if ((s = rr_mlp_set_params(m, params_host)) != RR_OK) return fail(s);
  *out = m;
  return RR_OK;
}

rr_status rr_mlp_set_metric(rr_mlp *m, const float *W_host) {
  if (!m) {
    rr_set_error("rr_mlp_set_metric: NULL network");
    return RR_INVALID_ARG;
  }
  if (!W_host) {
    m->metric = false;
    return RR_OK;
  }
  const int32_t k = m->k, kp = m->kp;
  float wmax = 0.0f, asym = 0.0f;
  for (int64_t e = 0; e < (int64_t)k * k; ++e) {
    if (!isfinite(W_host[e])) {
      rr_set_error("rr_mlp_set_metric: non-finite entry");
      return RR_INVALID_ARG;
    }
    wmax = fmaxf(wmax, fabsf(W_host[e]));
  }
  for (int32_t i = 0; i < k; ++i)
    for (int32_t j = 0; j < i; ++j)
      asym = fmaxf(asym, fabsf(W_host[(int64_t)i * k + j] - W_host[(int64_t)j * k + i]));
  if (asym > 1e-6f * wmax) {
    rr_set_error("rr_mlp_set_metric: W must be symmetric");
    return RR_INVALID_ARG;
  }
  if (!m->Wm) {
    RR_TRY(m->mem.alloc(&m->Wm, (int64_t)kp * kp));
    RR_TRY(m->mem.alloc(&m->dm, (int64_t)m->Bp_max * kp));
  }
  std::vector<__nv_bfloat16> pad((size_t)kp * kp, __float2bfloat16(0.0f));
  for (int32_t i = 0; i < k; ++i)
    for (int32_t j = 0; j < k; ++j)
      pad[(size_t)i * kp + j] = __float2bfloat16(W_host[(int64_t)i * k + j]);
  RR_CUDA(cudaMemcpyAsync(m->Wm, pad.data(), sizeof(__nv_bfloat16) * pad.size(),
                          cudaMemcpyHostToDevice, m->st));
  RR_CUDA(cudaStreamSynchronize(m->st));
  m->metric = true;
  return RR_OK;
}

rr_status rr_mlp_set_params(rr_mlp *m, const float *params_host) {
  if (!m || !params_host) {
    rr_set_error("rr_mlp_set_params: NULL argument");
    return RR_INVALID_ARG;
  }
  std::vector<float> pad;
  to_padded(m, params_host, pad);
  RR_CUDA(cudaMemcpyAsync(m->P, pad.data(), sizeof(float) * m->n_params, cudaMemcpyHostToDevice, m->st));
  RR_TRY(refresh(m));
  RR_CUDA(cudaStreamSynchronize(m->st));
  return RR_OK;
}

rr_status rr_mlp_get_params(const rr_mlp *m, float *params_host) {
  if (!m || !params_host) {
    rr_set_error("rr_mlp_get_params: NULL argument");
    return RR_INVALID_ARG;
  }
  std::vector<float> pad(m->n_params);
  RR_CUDA(cudaMemcpyAsync(pad.data(), m->P, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost, m->st));
  RR_CUDA(cudaStreamSynchronize(m->st));
  to_packed(m, pad, params_host);
  return RR_OK;
}

int64_t rr_mlp_param_count(int32_t k, int32_t hidden) {
  return 2LL * hidden * k + (int64_t)hidden * hidden + 2LL * hidden + k;
}

rr_status rr_mlp_forward(rr_mlp *m, int32_t B, const float *X, float *out) {
  if (!m || !X || !out || B < 1 || B > m->max_batch) {
    rr_set_error("rr_mlp_forward: NULL argument or batch outside [1, max_batch]");
    return RR_INVALID_ARG;
  }
  const int32_t Bp = round128(B);
  RR_TRY(pack_rows(m, B, nullptr, X, nullptr, 0));
  RR_TRY(forward(m, Bp));
  RR_CUDA(cudaMemcpy2DAsync(out, sizeof(float) * m->k, m->o, sizeof(float) * m->kp,
                            sizeof(float) * m->k, B, cudaMemcpyDeviceToDevice, m->st));
  return check_err(m, "rr_mlp_forward");
}

rr_status rr_mlp_grad(rr_mlp *m, int32_t B, const float *X, const float *T, float *grads_host,
                      float *loss_host) {
  if (!m || !X || !T || B < 1 || B > m->max_batch) {
    rr_set_error("rr_mlp_grad: NULL argument or batch outside [1, max_batch]");
    return RR_INVALID_ARG;
  }
  const int32_t Bp = round128(B);
  RR_TRY(pack_rows(m, B, nullptr, X, T, 0));
  RR_TRY(forward(m, Bp));
  RR_TRY(backward(m, B, Bp));
  RR_TRY(check_err(m, "rr_mlp_grad"));
  if (grads_host) {
    std::vector<float> pad(m->n_params);
    RR_CUDA(cudaMemcpyAsync(pad.data(), m->G, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost, m->st));
    RR_CUDA(cudaStreamSynchronize(m->st));
    to_packed(m, pad, grads_host);
  }
  if (loss_host) {
    RR_CUDA(cudaMemcpyAsync(loss_host, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->st));
    RR_CUDA(cudaStreamSynchronize(m->st));
  }
  return RR_OK;
}

rr_status rr_mlp_train(rr_mlp *m, int64_t n_pairs, const float *Xp, const float *Tp, int32_t batch,
                       int32_t steps, float lr, uint64_t seed, float *loss_host) {
  NvtxRange nvtx_range("rr_mlp_train");
  if (!m || !Xp || !Tp || n_pairs < 1 || batch < 1 || batch > m->max_batch || steps < 0 ||
      !(lr > 0.0f)) {
    rr_set_error("rr_mlp_train: bad arguments");
    return RR_INVALID_ARG;
  }
  const int32_t Bp = round128(batch);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int32_t s = 0; s < steps; ++s) {
    RR_LAUNCH(k_draw_rows, grid_for(batch, kThreads), kThreads, 0, m->st, batch, n_pairs, seed,
              (int64_t)s * batch, m->bidx);
    RR_TRY(pack_rows(m, batch, m->bidx, Xp, Tp, 1));
    RR_TRY(forward(m, Bp));
    RR_TRY(backward(m, batch, Bp));
    m->adam_t += 1;
    const float c1 = (float)(1.0 - pow((double)b1, (double)m->adam_t));
    const float c2 = (float)(1.0 - pow((double)b2, (double)m->adam_t));
    RR_LAUNCH(k_adam, grid_for(m->n_params, kThreads), kThreads, 0, m->st, m->n_params, m->P, m->G,
              m->Mo, m->Vo, lr, b1, b2, eps, c1, c2);
    RR_TRY(refresh(m));
    if (loss_host)
      RR_CUDA(cudaMemcpyAsync(loss_host + s, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->st));
  }
  return check_err(m, "rr_mlp_train");
}

void rr_mlp_free(rr_mlp *m) {
  if (!m) return;
  cudaStreamSynchronize(m->st);
  m->mem.free_all();
  delete m;
}

}  // extern "C"
