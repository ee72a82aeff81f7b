// Split form of the operator of Eq. (1) for the FP32 inner iterations of the
// mixed-precision solve, binary X:
//
//   X = [X_ones | X_head | X_tail]   (a partition of the feature columns)
//
//   X_ones  the columns that hold every row: (X_ones v)_r = sum of v over them
//           for every row r (a rank-one term), and (X_ones^T u)_j = sum of u;
//   X_head  the H most frequent other columns (H = 32 G, G a power of two),
//           kept as a row-major bitmap (G 32-bit words per row);
//   X_tail  the rest, as sliced patterns (k_sliced.cu) with FP32 piece sums.
//
// One apply: the tail gather over X (row pieces), then one pass over the rows
// (k_split_rows) that forms u_r = ones + head + tail and, reading the same
// bitmap words, adds u_r into the head columns' sums of X^T u; then the tail
// gather over X^T (column pieces), then the epilogue (k_split_epilogue) that
// completes every feature's (X^T u)_i + lambda v_i and applies the PCG step's
// epilogue in FP64. Every sum has a fixed assignment and order, so every run
// gives identical bits. Sums over rows and pieces are FP32 (the precision of
// the inner iterations); the epilogue and every dot product are FP64, each
// FP64 operation done by one lane per feature (GB300's FP64 pipe is narrow).
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "epilogue.cuh"
#include "kernels.h"

namespace rr {

namespace {

constexpr int kRowsAlign = 32;          // rows per block: a multiple of this
constexpr size_t kRowSmemMax = 160 * 1024;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Shared memory of one row block: bitmap words, slot pointers, slot sums;
// afterwards reused for the reduction of the head sums ([kWarps][G][33]).
struct RowSmem {
  size_t bits_words, ptr_ints, slots, red;
  __host__ __device__ size_t bytes() const {
    const size_t staged = bits_words + ptr_ints + slots;
    return 4 * (staged > red ? staged : red);
  }
};
__host__ __device__ inline RowSmem row_smem(int64_t rows, int G, int64_t max_slots) {
  RowSmem m;
  m.bits_words = (size_t)rows * G;
  m.ptr_ints = (size_t)((rows + 1 + 3) & ~3);
  m.slots = (size_t)((max_slots + 3) & ~3);
  m.red = (size_t)kWarps * G * 33;
  return m;
}

// The row pass. Block b owns rows [b R_B, (b + 1) R_B); it first copies its
// bitmap words, slot pointers and tail slot sums into shared memory
// (asynchronous copies, all in flight together), then each warp takes R =
// 32 / G consecutive rows per step, G lanes per row, lane `sub` holding the
// head columns of bitmap word `sub` (their v in registers, vh) and the
// running sums of X^T u over those columns (acc):
//   u_r = (sum of the row's tail slots + sum of vh over its set bits, summed
//          over the G lanes) + sum of v over the all-ones columns;
//   acc[b] += u_r for every set bit b.
// At the end the block's acc are reduced (over the row groups of a warp by
// shuffles, over the warps in shared memory) into zpart[b][0, H), and its
// sum of u into upart[b].
template <int G>
__global__ void __launch_bounds__(kThreads) k_split_rows(
    int64_t N, int64_t rows_per_blk, int64_t max_slots, const uint32_t *__restrict__ bits,
    const int32_t *__restrict__ head, const int32_t *__restrict__ ones, int32_t n_ones,
    const float *__restrict__ x32, const float *__restrict__ tsum,
    const int32_t *__restrict__ slot_ptr, float *__restrict__ u32, float *__restrict__ zpart,
    float *__restrict__ upart, const int32_t *__restrict__ stop) {
  pdl_wait();
  if (stop && *stop) return;
  constexpr int R = 32 / G;
  constexpr int H = 32 * G;
  extern __shared__ __align__(16) uint32_t rsm[];
  __shared__ float s_red[kWarps];
  __shared__ float s_ones;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sub = lane % G, grp = lane / G;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_blk;
  const int64_t r1 = min(N, r0 + rows_per_blk);
  const int64_t rows = r1 - r0;
  const RowSmem L = row_smem(rows_per_blk, G, max_slots);
  uint32_t *sbits = rsm;
  int32_t *sptr = reinterpret_cast<int32_t *>(rsm + L.bits_words);
  float *sslot = reinterpret_cast<float *>(rsm + L.bits_words + L.ptr_ints);

  // ---- stage the block's inputs (r0 * G words start 16-byte aligned: r0 % 32 == 0)
  const int32_t qbase = __ldg(slot_ptr + r0), qend = __ldg(slot_ptr + r1);
  {
    const int64_t nw = rows * G, n4 = nw >> 2;
    const uint32_t *gb = bits + r0 * G;
    for (int64_t i = threadIdx.x; i < n4; i += blockDim.x) cp_async16(sbits + 4 * i, gb + 4 * i);
    for (int64_t i = 4 * n4 + threadIdx.x; i < nw; i += blockDim.x) cp_async4(sbits + i, gb + i);
    for (int64_t i = threadIdx.x; i <= rows; i += blockDim.x) cp_async4(sptr + i, slot_ptr + r0 + i);
    for (int64_t i = threadIdx.x; i < qend - qbase; i += blockDim.x)
      cp_async4(sslot + i, tsum + qbase + i);
  }
  if (warp == 0) {   // sum of v over the all-ones columns: the lanes' loads in
                     // flight together, then a fixed shuffle tree
    float a = 0.f;
    for (int32_t i = lane; i < n_ones; i += 32) a += x32[ones[i]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) s_ones = a;
  }
  float vh[32];
#pragma unroll
  for (int b = 0; b < 32; ++b) {
    const int32_t c = __ldg(head + sub * 32 + b);
    vh[b] = c >= 0 ? __ldg(x32 + c) : 0.f;
  }
  cp_async_wait_all();
  __syncthreads();
  const float so = s_ones;

  float acc[32];
#pragma unroll
  for (int b = 0; b < 32; ++b) acc[b] = 0.f;
  float usum = 0.f;
  for (int64_t base = (int64_t)warp * R; base < rows; base += (int64_t)kWarps * R) {  // warp-uniform
    const int64_t lr = base + grp;   // local row
    const bool ok = lr < rows;
    const uint32_t w = ok ? sbits[lr * G + sub] : 0u;
    float s = 0.f;
    if (ok) {
      const int32_t q1 = sptr[lr + 1] - qbase;
      for (int32_t q = sptr[lr] - qbase + sub; q < q1; q += G) s += sslot[q];
    }
    float hs[4] = {0.f, 0.f, 0.f, 0.f};   // four independent chains of adds
#pragma unroll
    for (int b = 0; b < 32; ++b)
      if (w & (1u << b)) hs[b & 3] += vh[b];
    s += (hs[0] + hs[1]) + (hs[2] + hs[3]);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float u = s + so;
    if (ok && sub == 0) {
      u32[r0 + lr] = u;
      usum += u;
    }
#pragma unroll
    for (int b = 0; b < 32; ++b)
      if (w & (1u << b)) acc[b] += u;
  }

  // ---- reduce: over the row groups of the warp, then over the warps
#pragma unroll
  for (int o = G; o < 32; o <<= 1)
#pragma unroll
    for (int b = 0; b < 32; ++b) acc[b] += __shfl_xor_sync(0xffffffffu, acc[b], o);
  __syncthreads();   // the staged inputs are no longer read: reuse as [kWarps][G][33]
  float *red = reinterpret_cast<float *>(rsm);
  if (grp == 0) {
#pragma unroll
    for (int b = 0; b < 32; ++b) red[(warp * G + sub) * 33 + b] = acc[b];
  }
  for (int o = 16; o > 0; o >>= 1) usum += __shfl_xor_sync(0xffffffffu, usum, o);
  if (lane == 0) s_red[warp] = usum;
  __syncthreads();
  for (int c = threadIdx.x; c < H; c += blockDim.x) {
    float z = 0.f;
#pragma unroll
    for (int wv = 0; wv < kWarps; ++wv) z += red[(wv * G + c / 32) * 33 + (c & 31)];
    zpart[(int64_t)blockIdx.x * H + c] = z;
  }
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int wv = 0; wv < kWarps; ++wv) t += s_red[wv];
    upart[blockIdx.x] = t;
  }
}

// The epilogue of the split apply: t_i = (X^T u)_i from the tail's FP32 slot
// sums, the head columns' block sums or the sum of u, then t_i + lambda v_i
// and the mode's FP64 epilogue (POST with the precomputed omega / d_i). The
// special features (head, all-ones, tail columns with many slots) take one
// warp each; every other feature one lane, so each FP64 instruction works
// on 32 features. Per-block partial dots in a fixed order.
__global__ void __launch_bounds__(kThreads) k_split_epilogue(
    int64_t F, const int32_t *__restrict__ slot_ptr, const float *__restrict__ tsum,
    const uint8_t *__restrict__ is_spec, const int32_t *__restrict__ spec,
    const int32_t *__restrict__ spec_kind, int32_t n_spec, const float *__restrict__ zpart,
    const float *__restrict__ upart, int32_t nblk, int32_t H, const double *__restrict__ wd,
    CscEpilogue ep) {
  pdl_wait();
  if (ep.stop && *ep.stop) return;
  __shared__ double sm[kWarps + 1];
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double dot = 0.0;
  for (int64_t h = warp; h < n_spec; h += nwarps) {   // warp-uniform
    const int32_t i = spec[h], kind = spec_kind[h];
    double s = 0.0;
    // eight loads in flight per lane (block partials, then tail slots)
    if (kind != -2) {
      for (int32_t b0 = lane; b0 < nblk; b0 += 8 * 32) {
        float t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int32_t b = b0 + 32 * u;
          t[u] = b < nblk ? (kind >= 0 ? zpart[(int64_t)b * H + kind] : upart[b]) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) s += (double)t[u];
      }
    }
    const int32_t sq1 = slot_ptr[i + 1];
    for (int32_t q0 = slot_ptr[i] + lane; q0 < sq1; q0 += 8 * 32) {
      float t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = q0 + 32 * u < sq1 ? tsum[q0 + 32 * u] : 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u) s += (double)t[u];
    }
    s = warp_sum(s);
    if (lane == 0) epilogue(ep, i, s, dot, wd);
  }
  // every other feature: one lane each, two features per lane at a time
  // (feature i and i + stride, in that order, as the plain loop takes them);
  // the features' vectors are loaded before their slot sums (eight slot loads
  // in flight per feature), so the dependent rounds of loads overlap
  const bool need_r = ep.mode == CSC_PRE || ep.mode == CSC_POST || ep.mode == CSC_RESID;
  const int64_t stride = nwarps * 32;
  for (int64_t i0 = warp * 32; i0 < F; i0 += 2 * stride) {   // warp-uniform
    int64_t ii[2];
    bool act[2];
    int32_t q0[2], q1[2];
    double vi[2], ri[2], wdi[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      ii[h] = i0 + h * stride + lane;
      act[h] = ii[h] < F && !is_spec[ii[h]];
      q0[h] = act[h] ? slot_ptr[ii[h]] : 0;
      q1[h] = act[h] ? slot_ptr[ii[h] + 1] : 0;
      vi[h] = act[h] && ep.mode != CSC_RHS ? ep.v[ii[h]] : 0.0;
      ri[h] = act[h] && need_r ? ep.r[ii[h]] : 0.0;
      wdi[h] = act[h] && ep.mode == CSC_POST ? wd[ii[h]] : 0.0;
    }
    float s[2] = {0.f, 0.f};
    float t[2][8];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int u = 0; u < 8; ++u) t[h][u] = q0[h] + u < q1[h] ? tsum[q0[h] + u] : 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int u = 0; u < 8; ++u) s[h] += t[h][u];
      for (int32_t q = q0[h] + 8; q < q1[h]; q += 8) {   // features with more than 8 slots
        float w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) w[u] = q + u < q1[h] ? tsum[q + u] : 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) s[h] += w[u];
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (act[h]) epilogue_values(ep, ii[h], (double)s[h], vi[h], ri[h], wdi[h], dot);
  }
  const double tot = block_sum(dot, sm);
  if (threadIdx.x == 0 && ep.dot_part) ep.dot_part[blockIdx.x] = tot;
}

__global__ void k_set_wd(int64_t F, double omega, const double *__restrict__ d,
                         double *__restrict__ wd) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x)
    wd[i] = omega / d[i];
}

// row r's head bits: bit h % 32 of word h / 32 for every head column h in the row
__global__ void k_head_bits(int64_t N, int G, const int64_t *__restrict__ row_ptr,
                            const int32_t *__restrict__ col_idx, const int32_t *__restrict__ hidx,
                            uint32_t *__restrict__ bits) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < N; r += nwarps)
    for (int64_t e = row_ptr[r] + lane; e < row_ptr[r + 1]; e += 32) {
      const int32_t h = hidx[col_idx[e]];
      if (h >= 0) atomicOr(bits + r * G + (h >> 5), 1u << (h & 31));
    }
}

// entries of each row in tail columns
__global__ void k_tail_count(int64_t N, const int64_t *__restrict__ row_ptr,
                             const int32_t *__restrict__ col_idx, const uint8_t *__restrict__ cls,
                             int64_t *__restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < N; r += nwarps) {
    int64_t c = 0;
    for (int64_t e = row_ptr[r] + lane; e < row_ptr[r + 1]; e += 32) c += cls[col_idx[e]] == 0;
    c = warp_sum_i64(c);
    if (lane == 0) cnt[r] = c;
  }
}

// the tail entries of each row, in order (ballot compaction per 32 entries)
__global__ void k_tail_copy(int64_t N, const int64_t *__restrict__ row_ptr,
                            const int32_t *__restrict__ col_idx, const uint8_t *__restrict__ cls,
                            const int64_t *__restrict__ out_ptr, int32_t *__restrict__ out_idx) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < N; r += nwarps) {
    int64_t o = out_ptr[r];
    for (int64_t e0 = row_ptr[r]; e0 < row_ptr[r + 1]; e0 += 32) {
      const int64_t e = e0 + lane;
      const bool in = e < row_ptr[r + 1];
      const int32_t c = in ? col_idx[e] : 0;
      const bool keep = in && cls[c] == 0;
      const uint32_t m = __ballot_sync(0xffffffffu, keep);
      if (keep) out_idx[o + __popc(m & ((1u << lane) - 1u))] = c;
      o += __popc(m);
    }
  }
}

// the rows of the tail columns (the other columns' segments left empty)
__global__ void k_tail_csc(int64_t F, const int64_t *__restrict__ col_ptr,
                           const int32_t *__restrict__ row_idx, const int64_t *__restrict__ tptr,
                           int32_t *__restrict__ tidx) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = warp; j < F; j += nwarps) {
    const int64_t len = tptr[j + 1] - tptr[j];
    for (int64_t e = lane; e < len; e += 32) tidx[tptr[j] + e] = row_idx[col_ptr[j] + e];
  }
}

template <int G>
rr_status launch_rows(const SplitOperator &S, const int32_t *stop, cudaStream_t st) {
  const size_t smem = row_smem(S.rows_per_blk, G, S.max_slots).bytes();
  static bool attr = false;
  if (!attr) {
    RR_CUDA(cudaFuncSetAttribute(k_split_rows<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kRowSmemMax));
    attr = true;
  }
  RR_LAUNCH_PDL(k_split_rows<G>, S.nblk, kThreads, smem, st, S.N, S.rows_per_blk, S.max_slots,
                S.bits, S.head, S.ones, S.n_ones, static_cast<const float *>(S.xt.xq),
                reinterpret_cast<const float *>(S.xt.psum), S.xt.slot_ptr,
                static_cast<float *>(S.xtt.xq), S.zpart, S.upart, stop);
  return RR_OK;
}

}  // namespace

rr_status split_build(int64_t N, int64_t F, const int64_t *row_ptr, const int32_t *col_idx,
                      const int64_t *col_ptr, const int32_t *row_idx, int32_t head_opt,
                      int32_t gather_mode, SplitOperator &S, int32_t *err, cudaStream_t st) {
  S = SplitOperator{};
  if (head_opt < 0 || N < 1 || F < 1) return RR_OK;   // not used
  S.N = N;
  S.F = F;
  // ---- column classes from the column lengths (host)
  std::vector<int64_t> cp(F + 1);
  RR_CUDA(cudaMemcpyAsync(cp.data(), col_ptr, sizeof(int64_t) * (F + 1), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  std::vector<uint8_t> cls(F, 0);   // 0 tail, 1 head, 2 all-ones
  std::vector<int32_t> ones, cand;
  for (int64_t j = 0; j < F; ++j) {
    const int64_t n = cp[j + 1] - cp[j];
    if (n == N) {
      cls[j] = 2;
      ones.push_back((int32_t)j);
    } else {
      cand.push_back((int32_t)j);
    }
  }
  // the most frequent columns first (ties: lower column id)
  auto more = [&](int32_t a, int32_t b) {
    const int64_t na = cp[a + 1] - cp[a], nb = cp[b + 1] - cp[b];
    return na != nb ? na > nb : a < b;
  };
  const size_t top = std::min<size_t>(cand.size(), 1024);
  std::partial_sort(cand.begin(), cand.begin() + top, cand.end(), more);
  int32_t H = 0;
  if (head_opt > 0) {
    H = head_opt;
    if (H % 32 || H > 1024 || (H & (H - 1)) || (size_t)H > cand.size()) {
      rr_set_error("split operator: head size %d must be a power of two from 32 to 1024 and at "
                   "most the number of non-constant columns", H);
      return RR_INVALID_ARG;
    }
  } else {
    // the largest power-of-two multiple of 32 whose last column holds at
    // least N / 8 rows: a bitmap column costs two predicated adds per row in
    // the row pass whether its bit is set or not, a tail entry one gather in
    // each of the two streamed passes; on GB300 the two break even near a
    // column density of 1/8 (measured at 200,000 x 100,000: 128 head columns
    // 77.5 us per apply, 64: 79.2, 256: 81.6, 512: 93.9, none: 128.5)
    for (int32_t h = 1024; h >= 32; h >>= 1) {
      if ((size_t)h <= cand.size()) {
        const int32_t c = cand[h - 1];
        if (8 * (cp[c + 1] - cp[c]) >= N) {
          H = h;
          break;
        }
      }
    }
  }
  std::vector<int32_t> head(cand.begin(), cand.begin() + H);
  std::sort(head.begin(), head.end());
  std::vector<int32_t> hidx(F, -1);
  for (int32_t h = 0; h < H; ++h) {
    hidx[head[h]] = h;
    cls[head[h]] = 1;
  }
  S.H = H;
  S.G = std::max(1, H / 32);
  S.n_ones = (int32_t)ones.size();
  if (H == 0) {   // no bitmap: one (all-zero) word per row keeps the row pass uniform
    S.H = 32;
    S.G = 1;
    head.assign(32, -1);
  }
  // tail CSC pointers (host): the tail columns' lengths
  std::vector<int64_t> tptr(F + 1, 0);
  for (int64_t j = 0; j < F; ++j) tptr[j + 1] = tptr[j] + (cls[j] == 0 ? cp[j + 1] - cp[j] : 0);
  const int64_t tnnz = tptr[F];

  auto dalloc = [&](void **p, size_t bytes) -> rr_status {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      cudaGetLastError();
      rr_set_error("split operator: cudaMalloc of %zu bytes failed", bytes);
      return RR_OOM;
    }
    return RR_OK;
  };
  rr_status s = RR_OK;
  int32_t *d_hidx = nullptr, *t_idx = nullptr, *tt_idx = nullptr;
  int64_t *t_ptr = nullptr, *t_cnt = nullptr, *tt_ptr = nullptr, *scr = nullptr;
  uint8_t *d_cls = nullptr;
  auto run = [&]() -> rr_status {
    RR_TRY(dalloc((void **)&S.ones, sizeof(int32_t) * ones.size()));
    RR_TRY(dalloc((void **)&S.head, sizeof(int32_t) * S.H));
    RR_TRY(dalloc((void **)&S.bits, sizeof(uint32_t) * (size_t)N * S.G));
    RR_TRY(dalloc((void **)&d_hidx, sizeof(int32_t) * F));
    RR_TRY(dalloc((void **)&d_cls, F));
    if (!ones.empty())
      RR_CUDA(cudaMemcpyAsync(S.ones, ones.data(), sizeof(int32_t) * ones.size(),
                              cudaMemcpyHostToDevice, st));
    RR_CUDA(cudaMemcpyAsync(S.head, head.data(), sizeof(int32_t) * S.H, cudaMemcpyHostToDevice, st));
    RR_CUDA(cudaMemcpyAsync(d_hidx, hidx.data(), sizeof(int32_t) * F, cudaMemcpyHostToDevice, st));
    RR_CUDA(cudaMemcpyAsync(d_cls, cls.data(), F, cudaMemcpyHostToDevice, st));
    RR_CUDA(cudaMemsetAsync(S.bits, 0, sizeof(uint32_t) * (size_t)N * S.G, st));
    if (H > 0)
      RR_LAUNCH(k_head_bits, grid_for(N, kWarps), kThreads, 0, st, N, S.G, row_ptr, col_idx,
                d_hidx, S.bits);
    // tail CSR
    RR_TRY(dalloc((void **)&t_cnt, sizeof(int64_t) * (N + 1)));
    RR_TRY(dalloc((void **)&t_ptr, sizeof(int64_t) * (N + 1)));
    RR_TRY(dalloc((void **)&scr, sizeof(int64_t) * (scan_scratch_len(N + 1) + 8)));
    RR_LAUNCH(k_tail_count, grid_for(N, kWarps), kThreads, 0, st, N, row_ptr, col_idx, d_cls, t_cnt);
    RR_TRY(scan_exclusive(t_cnt, t_ptr, N, scr, st));
    RR_TRY(dalloc((void **)&t_idx, sizeof(int32_t) * tnnz));
    RR_LAUNCH(k_tail_copy, grid_for(N, kWarps), kThreads, 0, st, N, row_ptr, col_idx, d_cls, t_ptr,
              t_idx);
    // tail CSC
    RR_TRY(dalloc((void **)&tt_ptr, sizeof(int64_t) * (F + 1)));
    RR_TRY(dalloc((void **)&tt_idx, sizeof(int32_t) * tnnz));
    RR_CUDA(cudaMemcpyAsync(tt_ptr, tptr.data(), sizeof(int64_t) * (F + 1), cudaMemcpyHostToDevice, st));
    RR_LAUNCH(k_tail_csc, grid_for(F, kWarps), kThreads, 0, st, F, col_ptr, row_idx, tt_ptr, tt_idx);
    // sliced patterns of the tail, FP32 piece sums
    // (the streaming gather, the automatic choice, needs no staged chunks)
    const bool chunks = gather_mode != RR_GATHER_AUTO;
    RR_TRY(sliced_build(N, F, t_ptr, t_idx, S.xt, err, st, chunks));
    RR_TRY(sliced_build(F, N, tt_ptr, tt_idx, S.xtt, err, st, chunks));
    S.xt.psum32 = S.xtt.psum32 = true;
    if (gather_mode == RR_GATHER_AUTO) {   // the streaming gather on both passes
      RR_TRY(sliced_build_stream(S.xt, st));
      RR_TRY(sliced_build_stream(S.xtt, st));
    } else {   // a gather kernel named by the caller (comparisons, profiling)
      RR_TRY(sliced_choose_gather(S.xt, gather_mode == RR_GATHER_LANES_STAGED ? RR_GATHER_LANES
                                                                              : gather_mode, st));
      RR_TRY(sliced_choose_gather(S.xtt, gather_mode == RR_GATHER_LANES_STAGED ? RR_GATHER_STAGED
                                                                               : gather_mode, st));
    }
    // row blocks: about two per SM, a multiple of 32 rows each, their staged
    // inputs within the shared-memory budget
    std::vector<int32_t> sp(N + 1);
    RR_CUDA(cudaMemcpyAsync(sp.data(), S.xt.slot_ptr, sizeof(int32_t) * (N + 1),
                            cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    int64_t rpb = (N + 2 * kSMs - 1) / (2 * kSMs);
    rpb = std::max<int64_t>(kRowsAlign, (rpb + kRowsAlign - 1) / kRowsAlign * kRowsAlign);
    for (;;) {
      int64_t mx = 0;
      for (int64_t r0 = 0; r0 < N; r0 += rpb)
        mx = std::max<int64_t>(mx, sp[std::min(N, r0 + rpb)] - sp[r0]);
      if (row_smem(rpb, S.G, mx).bytes() <= kRowSmemMax) {
        S.max_slots = mx;
        break;
      }
      if (rpb == kRowsAlign) {
        S.xt.err = S.xtt.err = nullptr;
        return RR_OK;   // a few rows too long for the staged row pass: keep the plain form
      }
      rpb = std::max<int64_t>(kRowsAlign, rpb / 2 / kRowsAlign * kRowsAlign);
    }
    S.rows_per_blk = rpb;
    S.nblk = (int32_t)((N + rpb - 1) / rpb);
    RR_TRY(dalloc((void **)&S.zpart, sizeof(float) * (size_t)S.nblk * S.H));
    RR_TRY(dalloc((void **)&S.upart, sizeof(float) * S.nblk));
    RR_TRY(dalloc((void **)&S.wd, sizeof(double) * F));
    // features finished one warp each: head, all-ones, and long tail columns
    std::vector<int32_t> spec, kind;
    std::vector<uint8_t> is_spec(F, 0);
    std::vector<int32_t> csp(F + 1);
    RR_CUDA(cudaMemcpyAsync(csp.data(), S.xtt.slot_ptr, sizeof(int32_t) * (F + 1),
                            cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    for (int64_t j = 0; j < F; ++j) {
      int32_t kd = -3;
      if (cls[j] == 1) kd = hidx[j];
      else if (cls[j] == 2) kd = -1;
      else if (csp[j + 1] - csp[j] > 32) kd = -2;
      if (kd != -3) {
        spec.push_back((int32_t)j);
        kind.push_back(kd);
        is_spec[j] = 1;
      }
    }
    S.n_spec = (int32_t)spec.size();
    RR_TRY(dalloc((void **)&S.spec, sizeof(int32_t) * spec.size()));
    RR_TRY(dalloc((void **)&S.spec_kind, sizeof(int32_t) * spec.size()));
    RR_TRY(dalloc((void **)&S.is_spec, F));
    if (!spec.empty()) {
      RR_CUDA(cudaMemcpyAsync(S.spec, spec.data(), sizeof(int32_t) * spec.size(),
                              cudaMemcpyHostToDevice, st));
      RR_CUDA(cudaMemcpyAsync(S.spec_kind, kind.data(), sizeof(int32_t) * kind.size(),
                              cudaMemcpyHostToDevice, st));
    }
    RR_CUDA(cudaMemcpyAsync(S.is_spec, is_spec.data(), F, cudaMemcpyHostToDevice, st));
    RR_CUDA(cudaStreamSynchronize(st));
    S.active = true;
    return RR_OK;
  };
  s = run();
  cudaFree(d_hidx);
  cudaFree(d_cls);
  cudaFree(t_cnt);
  cudaFree(t_ptr);
  cudaFree(scr);
  cudaFree(t_idx);
  cudaFree(tt_ptr);
  cudaFree(tt_idx);
  if (s != RR_OK || !S.active) {
    split_free(S);
    S = SplitOperator{};
  }
  return s;
}

void split_free(SplitOperator &S) {
  cudaFree(S.ones);
  cudaFree(S.head);
  cudaFree(S.bits);
  cudaFree(S.zpart);
  cudaFree(S.upart);
  cudaFree(S.spec);
  cudaFree(S.spec_kind);
  cudaFree(S.is_spec);
  cudaFree(S.wd);
  sliced_free(S.xt);
  sliced_free(S.xtt);
  S = SplitOperator{};
}

rr_status split_set_wd(SplitOperator &S, double omega, const double *d, cudaStream_t st) {
  if (!S.active) return RR_OK;
  RR_LAUNCH(k_set_wd, grid_for(S.F, kThreads), kThreads, 0, st, S.F, omega, d, S.wd);
  return RR_OK;
}

rr_status split_apply(const SplitOperator &S, const double *v, const CscEpilogue &ep,
                      const int32_t *stop, cudaStream_t st, bool x32_ready) {
  RR_TRY(sliced_gather(S.xt, v, nullptr, stop, st, true, x32_ready));
  switch (S.G) {
    case 1: RR_TRY(launch_rows<1>(S, stop, st)); break;
    case 2: RR_TRY(launch_rows<2>(S, stop, st)); break;
    case 4: RR_TRY(launch_rows<4>(S, stop, st)); break;
    case 8: RR_TRY(launch_rows<8>(S, stop, st)); break;
    case 16: RR_TRY(launch_rows<16>(S, stop, st)); break;
    case 32: RR_TRY(launch_rows<32>(S, stop, st)); break;
    default:
      rr_set_error("split operator: bad bitmap width %d", S.G);
      return RR_UNSUPPORTED;
  }
  RR_TRY(sliced_gather(S.xtt, nullptr, nullptr, stop, st, true, true));
  RR_LAUNCH_PDL(k_split_epilogue, kVecGrid, kThreads, 0, st, S.F, S.xtt.slot_ptr,
                reinterpret_cast<const float *>(S.xtt.psum), S.is_spec, S.spec, S.spec_kind,
                S.n_spec, S.zpart, S.upart, S.nblk, S.H, S.wd, ep);
  return RR_OK;
}

}  // namespace rr
