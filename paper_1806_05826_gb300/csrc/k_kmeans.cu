// K-means++ clustering of the feature columns of binary X (Section 3.4,
// "K-means++"), Euclidean distance, in exact integer arithmetic:
//   seeding distance  D2(i, c) = n_i + n_c - 2 |x_i AND x_c|
//   Lloyd score       (Q_S - 2 n_S D_iS) / n_S^2, D_iS = x_i . c_S, Q_S = ||c_S||^2
// with c_S the integer column sum of cluster S. Scores are compared by exact
// 128-bit cross multiplication, ties to the smallest S, empty clusters skipped.
// Draws: SplitMix64 (Steele, Lea & Flood 2014) seeded with the user seed,
// u_t = (x_t >> 11) 2^-53; first centre floor(u_0 F); next centre the first
// feature whose running sum of D2 exceeds floor(u_t * sum D2), or the lowest
// unchosen feature if every D2 is zero.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace rr {

namespace {

constexpr int kTile = 1024;   // features per block in the seeding pass

__device__ __forceinline__ uint64_t splitmix64_out(uint64_t seed, int64_t t) {
  uint64_t z = seed + (uint64_t)(t + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform53(uint64_t seed, int64_t t) {
  return (double)(splitmix64_out(seed, t) >> 11) * 0x1.0p-53;
}

__device__ int64_t block_sum_i64(int64_t v, int64_t *sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum_i64(v);
  __syncthreads();
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t s = 0;
    for (int i = 0; i < kWarps; ++i) s += sm[i];
    sm[kWarps] = s;
  }
  __syncthreads();
  return sm[kWarps];
}

__device__ int64_t block_incl_scan_i64(int64_t v, int64_t *sm, int64_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  __syncthreads();
  if (lane == 31) sm[warp] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int w = 0; w < kWarps; ++w) {
      int64_t t = sm[w];
      sm[w] = run;
      run += t;
    }
    sm[kWarps] = run;
  }
  __syncthreads();
  *total = sm[kWarps];
  return sm[warp] + inc;
}

__global__ void k_first_center(int64_t F, uint64_t seed, int32_t *centers, uint8_t *chosen) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t c = (int64_t)floor(uniform53(seed, 0) * (double)F);
    if (c >= F) c = F - 1;
    centers[0] = (int32_t)c;
    chosen[c] = 1;
  }
}

// ov[j] += 1 for every feature j sharing a row with centre centers[t].
__global__ void k_seed_overlap(int32_t t, const int32_t *__restrict__ centers,
                               const int64_t *__restrict__ row_ptr,
                               const int32_t *__restrict__ col_idx,
                               const int64_t *__restrict__ col_ptr,
                               const int32_t *__restrict__ row_idx, int32_t *__restrict__ ov) {
  const int64_t c = centers[t];
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = col_ptr[c] + warp; p < col_ptr[c + 1]; p += nwarps) {
    const int64_t r = row_idx[p];
    for (int64_t e = row_ptr[r] + lane; e < row_ptr[r + 1]; e += 32) atomicAdd(&ov[col_idx[e]], 1);
  }
}

// d2[i] = min(d2[i], n_i + n_c - 2 ov[i]) (plain assignment for the first centre);
// ov reset; per-tile sums of d2.
__global__ void k_seed_update(int32_t t, int64_t F, const int32_t *__restrict__ centers,
                              const int64_t *__restrict__ col_ptr, int32_t *__restrict__ ov,
                              int64_t *__restrict__ d2, int64_t *__restrict__ tile_sum) {
  __shared__ int64_t sm[kWarps + 1];
  const int64_t c = centers[t];
  const int64_t nc = col_ptr[c + 1] - col_ptr[c];
  int64_t s = 0;
  for (int u = threadIdx.x; u < kTile; u += kThreads) {
    const int64_t i = (int64_t)blockIdx.x * kTile + u;
    if (i < F) {
      const int64_t ni = col_ptr[i + 1] - col_ptr[i];
      const int64_t dist = ni + nc - 2 * (int64_t)ov[i];
      ov[i] = 0;
      const int64_t v = (t == 0) ? dist : min(d2[i], dist);
      d2[i] = v;
      s += v;
    }
  }
  s = block_sum_i64(s, sm);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = s;
}

// Single block: draws centre t.
__global__ void k_seed_pick(int32_t t, int64_t F, int64_t ntiles, uint64_t seed,
                            const int64_t *__restrict__ d2, const int64_t *__restrict__ tile_sum,
                            int32_t *centers, uint8_t *chosen) {
  __shared__ int64_t sm[kWarps + 1];
  __shared__ int64_t found;
  int64_t s = 0;
  for (int64_t b = threadIdx.x; b < ntiles; b += kThreads) s += tile_sum[b];
  const int64_t total = block_sum_i64(s, sm);
  if (threadIdx.x == 0) found = -1;
  __syncthreads();
  if (total == 0) {
    // every remaining distance is zero: lowest index not chosen yet
    for (int64_t base = 0; base < F; base += kThreads) {
      int64_t i = base + threadIdx.x;
      int64_t cand = (i < F && !chosen[i]) ? i : INT64_MAX;
      // block min
      for (int o = 16; o > 0; o >>= 1) cand = min(cand, __shfl_xor_sync(0xffffffffu, cand, o));
      __syncthreads();
      if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = cand;
      __syncthreads();
      if (threadIdx.x == 0) {
        int64_t m = INT64_MAX;
        for (int w = 0; w < kWarps; ++w) m = min(m, sm[w]);
        if (m != INT64_MAX && found < 0) found = m;
      }
      __syncthreads();
      if (found >= 0) break;
    }
  } else {
    int64_t thr = (int64_t)floor(uniform53(seed, t) * (double)total);
    if (thr >= total) thr = total - 1;
    // tile holding the threshold
    __shared__ int64_t tile_found, tile_base;
    if (threadIdx.x == 0) tile_found = -1;
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < ntiles; b0 += kThreads) {
      const int64_t b = b0 + threadIdx.x;
      const int64_t v = b < ntiles ? tile_sum[b] : 0;
      int64_t tot;
      const int64_t inc = block_incl_scan_i64(v, sm, &tot);
      if (b < ntiles && carry + inc > thr && carry + inc - v <= thr) {
        tile_found = b;
        tile_base = carry + inc - v;
      }
      __syncthreads();
      carry += tot;
      if (tile_found >= 0) break;
    }
    // feature inside the tile
    const int64_t tb = tile_found;
    int64_t run = tile_base;
    for (int u0 = 0; u0 < kTile; u0 += kThreads) {
      const int64_t i = tb * kTile + u0 + threadIdx.x;
      const int64_t v = i < F ? d2[i] : 0;
      int64_t tot;
      const int64_t inc = block_incl_scan_i64(v, sm, &tot);
      if (i < F && run + inc > thr && run + inc - v <= thr) found = i;
      __syncthreads();
      run += tot;
      if (found >= 0) break;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    centers[t] = (int32_t)found;
    if (found >= 0) chosen[found] = 1;
  }
}

__global__ void k_init_labels(int64_t F, int32_t k, const int32_t *__restrict__ centers,
                              int32_t *__restrict__ labels) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x)
    labels[i] = -1;
}

__global__ void k_set_center_labels(int32_t k, const int32_t *__restrict__ centers,
                                    int32_t *__restrict__ labels) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < k; s += gridDim.x * blockDim.x)
    labels[centers[s]] = s;
}

__global__ void k_cluster_sizes(int64_t F, const int32_t *__restrict__ labels,
                                unsigned long long *__restrict__ n_S) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t l = labels[i];
    if (l >= 0) atomicAdd(&n_S[l], 1ULL);
  }
}

// work_i = sum of the row lengths over the rows of column i (the cost of D_i.)
__global__ void k_feature_work(int64_t F, const int64_t *__restrict__ row_ptr,
                               const int64_t *__restrict__ col_ptr,
                               const int32_t *__restrict__ row_idx, int64_t *__restrict__ work) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < F; i += nwarps) {
    int64_t s = 0;
    for (int64_t p = col_ptr[i] + lane; p < col_ptr[i + 1]; p += 32) {
      const int64_t r = row_idx[p];
      s += row_ptr[r + 1] - row_ptr[r];
    }
    s = warp_sum_i64(s);
    if (lane == 0) work[i] = s;
  }
}

constexpr int kBuckets = 64;

__device__ __forceinline__ int work_bucket(int64_t w) {
  // descending work: bucket 0 holds the heaviest features
  return w <= 0 ? kBuckets - 1 : (kBuckets - 1) - (63 - __clzll((unsigned long long)w));
}

__global__ void k_bucket_count(int64_t F, const int64_t *__restrict__ work,
                               unsigned long long *__restrict__ cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[work_bucket(work[i])], 1ULL);
}

__global__ void k_bucket_scatter(int64_t F, const int64_t *__restrict__ work,
                                 unsigned long long *__restrict__ cursor,
                                 int32_t *__restrict__ order) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x)
    order[atomicAdd(&cursor[work_bucket(work[i])], 1ULL)] = (int32_t)i;
}

// D[i, S] = x_i . c_S for every feature i, and Q_S += D[i, label_i].
// Persistent blocks take features heaviest-first from a shared counter; each
// block counts, in a shared-memory histogram over clusters, the labels of all
// entries of all rows of column i.
__global__ void __launch_bounds__(kThreads) k_lloyd_scores(
    int64_t F, int32_t k, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
    const int64_t *__restrict__ col_ptr, const int32_t *__restrict__ row_idx,
    const int32_t *__restrict__ labels, const int32_t *__restrict__ order, int32_t *work_ctr,
    int32_t *__restrict__ D, unsigned long long *__restrict__ Q) {
  extern __shared__ int32_t acc[];
  __shared__ int32_t cur;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) cur = atomicAdd(work_ctr, 1);
    for (int s = threadIdx.x; s < k; s += kThreads) acc[s] = 0;
    __syncthreads();
    const int32_t it = cur;
    if (it >= F) break;
    const int64_t i = order[it];
    for (int64_t p = col_ptr[i] + warp; p < col_ptr[i + 1]; p += kWarps) {
      const int64_t r = row_idx[p];
      for (int64_t e = row_ptr[r] + lane; e < row_ptr[r + 1]; e += 32) {
        const int32_t l = labels[col_idx[e]];
        if (l >= 0) atomicAdd(&acc[l], 1);
      }
    }
    __syncthreads();
    int32_t *Di = D + i * (int64_t)k;
    for (int s = threadIdx.x; s < k; s += kThreads) Di[s] = acc[s];
    if (threadIdx.x == 0) {
      const int32_t l = labels[i];
      if (l >= 0) atomicAdd(&Q[l], (unsigned long long)acc[l]);
    }
    __syncthreads();
  }
}

struct Cand {
  int64_t a;   // Q_S - 2 n_S D_iS
  int64_t w;   // n_S^2 (0: no candidate)
  int32_t s;
};

__device__ __forceinline__ bool better(const Cand &x, const Cand &y) {
  // is x strictly preferable to y?
  if (x.w == 0) return false;
  if (y.w == 0) return true;
  const __int128 lhs = (__int128)x.a * (__int128)y.w;
  const __int128 rhs = (__int128)y.a * (__int128)x.w;
  if (lhs != rhs) return lhs < rhs;
  return x.s < y.s;
}

// One warp per feature: next[i] = argmin_S score(i, S); counts changed labels.
__global__ void k_lloyd_argmin(int64_t F, int32_t k, const int32_t *__restrict__ D,
                               const unsigned long long *__restrict__ Q,
                               const unsigned long long *__restrict__ n_S,
                               const int32_t *__restrict__ labels, int32_t *__restrict__ next,
                               unsigned long long *changes) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long changed = 0;
  for (int64_t i = warp; i < F; i += nwarps) {
    const int32_t *Di = D + i * (int64_t)k;
    Cand best{0, 0, INT32_MAX};
    for (int s = lane; s < k; s += 32) {
      const int64_t n = (int64_t)n_S[s];
      if (n == 0) continue;
      Cand c{(int64_t)Q[s] - 2 * n * (int64_t)Di[s], n * n, s};
      if (better(c, best)) best = c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      Cand o_{__shfl_xor_sync(0xffffffffu, best.a, o), __shfl_xor_sync(0xffffffffu, best.w, o),
              __shfl_xor_sync(0xffffffffu, best.s, o)};
      if (better(o_, best)) best = o_;
    }
    if (lane == 0) {
      next[i] = best.s;
      changed += (best.s != labels[i]);
    }
  }
  if (lane == 0 && changed) atomicAdd(changes, changed);
}

}  // namespace

rr_status kmeanspp_seed(int64_t N, int64_t F, const int64_t *row_ptr, const int32_t *col_idx,
                        const int64_t *col_ptr, const int32_t *row_idx, int32_t k, uint64_t seed,
                        KmeansBuffers &b, cudaStream_t st) {
  (void)N;
  const int64_t ntiles = (F + kTile - 1) / kTile;
  uint8_t *chosen = reinterpret_cast<uint8_t *>(b.next);   // F bytes of the (unused yet) next[]
  RR_CUDA(cudaMemsetAsync(chosen, 0, F, st));
  RR_CUDA(cudaMemsetAsync(b.ov, 0, sizeof(int32_t) * F, st));
  RR_LAUNCH(k_first_center, 1, 32, 0, st, F, seed, b.centers, chosen);
  for (int32_t t = 0; t < k; ++t) {
    RR_LAUNCH(k_seed_overlap, kSMs * 2, kThreads, 0, st, t, b.centers, row_ptr, col_idx, col_ptr,
              row_idx, b.ov);
    RR_LAUNCH(k_seed_update, (unsigned)ntiles, kThreads, 0, st, t, F, b.centers, col_ptr, b.ov,
              b.d2, b.part_i);
    if (t + 1 < k)
      RR_LAUNCH(k_seed_pick, 1, kThreads, 0, st, t + 1, F, ntiles, seed, b.d2, b.part_i,
                b.centers, chosen);
  }
  return RR_OK;
}

rr_status kmeans_init_labels(int64_t F, int32_t k, KmeansBuffers &b, cudaStream_t st) {
  RR_LAUNCH(k_init_labels, grid_for(F, kThreads), kThreads, 0, st, F, k, b.centers, b.labels);
  RR_LAUNCH(k_set_center_labels, grid_for(k, kThreads), kThreads, 0, st, k, b.centers, b.labels);
  return RR_OK;
}

rr_status kmeans_work_order(int64_t F, const int64_t *row_ptr, const int64_t *col_ptr,
                            const int32_t *row_idx, KmeansBuffers &b, int64_t *scratch,
                            cudaStream_t st) {
  // scratch: >= F + 2 * kBuckets + scan scratch int64
  int64_t *work = scratch;
  int64_t *cnt = scratch + F;
  int64_t *offs = cnt + kBuckets;              // kBuckets + 1
  int64_t *sscr = offs + kBuckets + 1;
  RR_LAUNCH(k_feature_work, grid_for(F, kWarps), kThreads, 0, st, F, row_ptr, col_ptr, row_idx,
            work);
  RR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * kBuckets, st));
  RR_LAUNCH(k_bucket_count, grid_for(F, kThreads), kThreads, 0, st, F, work,
            (unsigned long long *)cnt);
  RR_TRY(scan_exclusive(cnt, offs, kBuckets, sscr, st));
  RR_LAUNCH(k_bucket_scatter, grid_for(F, kThreads), kThreads, 0, st, F, work,
            (unsigned long long *)offs, b.order);
  return RR_OK;
}

rr_status kmeans_lloyd_step(int64_t N, int64_t F, const int64_t *row_ptr, const int32_t *col_idx,
                            const int64_t *col_ptr, const int32_t *row_idx, int32_t k,
                            KmeansBuffers &b, int64_t *changes_host, cudaStream_t st) {
  (void)N;
  RR_CUDA(cudaMemsetAsync(b.n_S, 0, sizeof(int64_t) * k, st));
  RR_CUDA(cudaMemsetAsync(b.Q, 0, sizeof(int64_t) * k, st));
  RR_CUDA(cudaMemsetAsync(b.changes, 0, sizeof(int64_t), st));
  RR_CUDA(cudaMemsetAsync(b.work_ctr, 0, sizeof(int32_t), st));
  RR_LAUNCH(k_cluster_sizes, grid_for(F, kThreads), kThreads, 0, st, F, b.labels,
            (unsigned long long *)b.n_S);
  const size_t smem = sizeof(int32_t) * (size_t)k;
  RR_CUDA(cudaFuncSetAttribute(k_lloyd_scores, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)std::max<size_t>(smem, 1)));
  int per_sm = 0;
  RR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lloyd_scores, kThreads, smem));
  const int grid = kSMs * std::max(1, per_sm);
  RR_LAUNCH(k_lloyd_scores, grid, kThreads, smem, st, F, k, row_ptr, col_idx, col_ptr, row_idx,
            b.labels, b.order, b.work_ctr, b.D, (unsigned long long *)b.Q);
  RR_LAUNCH(k_lloyd_argmin, grid_for(F, kWarps), kThreads, 0, st, F, k, b.D,
            (const unsigned long long *)b.Q, (const unsigned long long *)b.n_S, b.labels, b.next,
            (unsigned long long *)b.changes);
  RR_CUDA(cudaMemcpyAsync(b.labels, b.next, sizeof(int32_t) * F, cudaMemcpyDeviceToDevice, st));
  RR_CUDA(cudaMemcpyAsync(changes_host, b.changes, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  return RR_OK;
}

}  // namespace rr
