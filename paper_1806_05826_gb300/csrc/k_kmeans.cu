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

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rr {

namespace {

constexpr int kTile = kThreads;   // features per block in the seeding pass (one each)
// below this many (row entry x delta pair) updates a Lloyd step pushes the
// changes with global atomics instead of re-gathering every feature
constexpr unsigned long long kPushWorkLimit = 200ull * 1000 * 1000;

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

// Overlaps of the newest centre c with every feature, |x_i AND x_c|, are
// counted in one of two ways (the same integers either way):
//  push: for every row of c, ov[j] += 1 for each feature j of that row (cost:
//        the entries of c's rows, about n_c nnz / N, as atomic increments);
//  pull: c's rows set in a bitmap of N bits, then every listed feature's
//        column is read in chunks of kSeedChunk entries and its rows tested
//        against the bitmap (cost: the listed columns' entries, read in order).
// Only features whose distance can still drop are listed for a pull. Since
// D2(i, c) = |x_i XOR x_c| >= |n_i - n_c|, a feature with d2[i] <= |n_i - n_c|
// keeps d2[i] = min(d2[i], D2(i, c)) whatever its overlap; its ov stays 0, and
// the update's n_i + n_c - 2 ov >= d2[i] leaves d2[i] as it is.
constexpr int kSeedChunk = 1024;   // CSC entries per pull chunk (32 per lane)

// pull_work: estimated push entries above which a centre is pulled (< 0: never)
__device__ __forceinline__ bool seed_pulls(int64_t nc, int64_t N, int64_t nnz, double pull_work) {
  return pull_work >= 0.0 && (double)nc * (double)nnz > pull_work * (double)N;
}

// Frequent features (at least kHotMin and N/128 rows; at most kHotBins of them)
// get a bin of a per-block shared histogram in the push form of the overlap
// pass: most rows of a centre hold many of them, and counting them in shared
// memory first keeps those increments off a few global addresses.
constexpr int kHotBins = 2048;
constexpr int64_t kHotMin = 64;

__global__ void k_hot_assign(int64_t F, int64_t N, const int64_t *__restrict__ col_ptr,
                             uint16_t *__restrict__ hot, int32_t *__restrict__ hot_col,
                             int32_t *__restrict__ hot_n) {
  const int64_t thr = max(kHotMin, N / 128);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint16_t bin = 0xFFFF;
    if (col_ptr[i + 1] - col_ptr[i] >= thr) {
      const int32_t s = atomicAdd(hot_n, 1);
      if (s < kHotBins) {
        bin = (uint16_t)s;
        hot_col[s] = (int32_t)i;
      }
    }
    hot[i] = bin;
  }
}

// Push: ov[j] += 1 for every feature j sharing a row with centre c, one row
// per warp. Integer counts, so the order of the increments does not matter.
// hist: kHotBins shared ints.
__device__ __forceinline__ void seed_overlap_push(int64_t c, const int64_t *__restrict__ row_ptr,
                                                  const int32_t *__restrict__ col_idx,
                                                  const int64_t *__restrict__ col_ptr,
                                                  const int32_t *__restrict__ row_idx,
                                                  const uint16_t *__restrict__ hot,
                                                  const int32_t *__restrict__ hot_col, int32_t nh,
                                                  int32_t *ov, int32_t *hist) {
  for (int s = threadIdx.x; s < kHotBins; s += blockDim.x) hist[s] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = col_ptr[c] + warp; p < col_ptr[c + 1]; p += nwarps) {
    const int64_t r = row_idx[p];
    const int64_t e1 = row_ptr[r + 1];
    // eight entries per lane at a time: their index and bin loads in flight together
    for (int64_t e0 = row_ptr[r] + lane; e0 < e1; e0 += 32 * 8) {
      int32_t j[8];
      uint16_t bin[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) j[u] = e0 + 32 * u < e1 ? col_idx[e0 + 32 * u] : -1;
#pragma unroll
      for (int u = 0; u < 8; ++u) bin[u] = j[u] >= 0 ? hot[j[u]] : (uint16_t)0xFFFF;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (j[u] < 0) continue;
        if (bin[u] != 0xFFFF)
          atomicAdd(&hist[bin[u]], 1);
        else
          atomicAdd(&ov[j[u]], 1);
      }
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < nh; s += blockDim.x) {
    const int32_t v = hist[s];
    if (v) atomicAdd(&ov[hot_col[s]], v);
  }
}

// Pull: one listed chunk (feature, chunk number) per warp at a time; each lane
// loads 32 of the chunk's row indices together, then tests them in rowbits.
__device__ __forceinline__ void seed_overlap_pull(const int64_t *__restrict__ col_ptr,
                                                  const int32_t *__restrict__ row_idx,
                                                  const uint32_t *__restrict__ rowbits,
                                                  const int2 *__restrict__ tasks, int32_t ntasks,
                                                  int32_t *ov) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t q = warp; q < ntasks; q += nwarps) {
    const int2 tk = tasks[q];
    const int64_t e = col_ptr[tk.x + 1];
    const int64_t s = col_ptr[tk.x] + (int64_t)tk.y * kSeedChunk + lane;
    int32_t r[kSeedChunk / 32];
#pragma unroll
    for (int u = 0; u < kSeedChunk / 32; ++u)
      r[u] = s + 32 * u < e ? __ldg(&row_idx[s + 32 * u]) : -1;
    uint32_t cnt = 0;
#pragma unroll
    for (int u = 0; u < kSeedChunk / 32; ++u)
      if (r[u] >= 0) cnt += (__ldg(&rowbits[r[u] >> 5]) >> (r[u] & 31)) & 1u;
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (lane == 0 && cnt) atomicAdd(&ov[tk.x], (int32_t)cnt);
  }
}

__global__ void __launch_bounds__(kThreads) k_seed_overlap(
    int32_t t, const int32_t *__restrict__ centers, int64_t N, int64_t nnz, double pull_work,
    const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
    const int64_t *__restrict__ col_ptr, const int32_t *__restrict__ row_idx,
    const uint32_t *__restrict__ rowbits, const int2 *__restrict__ tasks,
    const int32_t *__restrict__ ntasks, const uint16_t *__restrict__ hot,
    const int32_t *__restrict__ hot_col, const int32_t *__restrict__ hot_n,
    int32_t *__restrict__ ov) {
  __shared__ int32_t hist[kHotBins];
  pdl_wait();
  const int64_t c = centers[t];
  if (c < 0) return;
  const int64_t nc = col_ptr[c + 1] - col_ptr[c];
  if (seed_pulls(nc, N, nnz, pull_work)) {
    seed_overlap_pull(col_ptr, row_idx, rowbits, tasks, *ntasks, ov);
    return;
  }
  // a pushed centre's rows go one per warp: blocks past them have nothing to count
  if ((int64_t)blockIdx.x * (blockDim.x >> 5) >= nc) return;
  seed_overlap_push(c, row_ptr, col_idx, col_ptr, row_idx, hot, hot_col, min(*hot_n, kHotBins),
                    ov, hist);
}

// d2[i] = min(d2[i], n_i + n_c - 2 ov[i]) (plain assignment for the first centre);
// near[i] = t when centre t is strictly nearer than every earlier one (so the
// nearest centre with ties to the earliest); ov reset; tile_sum[tile] = sum of
// the tile's d2 (tiles of kTile features).
__device__ __forceinline__ void seed_update_tile(int32_t t, int64_t tile, int64_t F, int64_t nc,
                                                 const int64_t *__restrict__ col_ptr, int32_t *ov,
                                                 int64_t *d2, int32_t *near, int64_t *tile_sum,
                                                 int64_t *sm) {
  int64_t s = 0;
  const int64_t i = tile * kTile + threadIdx.x;
  if (i < F) {
    const int64_t ni = col_ptr[i + 1] - col_ptr[i];
    const int64_t dist = ni + nc - 2 * (int64_t)__ldcg(&ov[i]);
    ov[i] = 0;
    const int64_t old = t == 0 ? 0 : __ldcg(&d2[i]);
    const int64_t v = (t == 0) ? dist : min(old, dist);
    d2[i] = v;
    if (t == 0 || dist < old) near[i] = t;
    s = v;
  }
  s = block_sum_i64(s, sm);
  if (threadIdx.x == 0) tile_sum[tile] = s;
}

// Round t's distance update; also marks centre t chosen, empties the pull list
// and, after a pull, clears the row bitmap for the next round.
__global__ void __launch_bounds__(kThreads) k_seed_update(
    int32_t t, int64_t F, int64_t N, int64_t nnz, double pull_work,
    const int32_t *__restrict__ centers,
    const int64_t *__restrict__ col_ptr, int32_t *__restrict__ ov, int64_t *__restrict__ d2,
    int32_t *__restrict__ near, int64_t *__restrict__ tile_sum, uint8_t *__restrict__ chosen,
    uint32_t *__restrict__ rowbits, int32_t *__restrict__ ntasks) {
  pdl_wait();
  __shared__ int64_t sm[kWarps + 1];
  const int64_t c = centers[t];
  if (c < 0) return;
  const int64_t nc = col_ptr[c + 1] - col_ptr[c];
  seed_update_tile(t, blockIdx.x, F, nc, col_ptr, ov, d2, near, tile_sum, sm);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    chosen[c] = 1;
    *ntasks = 0;
  }
  if (seed_pulls(nc, N, nnz, pull_work))
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < (N + 31) / 32;
         w += (int64_t)gridDim.x * blockDim.x)
      rowbits[w] = 0;
}

// Draws centre t (1 <= t < k) from d2, the tile sums and chosen[] (whole
// block, reads only) and returns it to every thread of the block.
__device__ int64_t seed_pick(int32_t t, int64_t F, int64_t ntiles, uint64_t seed, const int64_t *d2,
                             const int64_t *tile_sum, const uint8_t *chosen, int64_t *sm) {
  __shared__ int64_t found;
  __shared__ int64_t tile_found, tile_base;
  int64_t s = 0;
  for (int64_t b = threadIdx.x; b < ntiles; b += kThreads) s += __ldcg(&tile_sum[b]);
  const int64_t total = block_sum_i64(s, sm);
  if (threadIdx.x == 0) found = -1;
  __syncthreads();
  if (total == 0) {
    // every remaining distance is zero: lowest index not chosen yet
    for (int64_t base = 0; base < F; base += kThreads) {
      int64_t i = base + threadIdx.x;
      int64_t cand = (i < F && !chosen[i]) ? i : INT64_MAX;
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
    if (threadIdx.x == 0) tile_found = -1;
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < ntiles; b0 += kThreads) {
      const int64_t b = b0 + threadIdx.x;
      const int64_t v = b < ntiles ? __ldcg(&tile_sum[b]) : 0;
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
      const int64_t v = i < F ? __ldcg(&d2[i]) : 0;
      int64_t tot;
      const int64_t inc = block_incl_scan_i64(v, sm, &tot);
      if (i < F && run + inc > thr && run + inc - v <= thr) found = i;
      __syncthreads();
      run += tot;
      if (found >= 0) break;
    }
  }
  __syncthreads();
  return found;
}

// Round t, every block: the block draws centre t itself (floor(u_0 F) at
// t = 0; the same inputs and integer arithmetic give every block the same
// centre) and block 0 stores it. When the centre's overlaps are to be pulled,
// the grid sets its rows in rowbits and lists the chunks of every feature whose
// distance can still drop (every feature at t = 0) in tasks[0 .. *ntasks).
__global__ void __launch_bounds__(kThreads) k_seed_pick(
    int32_t t, int64_t F, int64_t N, int64_t nnz, double pull_work, int64_t ntiles, uint64_t seed,
    const int64_t *__restrict__ d2, const int64_t *__restrict__ tile_sum,
    const uint8_t *__restrict__ chosen, const int64_t *__restrict__ col_ptr,
    const int32_t *__restrict__ row_idx, int32_t *__restrict__ centers,
    uint32_t *__restrict__ rowbits, int2 *__restrict__ tasks, int32_t *__restrict__ ntasks) {
  pdl_wait();
  __shared__ int64_t sm[kWarps + 1];
  __shared__ int32_t base;
  int64_t c;
  if (t == 0) {
    c = (int64_t)floor(uniform53(seed, 0) * (double)F);
    if (c >= F) c = F - 1;
  } else {
    c = seed_pick(t, F, ntiles, seed, d2, tile_sum, chosen, sm);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) centers[t] = (int32_t)c;
  if (c < 0) return;   // block-uniform: every feature chosen already (k > F)
  const int64_t nc = col_ptr[c + 1] - col_ptr[c];
  if (!seed_pulls(nc, N, nnz, pull_work)) return;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = col_ptr[c] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < col_ptr[c + 1];
       p += nthr) {
    const int32_t r = row_idx[p];
    atomicOr(&rowbits[r >> 5], 1u << (r & 31));
  }
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < F; i0 += nthr) {
    const int64_t i = i0 + threadIdx.x;
    int64_t nch = 0;
    if (i < F) {
      const int64_t ni = col_ptr[i + 1] - col_ptr[i];
      if (ni > 0 && (t == 0 || __ldcg(&d2[i]) > (ni > nc ? ni - nc : nc - ni)))
        nch = (ni + kSeedChunk - 1) / kSeedChunk;
    }
    int64_t tot;
    const int64_t inc = block_incl_scan_i64(nch, sm, &tot);
    if (threadIdx.x == 0 && tot > 0) base = atomicAdd(ntasks, (int32_t)tot);
    __syncthreads();
    for (int64_t q = 0; q < nch; ++q)
      tasks[base + inc - nch + q] = make_int2((int32_t)i, (int32_t)q);
    __syncthreads();
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

// work_i = sum of the row lengths over the rows of column i (the cost of D_i.)
// work[i] = sum over the rows of column i of their lengths (= (|X|^T |X| 1)_i):
// one block per column, so the longest columns do not serialise on one warp.
__global__ void __launch_bounds__(kThreads) k_feature_work(int64_t F,
                                                          const int64_t *__restrict__ row_ptr,
                                                          const int64_t *__restrict__ col_ptr,
                                                          const int32_t *__restrict__ row_idx,
                                                          int64_t *__restrict__ work) {
  __shared__ int64_t sm[kWarps + 1];
  for (int64_t i = blockIdx.x; i < F; i += gridDim.x) {
    int64_t s = 0;
    for (int64_t p = col_ptr[i] + threadIdx.x; p < col_ptr[i + 1]; p += kThreads) {
      const int64_t r = row_idx[p];
      s += row_ptr[r + 1] - row_ptr[r];
    }
    s = block_sum_i64(s, sm);
    if (threadIdx.x == 0) work[i] = s;
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

// Lloyd steps keep D[i, S] = x_i . c_S (integer) resident and update it only
// through the features whose label changed since the previous step:
//   D[i, new_j] += |x_i AND x_j|,  D[i, old_j] -= |x_i AND x_j|  for each moved j.
// The entries of X that belong to moved features are first compacted row by
// row into (old+1, new) pairs; then every feature accumulates, in a shared
// histogram over clusters, the pairs of all rows of its column. Exact integer
// arithmetic: the result equals a full recomputation.

// (cluster, delta) entries of the row delta lists: int2, or 32 bits (cluster
// in the low 16, delta as int16 in the high 16) when k < 65535 and no row has
// more than 32767 entries, so that every |delta| fits. The packed form halves
// the bytes the pull re-reads.
template <bool P> struct DeltaEntry;
template <> struct DeltaEntry<false> {
  using T = int2;
  __device__ static T make(int32_t s, int32_t d) { return make_int2(s, d); }
  __device__ static T none() { return make_int2(-1, 0); }
  __device__ static int32_t cluster(T e) { return e.x; }
  __device__ static int32_t delta(T e) { return e.y; }
};
template <> struct DeltaEntry<true> {
  using T = uint32_t;
  __device__ static T make(int32_t s, int32_t d) {
    return (uint32_t)(uint16_t)s | ((uint32_t)(uint16_t)(int16_t)d << 16);
  }
  __device__ static T none() { return 0xFFFFFFFFu; }
  __device__ static int32_t cluster(T e) {
    const int32_t s = (int32_t)(e & 0xFFFFu);
    return s == 0xFFFF ? -1 : s;
  }
  __device__ static int32_t delta(T e) { return (int32_t)(int16_t)(e >> 16); }
};

__global__ void k_max_row(int64_t N, const int64_t *__restrict__ row_ptr,
                          unsigned long long *__restrict__ mx) {
  unsigned long long m = 0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N;
       r += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (unsigned long long)(row_ptr[r + 1] - row_ptr[r]));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(mx, m);
}

// per row: number of entries whose feature moved
// the moved features' columns hold few entries (sw[0] of them): rows are found
// through those columns instead of a scan of every row
__device__ __forceinline__ bool moved_sparse(const unsigned long long *sw, int64_t nnz) {
  return *sw * 8ull < (unsigned long long)nnz;
}

__global__ void k_moved_count(int64_t N, const int64_t *__restrict__ row_ptr,
                              const int32_t *__restrict__ col_idx, const int32_t *__restrict__ prev,
                              const int32_t *__restrict__ cur, int64_t *__restrict__ cnt,
                              int64_t nnz, const unsigned long long *__restrict__ sw) {
  if (sw && moved_sparse(sw, nnz)) return;   // the scatter filled cnt
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < N; r += nwarps) {
    int c = 0;
    const int64_t e1 = row_ptr[r + 1];
    for (int64_t e0 = row_ptr[r] + lane; e0 < e1; e0 += 32 * 8) {
      int32_t j[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) j[u] = e0 + 32 * u < e1 ? col_idx[e0 + 32 * u] : -1;
#pragma unroll
      for (int u = 0; u < 8; ++u) c += j[u] >= 0 && prev[j[u]] != cur[j[u]];
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[r] = 2 * (int64_t)c;   // room for one (new) and one (old) pair each
  }
}

// A step that moved features holding few entries in all finds the rows holding
// them through their columns instead of scanning every row. The choice is made
// on the device: sw[0] = the moved features' entries; the scatter runs when
// 8 sw[0] < nnz, the full scan otherwise (each kernel returns at once when the
// other one is chosen).
// moved[0 .. n[0]) = the features whose label changed (one atomic per warp).
__global__ void k_moved_list(int64_t F, const int64_t *__restrict__ col_ptr,
                             const int32_t *__restrict__ prev, const int32_t *__restrict__ cur,
                             int32_t *__restrict__ moved, int32_t *__restrict__ n,
                             unsigned long long *__restrict__ sw) {
  const int lane = threadIdx.x & 31;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < F; i0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = i0 + threadIdx.x;
    const bool m = i < F && prev[i] != cur[i];
    const uint32_t bal = __ballot_sync(0xffffffffu, m);
    unsigned long long e = m ? (unsigned long long)(col_ptr[i + 1] - col_ptr[i]) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    int32_t base = 0;
    if (lane == 0 && bal) {
      base = atomicAdd(n, __popc(bal));
      atomicAdd(sw, e);
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    if (m) moved[base + __popc(bal & ((1u << lane) - 1u))] = (int32_t)i;
  }
}

// cnt[r] += 2 for every moved feature of row r (cnt zeroed before): one moved
// feature per warp over its column, eight entries per lane in flight, the
// increments without return values.
__global__ void k_moved_rows(int64_t nnz, const unsigned long long *__restrict__ sw,
                             const int32_t *__restrict__ moved, const int32_t *__restrict__ n,
                             const int64_t *__restrict__ col_ptr,
                             const int32_t *__restrict__ row_idx,
                             unsigned long long *__restrict__ cnt) {
  if (!moved_sparse(sw, nnz)) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int32_t nm = n[0];
  for (int64_t q = warp; q < nm; q += nwarps) {
    const int32_t j = moved[q];
    const int64_t e1 = col_ptr[j + 1];
    for (int64_t e0 = col_ptr[j] + lane; e0 < e1; e0 += 32 * 8) {
      int32_t r[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) r[u] = e0 + 32 * u < e1 ? row_idx[e0 + 32 * u] : -1;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (r[u] >= 0) atomicAdd(&cnt[r[u]], 2ull);
    }
  }
}

// rows[0 .. n[1]) = the rows with cnt[r] > 0 after a scatter; n[1] = -1 (every
// row) after a full scan.
__global__ void k_touched_rows(int64_t N, int64_t nnz, const unsigned long long *__restrict__ sw,
                               const int64_t *__restrict__ cnt, int32_t *__restrict__ rows,
                               int32_t *__restrict__ n) {
  if (!moved_sparse(sw, nnz)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) n[1] = -1;
    return;
  }
  const int lane = threadIdx.x & 31;
  for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x; r0 < N; r0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = r0 + threadIdx.x;
    const bool m = r < N && cnt[r] > 0;
    const uint32_t bal = __ballot_sync(0xffffffffu, m);
    int32_t base = 0;
    if (lane == 0 && bal) base = atomicAdd(&n[1], __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (m) rows[base + __popc(bal & ((1u << lane) - 1u))] = (int32_t)r;
  }
}

// per row r: the net change of the row's cluster counts C[r, .] between the
// previous and the current labels, as a list of distinct (cluster, delta)
// pairs (delta != 0). A warp owns a row and a private shared histogram over
// the clusters: moved entries add +1 at their new and -1 at their old
// cluster; then each nonzero bin is claimed once (atomicExch back to zero,
// which also leaves the histogram clean for the next row).
// *work += sum over rows of rownnz_r * |list_r| (the cost of applying them).
template <bool P>
__global__ void k_row_delta(int64_t N, int32_t k, const int64_t *__restrict__ row_ptr,
                            const int32_t *__restrict__ col_idx, const int32_t *__restrict__ prev,
                            const int32_t *__restrict__ cur, const int64_t *__restrict__ dptr,
                            typename DeltaEntry<P>::T *__restrict__ dlist,
                            int32_t *__restrict__ dcount, unsigned long long *__restrict__ work,
                            const int32_t *__restrict__ rows, const int32_t *__restrict__ nrows) {
  using E = DeltaEntry<P>;
  extern __shared__ int32_t hist_all[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t *hist = hist_all + (int64_t)wib * k;
  for (int s = lane; s < k; s += 32) hist[s] = 0;
  __syncwarp();
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long my_work = 0;
  // every row, or only the listed ones (the others' dcount is zero already)
  const bool listed = rows && *nrows >= 0;
  const int64_t nr = listed ? (int64_t)*nrows : N;
  for (int64_t q = warp; q < nr; q += nwarps) {
    const int64_t r = listed ? (int64_t)rows[q] : q;
    const int64_t b = row_ptr[r], e1 = row_ptr[r + 1];
    if (dptr[r + 1] == dptr[r]) {      // no moved entry in this row
      if (lane == 0) dcount[r] = 0;
      continue;
    }
    int64_t out = dptr[r];
    if (e1 - b <= 32 * 8) {
      // the whole row in registers: eight entries per lane, loads in flight together
      int32_t o[8], n[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t e = b + lane + 32 * u;
        const int32_t j = e < e1 ? col_idx[e] : -1;
        o[u] = j >= 0 ? prev[j] : -1;
        n[u] = j >= 0 ? cur[j] : -1;
        if (o[u] == n[u]) o[u] = n[u] = -1;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (n[u] >= 0) {
          atomicAdd(&hist[n[u]], 1);
          if (o[u] >= 0) atomicSub(&hist[o[u]], 1);
        }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int32_t vn = n[u] >= 0 ? atomicExch(&hist[n[u]], 0) : 0;
        const unsigned mn = __ballot_sync(0xffffffffu, vn != 0);
        if (vn != 0) dlist[out + __popc(mn & ((1u << lane) - 1u))] = E::make(n[u], vn);
        out += __popc(mn);
        const int32_t vo = o[u] >= 0 ? atomicExch(&hist[o[u]], 0) : 0;
        const unsigned mo = __ballot_sync(0xffffffffu, vo != 0);
        if (vo != 0) dlist[out + __popc(mo & ((1u << lane) - 1u))] = E::make(o[u], vo);
        out += __popc(mo);
      }
      __syncwarp();
      const int32_t cnt = (int32_t)(out - dptr[r]);
      if (lane == 0) dcount[r] = cnt;
      my_work += (unsigned long long)(e1 - b) * (unsigned long long)cnt;
      continue;
    }
    for (int64_t e = b + lane; e < e1; e += 32) {
      const int32_t j = col_idx[e];
      const int32_t o = prev[j], n = cur[j];
      if (o != n) {
        atomicAdd(&hist[n], 1);
        if (o >= 0) atomicSub(&hist[o], 1);
      }
    }
    __syncwarp();
    for (int64_t e0 = b; e0 < e1; e0 += 32) {
      const int64_t e = e0 + lane;
      int32_t o = -1, n = -1;
      if (e < e1) {
        const int32_t j = col_idx[e];
        o = prev[j];
        n = cur[j];
        if (o == n) o = n = -1;
      }
      const int32_t vn = n >= 0 ? atomicExch(&hist[n], 0) : 0;
      const unsigned mn = __ballot_sync(0xffffffffu, vn != 0);
      if (vn != 0) dlist[out + __popc(mn & ((1u << lane) - 1u))] = E::make(n, vn);
      out += __popc(mn);
      const int32_t vo = o >= 0 ? atomicExch(&hist[o], 0) : 0;
      const unsigned mo = __ballot_sync(0xffffffffu, vo != 0);
      if (vo != 0) dlist[out + __popc(mo & ((1u << lane) - 1u))] = E::make(o, vo);
      out += __popc(mo);
    }
    __syncwarp();
    const int32_t cnt = (int32_t)(out - dptr[r]);
    if (lane == 0) dcount[r] = cnt;
    my_work += (unsigned long long)(e1 - b) * (unsigned long long)cnt;
  }
  if (lane == 0 && my_work) atomicAdd(work, my_work);
}

// Pull: D[i, .] += sum over the rows of column i of their delta lists.
// Tasks are chunks of at most kPullRows rows of one column, features
// heaviest first (task_ptr / task_it built once per setup); persistent blocks
// take tasks from a shared counter and gather into a shared histogram
// (distinct clusters within a row, so no two lanes of one instruction hit the
// same bin). A column cut into several chunks adds its sums with integer
// atomics (exact, so the order does not matter); a one-chunk column is the
// only writer of its D row.
constexpr int64_t kPullRows = 1024;

template <bool P>
__global__ void __launch_bounds__(kThreads) k_lloyd_pull(
    int32_t k, const int64_t *__restrict__ col_ptr, const int32_t *__restrict__ row_idx,
    const int64_t *__restrict__ dptr, const int32_t *__restrict__ dcount,
    const typename DeltaEntry<P>::T *__restrict__ dlist, const int32_t *__restrict__ order,
    const int64_t *__restrict__ task_ptr, const int32_t *__restrict__ task_it, int64_t n_tasks,
    int32_t *work_ctr, int32_t *__restrict__ D, const unsigned long long *__restrict__ work,
    unsigned long long pull_work) {
  using E = DeltaEntry<P>;
  using T = typename E::T;
  if (*work <= pull_work) return;   // the push form applies this step's lists
  extern __shared__ int32_t acc[];
  __shared__ int32_t cur;
  __shared__ int32_t touched;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) {
      cur = atomicAdd(work_ctr, 1);
      touched = 0;
    }
    for (int s = threadIdx.x; s < k; s += kThreads) acc[s] = 0;
    __syncthreads();
    const int64_t t = cur;
    if (t >= n_tasks) break;
    const int32_t it = task_it[t];
    const int64_t i = order[it];
    const int64_t chunk = t - task_ptr[it];
    const bool shared_row = task_ptr[it + 1] - task_ptr[it] > 1;
    const int64_t pb = col_ptr[i] + chunk * kPullRows;
    const int64_t p1 = min(col_ptr[i + 1], pb + kPullRows);
    int any = 0;
    // two rows per warp at a time, eight list entries per lane at a time: the
    // loads of a batch are in flight together before its shared atomics
    for (int64_t p = pb + warp; p < p1; p += 2 * kWarps) {
      int32_t c[2];
      const T *lst[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t ph = p + h * kWarps;
        const int64_t r = ph < p1 ? row_idx[ph] : -1;
        c[h] = r >= 0 ? dcount[r] : 0;
        lst[h] = dlist + (r >= 0 ? dptr[r] : 0);
      }
      if (c[0] | c[1]) any = 1;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        for (int32_t q0 = lane; q0 < c[h]; q0 += 32 * 8) {
          T pr[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            pr[u] = q0 + 32 * u < c[h] ? lst[h][q0 + 32 * u] : E::none();
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int32_t sc = E::cluster(pr[u]);
            if (sc >= 0) atomicAdd(&acc[sc], E::delta(pr[u]));
          }
        }
      }
    }
    if (any) touched = 1;   // benign race: every writer stores 1
    __syncthreads();
    if (touched) {
      int32_t *Di = D + i * (int64_t)k;
      for (int s = threadIdx.x; s < k; s += kThreads) {
        const int32_t a = acc[s];
        if (a) {
          if (shared_row)
            atomicAdd(&Di[s], a);
          else
            Di[s] += a;
        }
      }
    }
    __syncthreads();
  }
}

// task_ptr[it] = first pull task of the it-th feature in work order
// (ceil(n_i / kPullRows) tasks each, at least one); task_it[t] = it.
__global__ void k_task_count(int64_t F, const int32_t *__restrict__ order,
                             const int64_t *__restrict__ col_ptr, int64_t *__restrict__ cnt) {
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < F;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = order[it];
    const int64_t n = col_ptr[i + 1] - col_ptr[i];
    cnt[it] = n <= kPullRows ? 1 : (n + kPullRows - 1) / kPullRows;
  }
}
__global__ void k_task_fill(int64_t F, const int64_t *__restrict__ task_ptr,
                            int32_t *__restrict__ task_it) {
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < F;
       it += (int64_t)gridDim.x * blockDim.x)
    for (int64_t t = task_ptr[it]; t < task_ptr[it + 1]; ++t) task_it[t] = (int32_t)it;
}

// Push: for every row with a delta list, D[i, S] += delta for each feature i of
// the row and each (S, delta) of the list (global atomics; used when few
// labels moved, so only a few rows carry work).
template <bool P>
__global__ void k_lloyd_push(int64_t N, int32_t k, const int64_t *__restrict__ row_ptr,
                             const int32_t *__restrict__ col_idx, const int64_t *__restrict__ dptr,
                             const int32_t *__restrict__ dcount,
                             const typename DeltaEntry<P>::T *__restrict__ dlist,
                             int32_t *__restrict__ D, const int32_t *__restrict__ rows,
                             const int32_t *__restrict__ nrows,
                             const unsigned long long *__restrict__ work,
                             unsigned long long pull_work) {
  using E = DeltaEntry<P>;
  const unsigned long long wk = *work;
  if (wk == 0 || wk > pull_work) return;   // nothing to apply, or the pull form does it
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool listed = rows && *nrows >= 0;
  const int64_t nr = listed ? (int64_t)*nrows : N;
  for (int64_t q = warp; q < nr; q += nwarps) {
    const int64_t r = listed ? (int64_t)rows[q] : q;
    const int32_t c = dcount[r];
    if (c == 0) continue;
    const typename E::T *lst = dlist + dptr[r];
    for (int64_t e = row_ptr[r] + lane; e < row_ptr[r + 1]; e += 32) {
      int32_t *Di = D + (int64_t)col_idx[e] * k;
      for (int32_t q = 0; q < c; ++q) {
        const typename E::T pr = lst[q];
        atomicAdd(&Di[E::cluster(pr)], E::delta(pr));
      }
    }
  }
}

// Q_S = ||c_S||^2 = sum over members i of S of D[i, S]; n_S = |S|.
__global__ void k_q_sizes(int64_t F, int32_t k, const int32_t *__restrict__ labels,
                          const int32_t *__restrict__ D, unsigned long long *__restrict__ Q,
                          unsigned long long *__restrict__ n_S) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t l = labels[i];
    if (l >= 0) {
      atomicAdd(&Q[l], (unsigned long long)D[i * (int64_t)k + l]);
      atomicAdd(&n_S[l], 1ULL);
    }
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

// FP32 approximations of the score's two terms per cluster S,
//   q_S ~ Q_S / n_S^2,  r_S ~ 2 / n_S,  score(i, S) ~ q_S - r_S D_iS,
// used only to skip clusters that cannot win (q_S = +inf for an empty one).
// Each of Q_S, n_S^2, D_iS rounds once to FP32 and each operation adds one
// rounding, so |computed - exact| <= 6 u (Q_S / n_S^2 + 2 D_iS / n_S) + O(u^2)
// with u = 2^-24; kScoreTol = 2^-20 = 16 u covers that and the roundings of the
// bounds themselves.
constexpr float kScoreTol = 0x1.0p-20f;
constexpr int kArgminBatch = 8;

__global__ void k_score_terms(int32_t k, const unsigned long long *__restrict__ Q,
                              const unsigned long long *__restrict__ n_S, float2 *__restrict__ qr) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= k) return;
  const unsigned long long n = n_S[s];
  const float nf = (float)n;
  qr[s] = n == 0 ? make_float2(INFINITY, 0.f) : make_float2((float)Q[s] / (nf * nf), 2.f / nf);
}

// One warp per feature: next[i] = argmin_S score(i, S); counts changed labels.
// The warp visits the clusters in batches of 32 x kArgminBatch and keeps U, the
// least upper bound (approximate score + its error bound) of every cluster
// seen so far, so U >= the exact score of the best of them. A cluster whose
// lower bound (approximate score - error bound) exceeds U is strictly worse
// than that one and is skipped (an empty cluster gives NaN and is skipped
// too); the others, usually only the batch's best, are compared exactly and
// kept per lane (clusters in increasing S). The exact argmin, ties to the
// smallest S, is never skipped, so the result is exact whatever the filter
// skips; a bound shared by the warp keeps the exact path off most batches.
__global__ void k_lloyd_argmin(int64_t F, int32_t k, const int32_t *__restrict__ D,
                               const unsigned long long *__restrict__ Q,
                               const unsigned long long *__restrict__ n_S,
                               const float2 *__restrict__ qr,
                               const int32_t *__restrict__ labels, int32_t *__restrict__ next,
                               unsigned long long *changes) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long changed = 0;
  for (int64_t i = warp; i < F; i += nwarps) {
    const int32_t *Di = D + i * (int64_t)k;
    Cand best{0, 0, INT32_MAX};
    float U = INFINITY;
    // eight clusters per lane at a time: their D and table loads in flight together
    for (int s0 = lane; s0 - lane < k; s0 += 32 * kArgminBatch) {   // warp-uniform
      int32_t d[kArgminBatch];
      float2 t[kArgminBatch];
#pragma unroll
      for (int u = 0; u < kArgminBatch; ++u) {
        const int s = s0 + 32 * u;
        d[u] = s < k ? __ldg(&Di[s]) : 0;
        t[u] = s < k ? __ldg(&qr[s]) : make_float2(INFINITY, 0.f);
      }
      float lo[kArgminBatch], hi = INFINITY;
#pragma unroll
      for (int u = 0; u < kArgminBatch; ++u) {
        const float df = (float)d[u];
        const float sc = fmaf(-t[u].y, df, t[u].x);
        const float m = fmaf(t[u].y, df, t[u].x);
        lo[u] = fmaf(-kScoreTol, m, sc);
        hi = fminf(hi, fmaf(kScoreTol, m, sc));   // fminf drops the NaN of an empty cluster
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) hi = fminf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      U = fminf(U, hi);
#pragma unroll
      for (int u = 0; u < kArgminBatch; ++u) {
        if (!(lo[u] <= U)) continue;
        const int s = s0 + 32 * u;
        const int64_t n = (int64_t)n_S[s];
        if (n == 0) continue;
        Cand c{(int64_t)Q[s] - 2 * n * (int64_t)d[u], n * n, s};
        if (better(c, best)) best = c;
      }
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

// The k rounds, issued from the host as three kernels each (draw of centre t
// with the pull list, overlaps with it, distance update), chained by
// programmatic dependent launch: each kernel's launch overlaps the previous
// one's tail, and no host synchronisation comes between rounds. The row bitmap
// and the pull list live in buffers the Lloyd steps fill only later. The last
// round's distances are computed too: prev[] ends holding every feature's
// nearest centre (ties to the earliest), the first Lloyd assignment.
rr_status kmeanspp_seed(int64_t N, int64_t F, int64_t nnz, const int64_t *row_ptr,
                        const int32_t *col_idx, const int64_t *col_ptr, const int32_t *row_idx,
                        int32_t k, uint64_t seed, int64_t pull_work, KmeansBuffers &b,
                        cudaStream_t st) {
  const int64_t ntiles = (F + kTile - 1) / kTile;
  const double pw = pull_work > 0 ? (double)pull_work : pull_work < 0 ? -1.0 : kSeedPullWork;
  uint8_t *chosen = reinterpret_cast<uint8_t *>(b.next);       // F bytes
  uint32_t *rowbits = reinterpret_cast<uint32_t *>(b.mcount);  // ceil(N/32) words of N int64
  int2 *tasks = b.dlist;     // sum over features of ceil(n_i / kSeedChunk) <= 2 nnz entries
  int32_t *ntasks = b.work_ctr;
  RR_CUDA(cudaMemsetAsync(chosen, 0, F, st));
  RR_CUDA(cudaMemsetAsync(b.ov, 0, sizeof(int32_t) * F, st));
  RR_CUDA(cudaMemsetAsync(rowbits, 0, sizeof(uint32_t) * ((N + 31) / 32), st));
  RR_CUDA(cudaMemsetAsync(ntasks, 0, sizeof(int32_t), st));
  RR_CUDA(cudaMemsetAsync(b.hot_n, 0, sizeof(int32_t), st));
  RR_LAUNCH(k_hot_assign, grid_for(F, kThreads), kThreads, 0, st, F, N, col_ptr, b.hot, b.hot_col,
            b.hot_n);
  for (int32_t t = 0; t < k; ++t) {
    RR_LAUNCH_PDL(k_seed_pick, kSMs * 2, kThreads, 0, st, t, F, N, nnz, pw, ntiles, seed, b.d2,
                  b.part_i, chosen, col_ptr, row_idx, b.centers, rowbits, tasks, ntasks);
    RR_LAUNCH_PDL(k_seed_overlap, kSMs * 2, kThreads, 0, st, t, b.centers, N, nnz, pw, row_ptr,
                  col_idx, col_ptr, row_idx, rowbits, tasks, ntasks, b.hot, b.hot_col, b.hot_n,
                  b.ov);
    RR_LAUNCH_PDL(k_seed_update, (unsigned)ntiles, kThreads, 0, st, t, F, N, nnz, pw, b.centers,
                  col_ptr, b.ov, b.d2, b.prev, b.part_i, chosen, rowbits, ntasks);
  }
  RR_CUDA(cudaStreamSynchronize(st));
  return RR_OK;
}

int64_t kmeans_seed_tiles(int64_t F) { return (F + kTile - 1) / kTile; }

int64_t kmeans_pull_tasks_max(int64_t F, int64_t nnz) { return F + nnz / kPullRows + 1; }

// The first Lloyd step from singleton clusters {c_S}: score(i, S) =
// n_{c_S} - 2 |x_i AND x_{c_S}| = D2(i, c_S) - n_i, so its assignment is the
// nearest centre with ties to the smallest S, which the seeding left in prev[].
// labels <- prev[], the count of labels that differ from the singleton
// labelling (-1 but labels[centers[S]] = S) into *changes_host; prev <- -1 and
// D <- 0, so that the next step builds D from scratch for these labels.
__global__ void k_count_diff(int64_t F, const int32_t *__restrict__ a, const int32_t *__restrict__ b,
                             unsigned long long *__restrict__ n) {
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x)
    c += a[i] != b[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(n, c);
}

rr_status kmeans_seeded_labels(int64_t F, int32_t k, KmeansBuffers &b, int64_t *changes_host,
                               cudaStream_t st) {
  RR_LAUNCH(k_init_labels, grid_for(F, kThreads), kThreads, 0, st, F, k, b.centers, b.next);
  RR_LAUNCH(k_set_center_labels, grid_for(k, kThreads), kThreads, 0, st, k, b.centers, b.next);
  RR_CUDA(cudaMemsetAsync(b.changes, 0, sizeof(int64_t), st));
  RR_LAUNCH(k_count_diff, grid_for(F, kThreads), kThreads, 0, st, F, b.prev, b.next,
            (unsigned long long *)b.changes);
  RR_CUDA(cudaMemcpyAsync(b.labels, b.prev, sizeof(int32_t) * F, cudaMemcpyDeviceToDevice, st));
  RR_LAUNCH(k_init_labels, grid_for(F, kThreads), kThreads, 0, st, F, k, b.centers, b.prev);
  RR_CUDA(cudaMemsetAsync(b.D, 0, sizeof(int32_t) * (size_t)F * k, st));
  RR_CUDA(cudaMemcpyAsync(changes_host, b.changes, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  return RR_OK;
}

rr_status kmeans_init_labels(int64_t F, int32_t k, KmeansBuffers &b, cudaStream_t st) {
  RR_LAUNCH(k_init_labels, grid_for(F, kThreads), kThreads, 0, st, F, k, b.centers, b.prev);
  RR_LAUNCH(k_init_labels, grid_for(F, kThreads), kThreads, 0, st, F, k, b.centers, b.labels);
  RR_LAUNCH(k_set_center_labels, grid_for(k, kThreads), kThreads, 0, st, k, b.centers, b.labels);
  RR_CUDA(cudaMemsetAsync(b.D, 0, sizeof(int32_t) * (size_t)F * k, st));
  return RR_OK;
}

rr_status feature_work(int64_t F, const int64_t *row_ptr, const int64_t *col_ptr,
                       const int32_t *row_idx, int64_t *work, cudaStream_t st) {
  RR_LAUNCH(k_feature_work, (unsigned)std::min<int64_t>(std::max<int64_t>(F, 1), kSMs * 64), kThreads,
            0, st, F, row_ptr, col_ptr, row_idx, work);
  return RR_OK;
}

rr_status kmeans_work_order(int64_t N, int64_t F, int32_t k, const int64_t *row_ptr,
                            const int64_t *col_ptr, const int32_t *row_idx, KmeansBuffers &b,
                            int64_t *work, int64_t *scratch, cudaStream_t st) {
  // scratch: >= 2 * kBuckets + 1 + scan scratch int64
  int64_t *cnt = scratch;
  int64_t *offs = cnt + kBuckets;              // kBuckets + 1
  int64_t *sscr = offs + kBuckets + 1;
  RR_LAUNCH(k_feature_work, (unsigned)std::min<int64_t>(std::max<int64_t>(F, 1), kSMs * 64), kThreads,
            0, st, F, row_ptr, col_ptr, row_idx, work);
  RR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * kBuckets, st));
  RR_LAUNCH(k_bucket_count, grid_for(F, kThreads), kThreads, 0, st, F, work,
            (unsigned long long *)cnt);
  RR_TRY(scan_exclusive(cnt, offs, kBuckets, sscr, st));
  RR_LAUNCH(k_bucket_scatter, grid_for(F, kThreads), kThreads, 0, st, F, work,
            (unsigned long long *)offs, b.order);
  // pull tasks (chunks of kPullRows rows per feature, in work order)
  int64_t *tcnt = reinterpret_cast<int64_t *>(b.dlist);   // >= F int64 (dlist is rewritten per step)
  RR_LAUNCH(k_task_count, grid_for(F, kThreads), kThreads, 0, st, F, b.order, col_ptr, tcnt);
  RR_TRY(scan_exclusive(tcnt, b.task_ptr, F, sscr, st));
  RR_CUDA(cudaMemcpyAsync(&b.n_tasks, b.task_ptr + F, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  RR_LAUNCH(k_task_fill, grid_for(F, kThreads), kThreads, 0, st, F, b.task_ptr, b.task_it);
  // the packed delta-list form needs every |delta| <= 32767 (rows of <= 32767 entries)
  RR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int64_t), st));
  RR_LAUNCH(k_max_row, grid_for(N, kThreads), kThreads, 0, st, N, row_ptr,
            (unsigned long long *)cnt);
  int64_t mx = 0;
  RR_CUDA(cudaMemcpyAsync(&mx, cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  b.packed = (mx <= 32767 && k < 65535) ? 1 : 0;
  return RR_OK;
}

// Delta lists of the rows (prev -> labels), then D += delta: pull per feature
// when much changed, push per row otherwise.
template <bool P>
rr_status lloyd_delta_apply(int64_t N, int64_t F, const int64_t *row_ptr, const int32_t *col_idx,
                            const int64_t *col_ptr, const int32_t *row_idx, int32_t k,
                            KmeansBuffers &b, unsigned long long pull_work, const int32_t *rows,
                            const int32_t *nrows, cudaStream_t st) {
  using T = typename DeltaEntry<P>::T;
  T *dlist = reinterpret_cast<T *>(b.dlist);
  const int warps_per_cta = (int)std::max<int64_t>(1, std::min<int64_t>(kWarps, (96 * 1024) / (4 * (int64_t)k)));
  const size_t hsmem = sizeof(int32_t) * (size_t)k * warps_per_cta;
  RR_CUDA(cudaFuncSetAttribute(k_row_delta<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem));
  RR_LAUNCH(k_row_delta<P>, std::min<int64_t>((N + warps_per_cta - 1) / warps_per_cta, kSMs * 16),
            32 * warps_per_cta, hsmem, st, N, k, row_ptr, col_idx, b.prev, b.labels, b.mptr,
            dlist, b.dcount, (unsigned long long *)b.work, rows, nrows);
  // pull per feature when the lists' work exceeds pull_work, else push per
  // row: both launched, each kernel reads the work on the device and one
  // returns at once (no host round trip)
  const unsigned long long *wk = (const unsigned long long *)b.work;
  RR_CUDA(cudaMemsetAsync(b.work_ctr, 0, sizeof(int32_t), st));
  const size_t smem = sizeof(int32_t) * (size_t)k;
  RR_CUDA(cudaFuncSetAttribute(k_lloyd_pull<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)std::max<size_t>(smem, 1)));
  int per_sm = 0;
  RR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lloyd_pull<P>, kThreads, smem));
  RR_LAUNCH(k_lloyd_pull<P>, kSMs * std::max(1, per_sm), kThreads, smem, st, k, col_ptr,
            row_idx, b.mptr, b.dcount, dlist, b.order, b.task_ptr, b.task_it, b.n_tasks,
            b.work_ctr, b.D, wk, pull_work);
  RR_LAUNCH(k_lloyd_push<P>, grid_for(N, kWarps), kThreads, 0, st, N, k, row_ptr, col_idx,
            b.mptr, b.dcount, dlist, b.D, rows, nrows, wk, pull_work);
  return RR_OK;
}

rr_status kmeans_lloyd_step(int64_t N, int64_t F, int64_t nnz, const int64_t *row_ptr,
                            const int32_t *col_idx, const int64_t *col_ptr, const int32_t *row_idx,
                            int32_t k, KmeansBuffers &b, int64_t *changes_host, int64_t pull_work,
                            int64_t moved, cudaStream_t st) {
  const unsigned long long pw = pull_work > 0 ? (unsigned long long)pull_work : kPushWorkLimit;
  // (1) per-row delta lists of the cluster counts (prev -> labels), with
  // cnt[r] = 2 x the moved entries of row r: after the first step the moved
  // features are listed and, when their columns hold few entries, the rows
  // holding them are found through those columns and only they are visited
  // (chosen on the device); otherwise every row counts its moved entries.
  const int32_t *rows = nullptr, *nrows = nullptr;
  unsigned long long *sw = nullptr;
  if (moved >= 0) {
    sw = reinterpret_cast<unsigned long long *>(b.sparse_n + 2);
    RR_CUDA(cudaMemsetAsync(b.sparse_n, 0, 4 * sizeof(int32_t), st));
    RR_CUDA(cudaMemsetAsync(b.mcount, 0, sizeof(int64_t) * N, st));
    RR_CUDA(cudaMemsetAsync(b.dcount, 0, sizeof(int32_t) * N, st));
    RR_LAUNCH(k_moved_list, grid_for(F, kThreads), kThreads, 0, st, F, col_ptr, b.prev, b.labels,
              b.moved, b.sparse_n, sw);
    RR_LAUNCH(k_moved_rows, kSMs * 8, kThreads, 0, st, nnz, sw, b.moved, b.sparse_n, col_ptr,
              row_idx, (unsigned long long *)b.mcount);
    rows = b.touched;
    nrows = b.sparse_n + 1;
  }
  RR_LAUNCH(k_moved_count, grid_for(N, kWarps), kThreads, 0, st, N, row_ptr, col_idx, b.prev,
            b.labels, b.mcount, nnz, sw);
  if (sw)
    RR_LAUNCH(k_touched_rows, grid_for(N, kThreads), kThreads, 0, st, N, nnz, sw, b.mcount,
              b.touched, b.sparse_n);
  RR_TRY(scan_exclusive(b.mcount, b.mptr, N, b.scan_scratch, st));
  RR_CUDA(cudaMemsetAsync(b.work, 0, sizeof(unsigned long long), st));
  if (b.packed)
    RR_TRY(lloyd_delta_apply<true>(N, F, row_ptr, col_idx, col_ptr, row_idx, k, b, pw, rows, nrows,
                                   st));
  else
    RR_TRY(lloyd_delta_apply<false>(N, F, row_ptr, col_idx, col_ptr, row_idx, k, b, pw, rows,
                                    nrows, st));
  // (3) sizes and Q from the updated D
  RR_CUDA(cudaMemsetAsync(b.n_S, 0, sizeof(int64_t) * k, st));
  RR_CUDA(cudaMemsetAsync(b.Q, 0, sizeof(int64_t) * k, st));
  RR_LAUNCH(k_q_sizes, grid_for(F, kThreads), kThreads, 0, st, F, k, b.labels, b.D,
            (unsigned long long *)b.Q, (unsigned long long *)b.n_S);
  // (4) assignment
  RR_CUDA(cudaMemsetAsync(b.changes, 0, sizeof(int64_t), st));
  RR_LAUNCH(k_score_terms, grid_for(k, kThreads), kThreads, 0, st, k,
            (const unsigned long long *)b.Q, (const unsigned long long *)b.n_S, b.qr);
  RR_LAUNCH(k_lloyd_argmin, grid_for(F, kWarps), kThreads, 0, st, F, k, b.D,
            (const unsigned long long *)b.Q, (const unsigned long long *)b.n_S, b.qr, b.labels,
            b.next, (unsigned long long *)b.changes);
  // (5) prev <- labels <- next
  RR_CUDA(cudaMemcpyAsync(b.prev, b.labels, sizeof(int32_t) * F, cudaMemcpyDeviceToDevice, st));
  RR_CUDA(cudaMemcpyAsync(b.labels, b.next, sizeof(int32_t) * F, cudaMemcpyDeviceToDevice, st));
  RR_CUDA(cudaMemcpyAsync(changes_host, b.changes, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  return RR_OK;
}

}  // namespace rr
