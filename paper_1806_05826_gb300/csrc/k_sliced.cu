// Sliced mat-vecs of binary X, the per-iteration hot loop of Eq. (1)'s
// operator: u = X v (rows gather v) and X^T u (columns gather u).
//
// Layout ("sliced pattern"): the gathered dimension is cut into nb slices of
// at most kSliceMax entries, so a slice of the FP64 vector fits in shared
// memory; inside a slice an index is a 16-bit offset (half the bytes of an
// int32 index). The entries of every (outer index, slice) segment are padded
// to whole 16-byte words (8 offsets; the pad offset W reads a zero kept in
// shared memory; the 8 offsets of word w stored rotated by (w / 4) mod 8 so
// that dense runs gather without bank conflicts) and the segment is cut into
// pieces of at most kPieceWords
// words. Pieces are stored slice-major, so one CTA streams a contiguous range
// of them against the one vector slice it holds; each piece is summed by one
// lane (in a fixed order) into its own slot, numbered outer-major, and the
// slots of one outer index are summed afterwards in a fixed order. No atomics:
// every run gives identical bits.
//
// FP32 passes (the mixed-precision inner iterations) use the staged form:
// each task's index words, contiguous in memory, stream through a ring of
// shared-memory buffers by bulk asynchronous copies (cp.async.bulk completing
// on mbarriers), so the HBM stream never waits on the gathers; the buffers
// hold chunks of whole pieces (at most kChunkWords words), consumed by four
// independent teams of 256 threads. Every thread of a team first sums the 8
// offsets of one word of the chunk, then every piece sums its words' partial
// sums in order: the same operations in the same order as the lane-per-piece
// form, so both forms give identical bits.
#include <cmath>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "epilogue.cuh"
#include "tc_common.cuh"

namespace rr {

namespace {

constexpr int kSliceThreads = 1024;
constexpr int kTeams = 4;                            // independent teams of a CTA
constexpr int kTeamThreads = kSliceThreads / kTeams; // 256 threads (8 warps) per team
constexpr int kChunkWords = kTeamThreads;            // words of one staged chunk (4 KiB), one per thread
constexpr int kStagesW = 4;                          // stages in each team's ring
constexpr int kStagePtrs = kChunkWords + 8;          // staged piece pointers / slots per stage
constexpr int kStageSmem = 16 * kChunkWords + 8 * kStagePtrs + 32;   // words, pointers, slots, meta
constexpr int kTeamSmem = 2 * 4 * kChunkWords + kStagesW * kStageSmem + 8 * kStagesW;

// one thread per (outer o, slice b): entry range of the segment by binary search
__global__ void k_seg_bounds(int64_t n_outer, int32_t nb, int32_t W,
                             const int64_t *__restrict__ outer_ptr,
                             const int32_t *__restrict__ inner, int64_t *__restrict__ words,
                             int64_t *__restrict__ pieces) {
  const int64_t total = n_outer * nb;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = (int32_t)(t / n_outer);
    const int64_t o = t - (int64_t)b * n_outer;
    const int64_t lo0 = outer_ptr[o], hi0 = outer_ptr[o + 1];
    auto lower = [&](int64_t key) {
      int64_t lo = lo0, hi = hi0;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (inner[mid] < key) lo = mid + 1; else hi = mid;
      }
      return lo;
    };
    const int64_t s = lower((int64_t)b * W), e = lower((int64_t)(b + 1) * W);
    const int64_t w = (e - s + 7) / 8;
    words[t] = w;                                     // slice-major index b * n_outer + o
    pieces[t] = (w + kPieceWords - 1) / kPieceWords;  // empty segments have no piece
  }
}

// pieces of each outer index over all slices (outer-major slot numbering)
__global__ void k_outer_pieces(int64_t n_outer, int32_t nb, const int64_t *__restrict__ pieces,
                               int64_t *__restrict__ per_outer) {
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n_outer;
       o += (int64_t)gridDim.x * blockDim.x) {
    int64_t s = 0;
    for (int32_t b = 0; b < nb; ++b) s += pieces[(int64_t)b * n_outer + o];
    per_outer[o] = s;
  }
}

// one warp per (outer o, slice b): piece pointers and slots, then the padded
// 16-bit offsets of the segment
__global__ void k_fill_pieces(int64_t n_outer, int32_t nb, int32_t W,
                              const int64_t *__restrict__ outer_ptr,
                              const int32_t *__restrict__ inner,
                              const int64_t *__restrict__ word_off,
                              const int64_t *__restrict__ piece_off,
                              const int64_t *__restrict__ pieces,
                              const int64_t *__restrict__ slot_base, int32_t *__restrict__ pw,
                              int32_t *__restrict__ slot, uint16_t *__restrict__ idx) {
  const int64_t total = n_outer * nb;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = warp; t < total; t += nwarps) {
    const int32_t b = (int32_t)(t / n_outer);
    const int64_t o = t - (int64_t)b * n_outer;
    const int64_t lo0 = outer_ptr[o], hi0 = outer_ptr[o + 1];
    const int64_t key = (int64_t)b * W, key_end = (int64_t)(b + 1) * W;
    int64_t lo = lo0, hi = hi0;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (inner[mid] < key) lo = mid + 1; else hi = mid;
    }
    const int64_t s = lo;
    hi = hi0;   // end of this slice's entries (not of the whole outer index)
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (inner[mid] < key_end) lo = mid + 1; else hi = mid;
    }
    const int64_t len = lo - s;
    const int64_t w0 = word_off[t], nw = word_off[t + 1] - w0;
    int64_t pre = 0;   // pieces of this outer index in earlier slices
    for (int32_t bb = 0; bb < b; ++bb) pre += pieces[(int64_t)bb * n_outer + o];
    const int64_t np = pieces[t], p0 = piece_off[t];
    for (int64_t q = lane; q < np; q += 32) {
      pw[p0 + q] = (int32_t)(w0 + q * kPieceWords);
      slot[p0 + q] = (int32_t)(slot_base[o] + pre + q);
    }
    // entry u goes to word u / 8 at position (u + rot) mod 8, rot = (word >> 2) mod 8:
    // in a dense run (consecutive offsets) the 8 lanes whose words are 4 apart
    // then read 8 different shared-memory banks at every step of the gather
    uint16_t *dst = idx + w0 * 8;
    for (int64_t u = lane; u < nw * 8; u += 32) {
      const int64_t wl = u >> 3;
      const int32_t rot = (int32_t)(((w0 + wl) >> 2) & 7);
      dst[(wl << 3) + ((u + rot) & 7)] = u < len ? (uint16_t)(inner[s + u] - key) : (uint16_t)W;
    }
  }
}

// task t of slice b starts at the first piece whose start word reaches
// word_begin(b) + t * words(b) / T
__global__ void k_tasks(int32_t nb, const int32_t *__restrict__ task_base, int64_t n_outer,
                        const int64_t *__restrict__ word_off,
                        const int64_t *__restrict__ piece_off, const int32_t *__restrict__ pw,
                        int32_t *__restrict__ task_slice, int32_t *__restrict__ task_p) {
  const int32_t total = task_base[nb];
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= total; i += gridDim.x * blockDim.x) {
    if (i == total) {
      task_p[total] = (int32_t)piece_off[(int64_t)nb * n_outer];
      continue;
    }
    int32_t bl = 0, bh = nb - 1;   // the slice: the last b with task_base[b] <= i
    while (bl < bh) {
      const int32_t mid = (bl + bh + 1) >> 1;
      if (task_base[mid] <= i) bl = mid; else bh = mid - 1;
    }
    const int32_t b = bl, t = i - task_base[b], T = task_base[b + 1] - task_base[b];
    const int64_t wb = word_off[(int64_t)b * n_outer], we = word_off[(int64_t)(b + 1) * n_outer];
    const int64_t pb = piece_off[(int64_t)b * n_outer], pe = piece_off[(int64_t)(b + 1) * n_outer];
    const int64_t target = wb + (we - wb) * t / T;
    int64_t lo = pb, hi = pe;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (pw[mid] < target) lo = mid + 1; else hi = mid;
    }
    task_slice[i] = b;
    task_p[i] = (int32_t)lo;
  }
}

// The pieces of each task in order of decreasing length (counting sort on the
// word count, capped at the piece limit), so that the 32 lanes of a warp,
// which take 32 consecutive entries, sum pieces of about the same length.
// Within one length the order is that of the atomics; a piece's sum does not
// depend on where it is processed, so results are unaffected.
__global__ void k_order_pieces(const int32_t *__restrict__ task_p, const int32_t *__restrict__ pw,
                               int32_t *__restrict__ order) {
  __shared__ int32_t cnt[kPieceWords + 1], cur[kPieceWords + 1];
  const int32_t p0 = task_p[blockIdx.x], p1 = task_p[blockIdx.x + 1];
  for (int i = threadIdx.x; i <= kPieceWords; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  for (int32_t p = p0 + threadIdx.x; p < p1; p += blockDim.x)
    atomicAdd(&cnt[min(pw[p + 1] - pw[p], kPieceWords)], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t run = p0;
    for (int len = kPieceWords; len >= 0; --len) {
      cur[len] = run;
      run += cnt[len];
    }
  }
  __syncthreads();
  for (int32_t p = p0 + threadIdx.x; p < p1; p += blockDim.x)
    order[atomicAdd(&cur[min(pw[p + 1] - pw[p], kPieceWords)], 1)] = p;
}

// Pre-pass: the gathered vector, once per pass, in the accumulation type T
// (FP64, or FP32 for the mixed-precision inner iterations). v = x, or
// (kCombine) the per-index sums of the previous pass's slots.
template <bool kCombine, typename T>
__global__ void k_slice_prep(int64_t n, const double *__restrict__ x,
                             const double *__restrict__ in_psum,
                             const int32_t *__restrict__ in_slot_ptr, T *__restrict__ xq,
                             const int32_t *__restrict__ stop) {
  pdl_wait();
  if (stop && *stop) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v;
    if (kCombine) {
      // slots in order, four loads in flight
      v = 0.0;
      const int32_t q1 = in_slot_ptr[i + 1];
      for (int32_t q = in_slot_ptr[i]; q < q1; q += 4) {
        double t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) t[u] = q + u < q1 ? in_psum[q + u] : 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u) v += t[u];
      }
    } else {
      v = x[i];
    }
    xq[i] = (T)v;
  }
}

template <typename T>
__device__ __forceinline__ T gather8(const T *__restrict__ xs, const uint4 q) {
  return ((xs[q.x & 0xffffu] + xs[q.x >> 16]) + (xs[q.y & 0xffffu] + xs[q.y >> 16])) +
         ((xs[q.z & 0xffffu] + xs[q.z >> 16]) + (xs[q.w & 0xffffu] + xs[q.w >> 16]));
}

// The gather pass. One CTA per task: copy the task's vector slice into shared
// memory, then every lane sums whole pieces: the 32 lanes of a warp take 32
// consecutive pieces, so piece pointers, slots and the words of short pieces
// are read coalesced, and each lane loads its piece's words four at a time.
// Sums in a fixed order in T; the piece sum is stored as PS (FP64, or FP32
// for the patterns whose consumers sum in FP32).
template <typename T, typename PS>
__global__ void __launch_bounds__(kSliceThreads, 1) k_sliced_gather(
    SlicedView P, const T *__restrict__ xq, PS *__restrict__ out_psum,
    const int32_t *__restrict__ stop) {
  pdl_wait();
  if (stop && *stop) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  const int task = blockIdx.x;
  const int32_t b = P.task_slice[task];
  const int64_t base = (int64_t)b * P.W;
  const int64_t width = min((int64_t)P.W, P.n_inner - base);
  for (int i0 = threadIdx.x; i0 <= P.W; i0 += 4 * kSliceThreads) {
    T v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * kSliceThreads;
      v[u] = i < width ? xq[base + i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * kSliceThreads;
      if (i <= P.W) xs[i] = v[u];
    }
  }
  __syncthreads();
  const int32_t p0 = P.task_p[task], p1 = P.task_p[task + 1];
  const uint4 pad = make_uint4(P.W | (P.W << 16), P.W | (P.W << 16), P.W | (P.W << 16),
                               P.W | (P.W << 16));
  // four pieces per lane at a time: their pointers and first words are loaded
  // together, so four independent 16-byte loads are in flight per lane
  constexpr int kILP = 4;
  for (int32_t pb = p0 + threadIdx.x; pb < p1; pb += kILP * kSliceThreads) {
    int32_t pp[kILP], w0[kILP], w1[kILP];
    uint4 first[kILP];
#pragma unroll
    for (int u = 0; u < kILP; ++u) {
      const int32_t p = pb + u * kSliceThreads;
      pp[u] = p < p1 ? __ldg(P.order + p) : 0;
    }
#pragma unroll
    for (int u = 0; u < kILP; ++u) {
      const int32_t p = pb + u * kSliceThreads;
      w0[u] = p < p1 ? __ldg(P.pw + pp[u]) : 0;
      w1[u] = p < p1 ? __ldg(P.pw + pp[u] + 1) : 0;
    }
#pragma unroll
    for (int u = 0; u < kILP; ++u) first[u] = w0[u] < w1[u] ? __ldg(P.idx + w0[u]) : pad;
#pragma unroll
    for (int u = 0; u < kILP; ++u) {
      const int32_t p = pb + u * kSliceThreads;
      if (p >= p1) break;
      T acc = gather8(xs, first[u]);
      for (int32_t w = w0[u] + 1; w < w1[u]; w += 4) {
        uint4 q[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) q[k] = (w + k < w1[u]) ? __ldg(P.idx + w + k) : pad;
        // gathers only for words of this piece (no shared loads for absent words)
        acc += gather8(xs, q[0]);
#pragma unroll
        for (int k = 1; k < 4; ++k)
          if (w + k < w1[u]) acc += gather8(xs, q[k]);
      }
      out_psum[__ldg(P.slot + pp[u])] = (PS)acc;
    }
  }
}

// The streaming gather (FP32 piece sums). One CTA per task: the vector slice
// in shared memory, then each of the 32 warps streams its own contiguous
// range of the task's words (ranges start at piece boundaries), 64 words per
// step, the next step loaded ahead: lane l loads words 2l and 2l + 1 of the
// step (coalesced) and their metadata, sums each word's 8 gathered values,
// folds its two words into the sum of its open tail, and a segmented
// inclusive scan of the tails over the 32 lanes (segments = pieces; a piece
// may continue from the previous step, whose running sum is carried) gives the
// running sum entering each lane, from which each piece's sum at its last word
// follows; that word's lane stores it in the piece's slot. No indirection
// before the loads: every load is coalesced and many are in flight per warp.
// The sums have a fixed order (each word's 8 values as in gather8, then the
// lane's two words, the scan tree and the carry), so every run gives
// identical bits.

constexpr int kStreamThreads = 512;   // 16 warps, two CTAs per SM (two slices resident)
constexpr int kStreamRanges = 32;     // word ranges per task (each warp takes two)
__global__ void __launch_bounds__(kStreamThreads, 2) k_stream_gather(
    SlicedView P, const int32_t *__restrict__ wmeta, const int32_t *__restrict__ wstart,
    const float *__restrict__ xq, float *__restrict__ out, const int32_t *__restrict__ stop,
    int32_t *err) {
  pdl_wait();
  if (stop && *stop) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *xs = reinterpret_cast<float *>(smem_raw);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + sizeof(float) * ((P.W + 1 + 3) & ~3));
  int32_t *abort_flag = reinterpret_cast<int32_t *>(bar + 1);
  const int task = blockIdx.x;
  const int32_t b = P.task_slice[task];
  const int64_t base = (int64_t)b * P.W;
  const int64_t width = min((int64_t)P.W, P.n_inner - base);
  // the vector slice: its 16-byte aligned head by one bulk copy (completing on
  // an mbarrier), the rest and the zero padding by plain loads meanwhile
  const int64_t nbulk = (base & 3) == 0 ? (width & ~(int64_t)3) : 0;
  if (threadIdx.x == 0) {
    *abort_flag = 0;
    if (nbulk > 0) {
      tc::mbar_init(bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      tc::mbar_expect_tx(bar, (uint32_t)(nbulk * 4));
      tc::bulk_load(xs, xq + base, (uint32_t)(nbulk * 4), bar);
    }
  }
  for (int i = (int)nbulk + threadIdx.x; i <= P.W; i += kStreamThreads)
    xs[i] = i < width ? xq[base + i] : 0.f;
  __syncthreads();
  if (nbulk > 0 && !tc::mbar_wait(bar, 0, abort_flag)) {
    set_dev_error(err, DEV_TIMEOUT);
    atomicExch(abort_flag, 1);
    // the copy lands before this thread leaves the CTA's shared memory
    const int32_t never = 0;
    (void)tc::mbar_wait(bar, 0, &never);
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint4 pad = make_uint4(P.W | (P.W << 16), P.W | (P.W << 16), P.W | (P.W << 16),
                               P.W | (P.W << 16));
  for (int rg = warp; rg < kStreamRanges; rg += kStreamThreads / 32) {
  const int32_t w0 = wstart[task * (kStreamRanges + 1) + rg];
  const int32_t w1 = wstart[task * (kStreamRanges + 1) + rg + 1];
  float carry = 0.f;   // running sum of the piece open at the end of the previous step
  bool open = false;
  // one step = 64 words, lane l taking words 2l and 2l + 1; the next step's
  // loads are issued before this step is summed
  uint4 qa[2], qn[2];
  int32_t ma[2], mn[2];
  auto load = [&](int32_t c, uint4 *q, int32_t *m) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int32_t w = c + 2 * lane + h;
      q[h] = w < w1 ? __ldg(P.idx + w) : pad;
      m[h] = w < w1 ? __ldg(wmeta + w) : -2;   // -2: past the range
    }
  };
  if (w0 < w1) load(w0, qa, ma);
  for (int32_t c = w0; c < w1; c += 64) {   // warp-uniform
    if (c + 64 < w1) load(c + 64, qn, mn);
    const float x0 = gather8(xs, qa[0]), x1 = gather8(xs, qa[1]);
    // starts: element 0 of lane l starts a piece when element 1 of lane l - 1
    // ended one (lane 0: when no piece is open); element 1 when element 0 did
    const uint32_t ends1 = __ballot_sync(0xffffffffu, ma[1] >= 0);
    const bool s0 = lane == 0 ? !open : ((ends1 >> (lane - 1)) & 1u) != 0;
    const bool s1 = ma[0] >= 0;
    // the lane's open tail (the sum since its last start, or of both words),
    // then a segmented inclusive scan of the tails over the lanes (a segment
    // begins at a lane holding a start; dist = lanes since it began)
    float v = s1 ? x1 : x0 + x1;
    const uint32_t starts = __ballot_sync(0xffffffffu, s0 || s1);
    const uint32_t upto = starts & (0xffffffffu >> (31 - lane));
    const int dist = upto ? lane - (31 - __clz((int)upto)) : 32;   // 32: began earlier
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const float vy = __shfl_up_sync(0xffffffffu, v, d);
      if (lane >= d && dist >= d) v = vy + v;
    }
    if (!upto) v = carry + v;   // still in the piece carried from the previous step
    // the running sum entering this lane, then each word's running sum
    float excl = __shfl_up_sync(0xffffffffu, v, 1);
    if (lane == 0) excl = open ? carry : 0.f;
    const float inc0 = s0 ? x0 : excl + x0;
    const float inc1 = s1 ? x1 : inc0 + x1;
    if (ma[0] >= 0) out[ma[0]] = inc0;
    if (ma[1] >= 0) out[ma[1]] = inc1;
    carry = __shfl_sync(0xffffffffu, inc1, 31);
    open = (__ballot_sync(0xffffffffu, ma[1] == -1) >> 31) & 1u;
    if (!open) carry = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      qa[h] = qn[h];
      ma[h] = mn[h];
    }
  }
  }
}

// wmeta: the slot of each piece at its last word (-1 elsewhere, set before)
__global__ void k_word_meta(int64_t npieces, const int32_t *__restrict__ pw,
                            const int32_t *__restrict__ slot, int32_t *__restrict__ wmeta) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npieces;
       p += (int64_t)gridDim.x * blockDim.x)
    wmeta[pw[p + 1] - 1] = slot[p];
}

// wstart[t * 33 + w]: the first word of warp w's range in task t, the first
// piece start at or after an even split of the task's words (33rd: the end)
__global__ void k_warp_ranges(int32_t ntasks, const int32_t *__restrict__ task_p,
                              const int32_t *__restrict__ pw, int32_t *__restrict__ wstart) {
  const int64_t total = (int64_t)ntasks * 33;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = (int32_t)(e / 33), w = (int32_t)(e % 33);
    const int32_t p0 = task_p[t], p1 = task_p[t + 1];
    const int32_t wb = pw[p0], we = pw[p1];
    if (w == 32) {
      wstart[e] = we;
      continue;
    }
    const int64_t target = wb + (int64_t)(we - wb) * w / 32;
    int32_t lo = p0, hi = p1;
    while (lo < hi) {
      const int32_t mid = (lo + hi) >> 1;
      if (pw[mid] < target) lo = mid + 1; else hi = mid;
    }
    wstart[e] = lo < p1 ? pw[lo] : we;
  }
}

// The staged gather (see the file comment). The CTA's 32 warps form kTeams
// independent teams of 8 warps; team j consumes chunks j, j + kTeams, ... of
// the task through its own ring of kStagesW stages and syncs only its own 256
// threads (named barrier 1 + j), so one team's waits overlap the others' work.
// A stage holds the chunk's index words, its pieces' word pointers and slots
// (both copied as 16-byte aligned supersets of the chunk's range) and the
// chunk's metadata, written by the team's producer thread before it issues
// the copies: a consumer touches no global memory but the piece sums it
// stores. Waits on the mbarriers are bounded: on expiry the CTA records
// DEV_TIMEOUT, every team stops, waits (bounded) for the copies it issued and
// returns.
struct StageMeta {
  int32_t pa, pb;   // pieces [pa, pb) of the chunk
  int32_t wa, nw;   // its words [wa, wa + nw)
  int32_t pal;      // first piece of the staged pointer/slot range (pa rounded down to 4)
  int32_t pad[3];
};

__device__ __forceinline__ void team_sync(int team) {
  asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(kTeamThreads) : "memory");
}

template <typename PS>
__global__ void __launch_bounds__(kSliceThreads, 1) k_sliced_gather_staged(
    SlicedView P, const int32_t *__restrict__ chunk_p, const int32_t *__restrict__ chunk_w,
    const int32_t *__restrict__ task_c, const float *__restrict__ xq,
    PS *__restrict__ out_psum, const int32_t *__restrict__ stop, int32_t *err) {
  pdl_wait();
  if (stop && *stop) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int slice_floats = (P.W + 1 + 3) & ~3;
  const int team = threadIdx.x / kTeamThreads, tt = threadIdx.x % kTeamThreads;
  float *xs = reinterpret_cast<float *>(smem_raw);
  unsigned char *team_base = smem_raw + sizeof(float) * slice_floats + (size_t)team * kTeamSmem;
  float *wsum = reinterpret_cast<float *>(team_base);
  unsigned char *stage0 = team_base + 2 * sizeof(float) * kChunkWords;
  uint64_t *full = reinterpret_cast<uint64_t *>(stage0 + (size_t)kStagesW * kStageSmem);
  int32_t *abort_flag = reinterpret_cast<int32_t *>(smem_raw + sizeof(float) * slice_floats +
                                                    (size_t)kTeams * kTeamSmem);
  auto words_of = [&](int s) { return reinterpret_cast<uint4 *>(stage0 + (size_t)s * kStageSmem); };
  auto pw_of = [&](int s) {
    return reinterpret_cast<int32_t *>(stage0 + (size_t)s * kStageSmem + 16 * kChunkWords);
  };
  auto slot_of = [&](int s) { return pw_of(s) + kStagePtrs; };
  auto meta_of = [&](int s) { return reinterpret_cast<StageMeta *>(slot_of(s) + kStagePtrs); };

  const int task = blockIdx.x;
  const int32_t b = P.task_slice[task];
  const int32_t c0 = task_c[task], nch = task_c[task + 1] - c0;
  // this team's chunks: c0 + team + kTeams q, q = 0 .. nq-1
  const int nq = nch > team ? (nch - team + kTeams - 1) / kTeams : 0;

  // producer (tt == 0): the metadata of the next chunk to issue, loaded ahead
  int32_t m_pa = 0, m_pb = 0, m_wa = 0, m_wb = 0;
  auto load_meta = [&](int q) {
    const int32_t c = c0 + team + kTeams * q;
    m_pa = chunk_p[c];
    m_pb = chunk_p[c + 1];
    m_wa = chunk_w[c];
    m_wb = chunk_w[c + 1];
  };
  auto issue = [&](int q) {   // the team's chunk q into stage q % kStagesW, metadata in m_*
    const int s = q % kStagesW;
    const int32_t pal = m_pa & ~3;
    const int32_t pend = (m_pb + 1 + 3) & ~3;   // pointers [pal, pend) cover pw[pa..pb]
    const int32_t send = (m_pb + 3) & ~3;       // slots [pal, send) cover slot[pa..pb-1]
    StageMeta *m = meta_of(s);
    m->pa = m_pa;
    m->pb = m_pb;
    m->wa = m_wa;
    m->nw = m_wb - m_wa;
    m->pal = pal;
    const uint32_t wbytes = (uint32_t)(m_wb - m_wa) * 16u;
    const uint32_t pbytes = (uint32_t)(pend - pal) * 4u, sbytes = (uint32_t)(send - pal) * 4u;
    uint64_t *bar = &full[s];
    tc::mbar_expect_tx(bar, wbytes + pbytes + sbytes);
    tc::bulk_load(words_of(s), P.idx + m_wa, wbytes, bar);
    tc::bulk_load(pw_of(s), P.pw + pal, pbytes, bar);
    tc::bulk_load(slot_of(s), P.slot + pal, sbytes, bar);
  };

  if (threadIdx.x == 0) *abort_flag = 0;
  int issued = min(kStagesW, nq);
  if (tt == 0) {
    for (int s = 0; s < kStagesW; ++s) tc::mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int q = 0; q < issued; ++q) {
      load_meta(q);
      issue(q);
    }
    if (issued < nq) load_meta(issued);
  }
  // the vector slice, while the first chunks are in flight
  const int64_t base = (int64_t)b * P.W;
  const int64_t width = min((int64_t)P.W, P.n_inner - base);
  for (int i = threadIdx.x; i <= P.W; i += kSliceThreads) xs[i] = i < width ? xq[base + i] : 0.0f;
  __syncthreads();

  int q = 0;
  for (; q < nq; ++q) {
    const int s = q % kStagesW;
    const bool ok = tc::mbar_wait(&full[s], (uint32_t)((q / kStagesW) & 1), abort_flag);
    if (!ok) {
      set_dev_error(err, DEV_TIMEOUT);
      atomicExch(abort_flag, 1);
    }
    const StageMeta m = *meta_of(s);
    float *ws = wsum + (q & 1) * kChunkWords;   // word sums: two buffers, alternating
    if (ok && tt < m.nw) {
      const uint4 w = words_of(s)[tt];
      ws[tt] = ((xs[w.x & 0xffffu] + xs[w.x >> 16]) + (xs[w.y & 0xffffu] + xs[w.y >> 16])) +
               ((xs[w.z & 0xffffu] + xs[w.z >> 16]) + (xs[w.w & 0xffffu] + xs[w.w >> 16]));
    }
    // one barrier per chunk: it publishes this chunk's word sums, and every
    // thread has finished the previous chunk's piece sums, so that chunk's
    // stage can be refilled and its word-sum buffer reused by the next chunk
    team_sync(team);
    if (*(volatile int32_t *)abort_flag) break;
    if (tt == 0 && q >= 1 && issued < nq) {
      tc::fence_proxy_async_smem();
      issue(issued);   // into the stage of chunk q - 1
      ++issued;
      if (issued < nq) load_meta(issued);
    }
    const int32_t *pws = pw_of(s) - m.pal, *sls = slot_of(s) - m.pal;
    for (int32_t p = m.pa + tt; p < m.pb; p += kTeamThreads) {
      const int32_t w0 = pws[p] - m.wa, w1 = pws[p + 1] - m.wa;
      float acc = ws[w0];
      for (int32_t w = w0 + 1; w < w1; ++w) acc += ws[w];
      out_psum[sls[p]] = (PS)acc;
    }
  }
  if (tt == 0 && *(volatile int32_t *)abort_flag) {
    // copies issued but not consumed (chunks q..issued-1 of this team) must
    // land before the CTA's shared memory is released
    const int32_t never = 0;
    for (int j = q; j < issued; ++j)
      (void)tc::mbar_wait(&full[j % kStagesW], (uint32_t)((j / kStagesW) & 1), &never);
  }
}

// Chunks of whole pieces of at most kChunkWords words, per task: chunk j of
// a task holds the pieces that start in words [w0 + j S, w0 + (j + 1) S) of it
// (w0 its first word, S = kChunkWords - kPieceWords), so a chunk spans at most
// S + kPieceWords words, and every chunk holds a piece (pieces are contiguous
// and at most kPieceWords long). count: chunks of each task; fill: the first
// piece and word of every chunk (chunk_p[total] = npieces), by a search that
// resumes where the previous chunk's ended.
constexpr int32_t kChunkStep = kChunkWords - kPieceWords;
__global__ void k_chunk_count(int32_t ntasks, const int32_t *__restrict__ task_p,
                              const int32_t *__restrict__ pw, int64_t *__restrict__ cnt) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntasks; t += gridDim.x * blockDim.x) {
    const int32_t p0 = task_p[t], p1 = task_p[t + 1];
    cnt[t] = p1 > p0 ? (pw[p1 - 1] - pw[p0]) / kChunkStep + 1 : 0;
  }
}

__global__ void k_chunk_fill(int32_t ntasks, const int32_t *__restrict__ task_p,
                             const int32_t *__restrict__ pw, const int64_t *__restrict__ off,
                             int32_t *__restrict__ chunk_p, int32_t *__restrict__ chunk_w,
                             int32_t *__restrict__ task_c, int64_t total, int32_t npieces) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntasks; t += gridDim.x * blockDim.x) {
    const int64_t n0 = off[t], n1 = off[t + 1];
    task_c[t] = (int32_t)n0;
    const int32_t p0 = task_p[t], p1 = task_p[t + 1];
    const int32_t w0 = p1 > p0 ? pw[p0] : 0;
    int32_t lo = p0;
    for (int64_t n = n0; n < n1; ++n) {
      const int32_t target = w0 + (int32_t)(n - n0) * kChunkStep;
      int32_t hi = p1;
      while (lo < hi) {   // first piece of the task starting at or after target
        const int32_t mid = (lo + hi) >> 1;
        if (pw[mid] < target) lo = mid + 1; else hi = mid;
      }
      chunk_p[n] = lo;
      chunk_w[n] = pw[lo];
    }
    if (t == ntasks - 1) {
      task_c[ntasks] = (int32_t)total;
      chunk_p[total] = npieces;
      chunk_w[total] = pw[npieces];
    }
  }
}

// Reorders the 8 offsets inside index words so that the staged gather's reads
// spread over the shared-memory banks. In that kernel the 32 lanes of a warp
// read position u of 32 consecutive words of a chunk at the same time; here one
// warp takes such a group of 32 words and, for u = 0..7 in turn, lets the lanes
// pick (one after the other) the remaining offset of their word whose bank
// (offset mod 32) has been picked least often at this position, padding
// entries (offset W, one shared address) costing nothing. A word's 8 values
// are the same in any order, so this changes only the order of the FP32 sums
// inside a word (both gather kernels read the same words, so they keep giving
// identical bits).
constexpr int kBalThreads = 64;
// One group of n <= 32 words idx[w0 + stride l], the words one warp
// instruction reads at once (thread-private rows of the block's shared arrays).
__device__ void balance_group(uint4 *__restrict__ idx, int64_t w0, int stride, int n, int32_t W,
                              uint16_t *outs, uint8_t *usedm, uint8_t *cnts) {
  const uint16_t padv = (uint16_t)W;
  for (int l = 0; l < n; ++l) usedm[l] = 0;
  for (int u = 0; u < 8; ++u) {
    for (int bk = 0; bk < 32; ++bk) cnts[bk] = 0;
    for (int l = 0; l < n; ++l) {
      const uint4 q = idx[w0 + (int64_t)stride * l];
      const uint16_t off[8] = {(uint16_t)(q.x & 0xffffu), (uint16_t)(q.x >> 16),
                               (uint16_t)(q.y & 0xffffu), (uint16_t)(q.y >> 16),
                               (uint16_t)(q.z & 0xffffu), (uint16_t)(q.z >> 16),
                               (uint16_t)(q.w & 0xffffu), (uint16_t)(q.w >> 16)};
      const uint32_t used = usedm[l];
      int best = 0, best_cost = 0x7fffffff;
      uint16_t bo = padv;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (used & (1u << j)) continue;
        const int cost = off[j] == padv ? -1 : (int)cnts[off[j] & 31];
        if (cost < best_cost) {
          best_cost = cost;
          best = j;
          bo = off[j];
        }
      }
      usedm[l] = (uint8_t)(used | (1u << best));
      outs[l * 8 + u] = bo;
      if (bo != padv) cnts[bo & 31] += 1;
    }
  }
  for (int l = 0; l < n; ++l) {
    const uint16_t *o = &outs[l * 8];
    idx[w0 + (int64_t)stride * l] = make_uint4((uint32_t)o[0] | ((uint32_t)o[1] << 16),
                                               (uint32_t)o[2] | ((uint32_t)o[3] << 16),
                                               (uint32_t)o[4] | ((uint32_t)o[5] << 16),
                                               (uint32_t)o[6] | ((uint32_t)o[7] << 16));
  }
}

__global__ void __launch_bounds__(kBalThreads) k_balance_words(int64_t n_chunks,
                                                               const int32_t *__restrict__ chunk_w,
                                                               int32_t W, uint4 *__restrict__ idx) {
  // thread-private rows (padded so that the threads' rows start in different banks)
  __shared__ uint16_t outs[kBalThreads][32 * 8 + 2];
  __shared__ uint8_t usedm[kBalThreads][36];
  __shared__ uint8_t cnts[kBalThreads][36];
  const int t = threadIdx.x;
  constexpr int kGroups = kChunkWords / 32;
  for (int64_t g = (int64_t)blockIdx.x * kBalThreads + t; g < n_chunks * kGroups;
       g += (int64_t)gridDim.x * kBalThreads) {
    const int64_t c = g / kGroups;
    const int64_t w0 = (int64_t)chunk_w[c] + 32 * (g % kGroups), w1 = chunk_w[c + 1];
    if (w0 >= w1) continue;
    const int n = (int)min((int64_t)32, w1 - w0);
    balance_group(idx, w0, 1, n, W, outs[t], usedm[t], cnts[t]);
  }
}

// The same for the streaming gather's reads: in every 64-word step of a warp's
// range, lane l reads words 2l and 2l + 1, so the even and the odd words of
// the step are the groups (one thread per group: range, step, half).
__global__ void __launch_bounds__(kBalThreads) k_balance_stream(int64_t n_ranges, int32_t max_steps,
                                                                const int32_t *__restrict__ wstart,
                                                                int32_t W, uint4 *__restrict__ idx) {
  __shared__ uint16_t outs[kBalThreads][32 * 8 + 2];
  __shared__ uint8_t usedm[kBalThreads][36];
  __shared__ uint8_t cnts[kBalThreads][36];
  const int t = threadIdx.x;
  const int64_t total = n_ranges * max_steps * 2;
  for (int64_t g = (int64_t)blockIdx.x * kBalThreads + t; g < total;
       g += (int64_t)gridDim.x * kBalThreads) {
    const int h = (int)(g & 1);
    const int64_t j = (g >> 1) % max_steps, r = (g >> 1) / max_steps;
    const int64_t task = r / kStreamRanges, rg = r % kStreamRanges;
    const int32_t w0 = wstart[task * (kStreamRanges + 1) + rg];
    const int32_t w1 = wstart[task * (kStreamRanges + 1) + rg + 1];
    const int64_t c = (int64_t)w0 + 64 * j;
    const int n = (int)min((int64_t)32, ((int64_t)w1 - c - h + 1) / 2);
    if (n > 0) balance_group(idx, c + h, 2, n, W, outs[t], usedm[t], cnts[t]);
  }
}

// Sum of the slots of every outer index -> out[o] (u = X v on its own).
__global__ void k_slot_sum(int64_t n, const int32_t *__restrict__ slot_ptr,
                           const double *__restrict__ psum, double *__restrict__ out) {
  pdl_wait();
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n;
       o += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int32_t q = slot_ptr[o]; q < slot_ptr[o + 1]; ++q) v += psum[q];
    out[o] = v;
  }
}

// t_i = sum of the slots of feature i, then the mode's epilogue; per-block
// partial dots in a fixed order. Features with more than kLightSlots slots
// (the long columns, listed in heavy[]) are summed first, one warp each (32
// lanes strided, then a fixed shuffle tree); every other feature by one 8-lane
// group with up to 4 slot loads in flight per lane. Fixed assignment and
// order: every run gives identical bits.
constexpr int kLightSlots = 32;

__global__ void __launch_bounds__(kThreads) k_sliced_epilogue(int64_t F, const int32_t *__restrict__ slot_ptr,
                                                              const double *__restrict__ psum,
                                                              const int32_t *__restrict__ heavy,
                                                              int32_t n_heavy, CscEpilogue ep) {
  pdl_wait();
  if (ep.stop && *ep.stop) return;
  __shared__ double sm[kWarps + 1];
  const int lane = threadIdx.x & 31;
  const int lane8 = threadIdx.x & 7, gw = (threadIdx.x >> 3) & 3;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double dot = 0.0;
  for (int64_t h = warp; h < n_heavy; h += nwarps) {   // warp-uniform loop
    const int32_t i = heavy[h];
    const int32_t q0 = slot_ptr[i], q1 = slot_ptr[i + 1];
    double s0 = 0.0, s1 = 0.0;
    int32_t q = q0 + lane;
    for (; q + 32 < q1; q += 64) {
      s0 += psum[q];
      s1 += psum[q + 32];
    }
    if (q < q1) s0 += psum[q];
    double s = warp_sum(s0 + s1);
    if (lane == 0) epilogue(ep, i, s, dot);
  }
  // four features per 8-lane group at a time (features i0 + 4h + gw, h < 4):
  // their slot loads are in flight together
  constexpr int kH = 4;
  for (int64_t i0 = warp * 4 * kH; i0 < F; i0 += nwarps * 4 * kH) {   // warp-uniform loop
    int64_t ii[kH];
    int32_t q0[kH], q1[kH];
    bool light[kH];
#pragma unroll
    for (int h = 0; h < kH; ++h) {
      ii[h] = i0 + 4 * h + gw;
      q0[h] = ii[h] < F ? slot_ptr[ii[h]] : 0;
      q1[h] = ii[h] < F ? slot_ptr[ii[h] + 1] : 0;
      light[h] = ii[h] < F && q1[h] - q0[h] <= kLightSlots;
    }
    double v[kH][4];
#pragma unroll
    for (int h = 0; h < kH; ++h)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int32_t q = q0[h] + lane8 + 8 * u;
        v[h][u] = light[h] && q < q1[h] ? psum[q] : 0.0;
      }
#pragma unroll
    for (int h = 0; h < kH; ++h) {
      double s = (v[h][0] + v[h][1]) + (v[h][2] + v[h][3]);
      s += __shfl_xor_sync(0xffffffffu, s, 4);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      if (light[h] && lane8 == 0) epilogue(ep, ii[h], s, dot);
    }
  }
  const double tot = block_sum(dot, sm);
  if (threadIdx.x == 0 && ep.dot_part) ep.dot_part[blockIdx.x] = tot;
}

__global__ void k_to_i32(int64_t n, const int64_t *__restrict__ in, int32_t *__restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int32_t)in[i];
}

template <typename T>
size_t slice_smem(int32_t W) { return sizeof(T) * ((size_t)W + 1); }

// the stream gather: the FP32 slice (rounded up to 16 bytes), its mbarrier and
// an abort flag
inline size_t stream_smem(int32_t W) { return sizeof(float) * (size_t)((W + 1 + 3) & ~3) + 16; }

template <typename T>
size_t staged_smem(int32_t W) {
  return sizeof(float) * (size_t)((W + 1 + 3) & ~3) + (size_t)kTeams * kTeamSmem + 16;
}

size_t staged_smem(int32_t W) {
  return sizeof(float) * (size_t)((W + 1 + 3) & ~3) + (size_t)kTeams * kTeamSmem + 16;
}

template <typename T, typename PS>
rr_status set_smem_attr() {
  static bool done = false;
  if (!done) {
    RR_CUDA(cudaFuncSetAttribute(k_sliced_gather<T, PS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)slice_smem<T>(kSliceMax)));
    done = true;
  }
  return RR_OK;
}

template <typename PS>
rr_status set_staged_attr() {
  static bool done = false;
  if (!done) {   // the largest slice any pattern can have
    RR_CUDA(cudaFuncSetAttribute(k_sliced_gather_staged<PS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)staged_smem(kSliceMax)));
    done = true;
  }
  return RR_OK;
}

// The gather kernel of P (lanes or staged) with P's piece-sum type.
template <typename T, typename PS>
rr_status launch_gather(const SlicedPattern &P, const T *xq, const int32_t *stop, cudaStream_t st,
                        bool pdl) {
  PS *out = reinterpret_cast<PS *>(P.psum);
  if constexpr (std::is_same<T, float>::value && std::is_same<PS, float>::value) {
    if (P.wmeta) {
      static bool attr = false;
      if (!attr) {
        RR_CUDA(cudaFuncSetAttribute(k_stream_gather, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)stream_smem(kSliceMax)));
        RR_CUDA(cudaFuncSetAttribute(k_stream_gather,
                                     cudaFuncAttributePreferredSharedMemoryCarveout, 100));
        attr = true;
      }
      if (pdl)
        RR_LAUNCH_PDL(k_stream_gather, P.ntasks, kStreamThreads, stream_smem(P.W), st,
                      P.view(), P.wmeta, P.wstart, xq, out, stop, P.err);
      else
        RR_LAUNCH(k_stream_gather, P.ntasks, kStreamThreads, stream_smem(P.W), st, P.view(),
                  P.wmeta, P.wstart, xq, out, stop, P.err);
      return RR_OK;
    }
  }
  if (std::is_same<T, float>::value && P.staged && P.chunk_p) {
    RR_TRY(set_staged_attr<PS>());
    const float *x = reinterpret_cast<const float *>(xq);
    if (pdl)
      RR_LAUNCH_PDL(k_sliced_gather_staged<PS>, P.ntasks, kSliceThreads, staged_smem(P.W), st,
                    P.view(), P.chunk_p, P.chunk_w, P.task_c, x, out, stop, P.err);
    else
      RR_LAUNCH(k_sliced_gather_staged<PS>, P.ntasks, kSliceThreads, staged_smem(P.W), st,
                P.view(), P.chunk_p, P.chunk_w, P.task_c, x, out, stop, P.err);
    return RR_OK;
  }
  RR_TRY((set_smem_attr<T, PS>()));
  if (pdl)
    RR_LAUNCH_PDL((k_sliced_gather<T, PS>), P.ntasks, kSliceThreads, slice_smem<T>(P.W), st,
                  P.view(), xq, out, stop);
  else
    RR_LAUNCH((k_sliced_gather<T, PS>), P.ntasks, kSliceThreads, slice_smem<T>(P.W), st,
              P.view(), xq, out, stop);
  return RR_OK;
}

template <typename T>
rr_status gather_t(const SlicedPattern &P, const double *x, const SlicedPattern *in,
                   const int32_t *stop, cudaStream_t st, bool xq_ready) {
  const int64_t n = P.n_inner;
  T *xq = reinterpret_cast<T *>(P.xq);
  if (xq_ready && !in) {
    // the vector's producer already wrote its copy in T into P.xq
  } else if (in)
    RR_LAUNCH_PDL((k_slice_prep<true, T>), grid_for(n, kThreads), kThreads, 0, st, n, nullptr,
              in->psum, in->slot_ptr, xq, stop);
  else
    RR_LAUNCH_PDL((k_slice_prep<false, T>), grid_for(n, kThreads), kThreads, 0, st, n, x, nullptr,
              nullptr, xq, stop);
  return P.psum32 ? launch_gather<T, float>(P, xq, stop, st, true)
                  : launch_gather<T, double>(P, xq, stop, st, true);
}

}  // namespace

rr_status sliced_build(int64_t n_outer, int64_t n_inner, const int64_t *outer_ptr,
                       const int32_t *inner, SlicedPattern &P, int32_t *err, cudaStream_t st,
                       bool chunks) {
  P = SlicedPattern{};
  P.err = err;
  P.n_outer = n_outer;
  P.n_inner = n_inner;
  P.nb = (int32_t)std::max<int64_t>(1, (n_inner + kSliceMax - 1) / kSliceMax);
  P.W = (int32_t)((n_inner + P.nb - 1) / P.nb);
  const int64_t nseg = n_outer * P.nb;
  int64_t *buf = nullptr;
  const int64_t scan_len = scan_scratch_len(std::max(nseg, n_outer)) + 8;
  RR_CUDA(cudaMalloc(&buf, sizeof(int64_t) * (4 * (nseg + 1) + 2 * (n_outer + 1) + scan_len)));
  int64_t *words = buf, *pieces = buf + (nseg + 1), *word_off = buf + 2 * (nseg + 1),
          *piece_off = buf + 3 * (nseg + 1), *per_outer = buf + 4 * (nseg + 1),
          *slot_base = per_outer + (n_outer + 1), *scr = slot_base + (n_outer + 1);
  rr_status s = RR_OK;
  auto run = [&]() -> rr_status {
    RR_LAUNCH(k_seg_bounds, grid_for(nseg, kThreads), kThreads, 0, st, n_outer, P.nb, P.W,
              outer_ptr, inner, words, pieces);
    RR_TRY(scan_exclusive(words, word_off, nseg, scr, st));
    RR_TRY(scan_exclusive(pieces, piece_off, nseg, scr, st));
    RR_LAUNCH(k_outer_pieces, grid_for(n_outer, kThreads), kThreads, 0, st, n_outer, P.nb, pieces,
              per_outer);
    RR_TRY(scan_exclusive(per_outer, slot_base, n_outer, scr, st));
    int64_t tot[2];
    RR_CUDA(cudaMemcpyAsync(&tot[0], word_off + nseg, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaMemcpyAsync(&tot[1], piece_off + nseg, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    P.nwords = tot[0];
    P.npieces = tot[1];
    if (P.nwords >= (1LL << 31) || P.npieces >= (1LL << 31)) {
      rr_set_error("sliced pattern too large");
      return RR_UNSUPPORTED;
    }
    // +8 entries: the staged gather copies 16-byte aligned supersets of piece ranges
    RR_CUDA(cudaMalloc(&P.pw, sizeof(int32_t) * (P.npieces + 1 + 8)));
    RR_CUDA(cudaMalloc(&P.slot, sizeof(int32_t) * (P.npieces + 8)));
    RR_CUDA(cudaMalloc(&P.slot_ptr, sizeof(int32_t) * (n_outer + 1)));
    RR_CUDA(cudaMalloc(&P.idx, 16 * std::max<int64_t>(1, P.nwords)));
    RR_CUDA(cudaMalloc(&P.psum, sizeof(double) * std::max<int64_t>(1, P.npieces)));
    RR_CUDA(cudaMalloc(&P.xq, sizeof(double) * n_inner));
    RR_LAUNCH(k_fill_pieces, grid_for(nseg, kWarps), kThreads, 0, st, n_outer, P.nb, P.W,
              outer_ptr, inner, word_off, piece_off, pieces, slot_base, P.pw, P.slot,
              reinterpret_cast<uint16_t *>(P.idx));
    const int32_t last = (int32_t)P.nwords;
    RR_CUDA(cudaMemcpyAsync(P.pw + P.npieces, &last, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    RR_LAUNCH(k_to_i32, grid_for(n_outer + 1, kThreads), kThreads, 0, st, n_outer + 1, slot_base,
              P.slot_ptr);
    {   // outer indices with more than kLightSlots slots (summed one warp each)
      std::vector<int32_t> sp(n_outer + 1), hv;
      RR_CUDA(cudaMemcpyAsync(sp.data(), P.slot_ptr, sizeof(int32_t) * (n_outer + 1),
                              cudaMemcpyDeviceToHost, st));
      RR_CUDA(cudaStreamSynchronize(st));
      for (int64_t o = 0; o < n_outer; ++o)
        if (sp[o + 1] - sp[o] > kLightSlots) hv.push_back((int32_t)o);
      P.n_heavy = (int32_t)hv.size();
      RR_CUDA(cudaMalloc(&P.heavy, sizeof(int32_t) * std::max<size_t>(1, hv.size())));
      if (!hv.empty())
        RR_CUDA(cudaMemcpyAsync(P.heavy, hv.data(), sizeof(int32_t) * hv.size(),
                                cudaMemcpyHostToDevice, st));
    }
    // tasks: about two CTAs per SM in total, given to the slices in proportion
    // to their words (at least one each), so that the tasks are of one size
    std::vector<int32_t> task_base(P.nb + 1, 0);
    {
      std::vector<int64_t> wsl(P.nb + 1);
      for (int32_t b = 0; b <= P.nb; ++b)
        RR_CUDA(cudaMemcpyAsync(&wsl[b], word_off + (int64_t)b * n_outer, sizeof(int64_t),
                                cudaMemcpyDeviceToHost, st));
      RR_CUDA(cudaStreamSynchronize(st));
      const double per_task = (double)std::max<int64_t>(1, P.nwords) / (2.0 * kSMs);
      for (int32_t b = 0; b < P.nb; ++b) {
        const int64_t t = llround((double)(wsl[b + 1] - wsl[b]) / per_task);
        task_base[b + 1] = task_base[b] + (int32_t)std::max<int64_t>(1, t);
      }
    }
    P.ntasks = task_base[P.nb];
    RR_CUDA(cudaMalloc(&P.task_slice, sizeof(int32_t) * P.ntasks));
    RR_CUDA(cudaMalloc(&P.task_p, sizeof(int32_t) * (P.ntasks + 1)));
    int32_t *d_base = nullptr;
    RR_CUDA(cudaMalloc(&d_base, sizeof(int32_t) * (P.nb + 1)));
    RR_CUDA(cudaMemcpyAsync(d_base, task_base.data(), sizeof(int32_t) * (P.nb + 1),
                            cudaMemcpyHostToDevice, st));
    RR_LAUNCH(k_tasks, grid_for(P.ntasks + 1, kThreads), kThreads, 0, st, P.nb, d_base, n_outer,
              word_off, piece_off, P.pw, P.task_slice, P.task_p);
    RR_CUDA(cudaStreamSynchronize(st));
    cudaFree(d_base);
    RR_CUDA(cudaMalloc(&P.order, sizeof(int32_t) * std::max<int64_t>(1, P.npieces)));
    RR_LAUNCH(k_order_pieces, P.ntasks, kThreads, 0, st, P.task_p, P.pw, P.order);
    // chunks of the staged (FP32) gather, when its shared memory fits
    if (chunks && staged_smem(P.W) <= 227 * 1024) {
      int64_t *cbuf = nullptr;
      const int64_t nt1 = (int64_t)P.ntasks + 1;
      RR_CUDA(cudaMalloc(&cbuf, sizeof(int64_t) * (2 * nt1 + scan_scratch_len(nt1) + 8)));
      int64_t *ccnt = cbuf, *coff = cbuf + nt1, *cscr = cbuf + 2 * nt1;
      rr_status cs = RR_OK;
      auto chunks = [&]() -> rr_status {
        RR_LAUNCH(k_chunk_count, grid_for(P.ntasks, kThreads), kThreads, 0, st, P.ntasks, P.task_p,
                  P.pw, ccnt);
        RR_TRY(scan_exclusive(ccnt, coff, P.ntasks, cscr, st));
        int64_t nch = 0;
        RR_CUDA(cudaMemcpyAsync(&nch, coff + P.ntasks, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        RR_CUDA(cudaStreamSynchronize(st));
        P.n_chunks = nch;
        RR_CUDA(cudaMalloc(&P.chunk_p, sizeof(int32_t) * (nch + 1)));
        RR_CUDA(cudaMalloc(&P.chunk_w, sizeof(int32_t) * (nch + 1)));
        RR_CUDA(cudaMalloc(&P.task_c, sizeof(int32_t) * (P.ntasks + 1)));
        RR_LAUNCH(k_chunk_fill, grid_for(P.ntasks, kThreads), kThreads, 0, st, P.ntasks, P.task_p,
                  P.pw, coff, P.chunk_p, P.chunk_w, P.task_c, nch, (int32_t)P.npieces);
        RR_LAUNCH(k_balance_words,
                  (unsigned)std::max<int64_t>(1, std::min<int64_t>((nch * (kChunkWords / 32) + kBalThreads - 1) / kBalThreads, 1 << 20)),
                  kBalThreads, 0, st, nch, P.chunk_w, P.W, P.idx);
        RR_CUDA(cudaStreamSynchronize(st));
        return RR_OK;
      };
      cs = chunks();
      cudaFree(cbuf);
      RR_TRY(cs);
    }
    RR_CUDA(cudaStreamSynchronize(st));
    return RR_OK;
  };
  s = run();
  cudaFree(buf);
  if (s != RR_OK) sliced_free(P);
  return s;
}

void sliced_free(SlicedPattern &P) {
  cudaFree(P.pw);
  cudaFree(P.slot);
  cudaFree(P.slot_ptr);
  cudaFree(P.idx);
  cudaFree(P.psum);
  cudaFree(P.task_slice);
  cudaFree(P.task_p);
  cudaFree(P.order);
  cudaFree(P.chunk_p);
  cudaFree(P.chunk_w);
  cudaFree(P.heavy);
  cudaFree(P.task_c);
  cudaFree(P.xq);
  cudaFree(P.wmeta);
  cudaFree(P.wstart);
  P = SlicedPattern{};
}

rr_status sliced_gather(const SlicedPattern &P, const double *x, const SlicedPattern *in,
                        const int32_t *stop, cudaStream_t st, bool fp32, bool x32_ready) {
  return fp32 ? gather_t<float>(P, x, in, stop, st, x32_ready)
              : gather_t<double>(P, x, in, stop, st, false);
}

rr_status sliced_build_stream(SlicedPattern &P, cudaStream_t st) {
  if (!P.psum32) {
    rr_set_error("sliced_build_stream: the streaming gather stores FP32 piece sums");
    return RR_UNSUPPORTED;
  }
  RR_CUDA(cudaMalloc(&P.wmeta, sizeof(int32_t) * std::max<int64_t>(1, P.nwords)));
  RR_CUDA(cudaMalloc(&P.wstart, sizeof(int32_t) * (size_t)P.ntasks * 33));
  RR_CUDA(cudaMemsetAsync(P.wmeta, 0xFF, sizeof(int32_t) * std::max<int64_t>(1, P.nwords), st));
  if (P.npieces > 0)
    RR_LAUNCH(k_word_meta, grid_for(P.npieces, kThreads), kThreads, 0, st, P.npieces, P.pw, P.slot,
              P.wmeta);
  RR_LAUNCH(k_warp_ranges, grid_for((int64_t)P.ntasks * 33, kThreads), kThreads, 0, st, P.ntasks,
            P.task_p, P.pw, P.wstart);
  // the words' offsets ordered for the streaming gather's reads
  std::vector<int32_t> ws((size_t)P.ntasks * (kStreamRanges + 1));
  RR_CUDA(cudaMemcpyAsync(ws.data(), P.wstart, sizeof(int32_t) * ws.size(), cudaMemcpyDeviceToHost,
                          st));
  RR_CUDA(cudaStreamSynchronize(st));
  int32_t max_words = 0;
  for (int32_t t = 0; t < P.ntasks; ++t)
    for (int r = 0; r < kStreamRanges; ++r)
      max_words = std::max(max_words, ws[(size_t)t * (kStreamRanges + 1) + r + 1] -
                                          ws[(size_t)t * (kStreamRanges + 1) + r]);
  const int64_t n_ranges = (int64_t)P.ntasks * kStreamRanges;
  const int32_t max_steps = (max_words + 63) / 64;
  if (max_steps > 0) {
    const int64_t groups = n_ranges * max_steps * 2;
    RR_LAUNCH(k_balance_stream,
              (unsigned)std::min<int64_t>((groups + kBalThreads - 1) / kBalThreads, 1 << 20),
              kBalThreads, 0, st, n_ranges, max_steps, P.wstart, P.W, P.idx);
  }
  RR_CUDA(cudaStreamSynchronize(st));
  return RR_OK;
}

rr_status sliced_choose_gather(SlicedPattern &P, int32_t mode, cudaStream_t st) {
  if (!P.chunk_p || mode == RR_GATHER_LANES) {
    P.staged = false;
    return RR_OK;
  }
  if (mode == RR_GATHER_STAGED) {
    P.staged = true;
    return RR_OK;
  }
  // time both (after one untimed run each) on the FP32 copy of a zero vector
  RR_CUDA(cudaMemsetAsync(P.xq, 0, sizeof(float) * P.n_inner, st));
  float best[2] = {0.f, 0.f};
  cudaEvent_t e0, e1;
  RR_CUDA(cudaEventCreate(&e0));
  RR_CUDA(cudaEventCreate(&e1));
  rr_status s = RR_OK;
  for (int v = 0; v < 2 && s == RR_OK; ++v) {
    P.staged = v == 1;
    for (int rep = 0; rep < 3 && s == RR_OK; ++rep) {
      if (cudaEventRecord(e0, st) != cudaSuccess) s = RR_CUDA_ERROR;
      const float *xq = reinterpret_cast<const float *>(P.xq);
      if (s == RR_OK)
        s = P.psum32 ? launch_gather<float, float>(P, xq, nullptr, st, false)
                     : launch_gather<float, double>(P, xq, nullptr, st, false);
      if (s == RR_OK && (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
                         cudaEventSynchronize(e1) != cudaSuccess))
        s = RR_CUDA_ERROR;
      float ms = 0.f;
      if (s == RR_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) s = RR_CUDA_ERROR;
      if (rep > 0) best[v] = (rep == 1) ? ms : std::min(best[v], ms);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != RR_OK) {
    rr_set_error("sliced_choose_gather: a timing launch failed");
    return s;
  }
  P.staged = best[1] < best[0];
  return RR_OK;
}

rr_status sliced_slot_sum(const SlicedPattern &P, double *out, cudaStream_t st) {
  RR_LAUNCH_PDL(k_slot_sum, grid_for(P.n_outer, kThreads), kThreads, 0, st, P.n_outer, P.slot_ptr,
            P.psum, out);
  return RR_OK;
}

rr_status sliced_epilogue(const SlicedPattern &P, const CscEpilogue &ep, cudaStream_t st) {
  RR_LAUNCH_PDL(k_sliced_epilogue, kVecGrid, kThreads, 0, st, P.n_outer, P.slot_ptr, P.psum, P.heavy,
            P.n_heavy, ep);
  return RR_OK;
}

}  // namespace rr
