// Sliced mat-vecs of binary X, the per-iteration hot loop of Eq. (1)'s
// operator: u = X v (rows gather v) and X^T u (columns gather u).
//
// Layout ("sliced pattern"): the gathered dimension is cut into nb slices of
// at most kSliceMax entries, so a slice of the FP64 vector fits in shared
// memory; inside a slice an index is a 16-bit offset (half the bytes of an
// int32 index). The entries of every (outer index, slice) segment are padded
// to whole 16-byte words (8 offsets; the pad offset W reads a zero kept in
// shared memory) and the segment is cut into pieces of at most kPieceWords
// words. Pieces are stored slice-major, so one CTA streams a contiguous range
// of them against the one vector slice it holds; each piece is summed by one
// lane (in a fixed order) into its own slot, numbered outer-major, and the
// slots of one outer index are summed afterwards in a fixed order. No atomics:
// every run gives identical bits.
#include "common.cuh"
#include "kernels.h"

namespace rr {

namespace {

constexpr int kSliceThreads = 1024;

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
    uint16_t *dst = idx + w0 * 8;
    for (int64_t u = lane; u < nw * 8; u += 32)
      dst[u] = u < len ? (uint16_t)(inner[s + u] - key) : (uint16_t)W;
  }
}

// task t of slice b starts at the first piece whose start word reaches
// word_begin(b) + t * words(b) / T
__global__ void k_tasks(int32_t nb, int32_t T, int64_t n_outer, const int64_t *__restrict__ word_off,
                        const int64_t *__restrict__ piece_off, const int32_t *__restrict__ pw,
                        int32_t *__restrict__ task_slice, int32_t *__restrict__ task_p) {
  const int32_t total = nb * T;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= total; i += gridDim.x * blockDim.x) {
    if (i == total) {
      task_p[total] = (int32_t)piece_off[(int64_t)nb * n_outer];
      continue;
    }
    const int32_t b = i / T, t = i % T;
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

// Pre-pass: the gathered vector, once per pass, in the accumulation type T
// (FP64, or FP32 for the mixed-precision inner iterations). v = x, or
// (kCombine) the per-index sums of the previous pass's slots.
template <bool kCombine, typename T>
__global__ void k_slice_prep(int64_t n, const double *__restrict__ x,
                             const double *__restrict__ in_psum,
                             const int32_t *__restrict__ in_slot_ptr, T *__restrict__ xq,
                             const int32_t *__restrict__ stop) {
  if (stop && *stop) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v;
    if (kCombine) {
      v = 0.0;
      for (int32_t q = in_slot_ptr[i]; q < in_slot_ptr[i + 1]; ++q) v += in_psum[q];
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
// Sums in a fixed order in T; the piece sum is stored in FP64.
template <typename T>
__global__ void __launch_bounds__(kSliceThreads, 1) k_sliced_gather(
    SlicedView P, const T *__restrict__ xq, double *__restrict__ out_psum,
    const int32_t *__restrict__ stop) {
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
    int32_t w0[kILP], w1[kILP];
    uint4 first[kILP];
#pragma unroll
    for (int u = 0; u < kILP; ++u) {
      const int32_t p = pb + u * kSliceThreads;
      w0[u] = p < p1 ? __ldg(P.pw + p) : 0;
      w1[u] = p < p1 ? __ldg(P.pw + p + 1) : 0;
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
      out_psum[__ldg(P.slot + p)] = (double)acc;
    }
  }
}

// Sum of the slots of every outer index -> out[o] (u = X v on its own).
__global__ void k_slot_sum(int64_t n, const int32_t *__restrict__ slot_ptr,
                           const double *__restrict__ psum, double *__restrict__ out) {
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n;
       o += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int32_t q = slot_ptr[o]; q < slot_ptr[o + 1]; ++q) v += psum[q];
    out[o] = v;
  }
}

__device__ __forceinline__ void epilogue(const CscEpilogue &ep, int64_t i, double sum, double &dot) {
  switch (ep.mode) {
    case CSC_RHS:
      ep.out[i] = sum;
      break;
    case CSC_APPLY:
      ep.out[i] = sum + ep.lambda * ep.v[i];
      break;
    case CSC_PRE:
      ep.out[i] = ep.r[i] - (sum + ep.lambda * ep.v[i]);
      break;
    case CSC_POST: {
      const double r2 = ep.r[i] - (sum + ep.lambda * ep.v[i]);
      const double z = ep.v[i] + ep.omega * r2 / ep.d[i];
      ep.out[i] = z;
      dot += ep.r[i] * z;
      break;
    }
    case CSC_PCG: {
      const double t = sum + ep.lambda * ep.v[i];
      ep.out[i] = t;
      dot += ep.v[i] * t;
      break;
    }
    default: {  // CSC_RESID
      const double t = ep.r[i] - (sum + ep.lambda * ep.v[i]);
      ep.out[i] = t;
      dot += t * t;
      break;
    }
  }
}

// One 8-lane group per feature: t_i = sum of its slots; then the mode's epilogue;
// per-block partial dots in a fixed order.
__global__ void __launch_bounds__(kThreads) k_sliced_epilogue(int64_t F, const int32_t *__restrict__ slot_ptr,
                                                              const double *__restrict__ psum,
                                                              CscEpilogue ep) {
  if (ep.stop && *ep.stop) return;
  __shared__ double sm[kWarps + 1];
  const int lane8 = threadIdx.x & 7, gw = (threadIdx.x >> 3) & 3;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double dot = 0.0;
  for (int64_t i0 = warp * 4; i0 < F; i0 += nwarps * 4) {   // warp-uniform loop
    const int64_t i = i0 + gw;
    double s = 0.0;
    if (i < F)
      for (int32_t q = slot_ptr[i] + lane8; q < slot_ptr[i + 1]; q += 8) s += psum[q];
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    if (i < F && lane8 == 0) epilogue(ep, i, s, dot);
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

template <typename T>
rr_status set_smem_attr() {
  static bool done = false;
  if (!done) {
    RR_CUDA(cudaFuncSetAttribute(k_sliced_gather<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)slice_smem<T>(kSliceMax)));
    done = true;
  }
  return RR_OK;
}

template <typename T>
rr_status gather_t(const SlicedPattern &P, const double *x, const SlicedPattern *in,
                   const int32_t *stop, cudaStream_t st) {
  const int64_t n = P.n_inner;
  T *xq = reinterpret_cast<T *>(P.xq);
  if (in)
    RR_LAUNCH((k_slice_prep<true, T>), grid_for(n, kThreads), kThreads, 0, st, n, nullptr,
              in->psum, in->slot_ptr, xq, stop);
  else
    RR_LAUNCH((k_slice_prep<false, T>), grid_for(n, kThreads), kThreads, 0, st, n, x, nullptr,
              nullptr, xq, stop);
  RR_TRY(set_smem_attr<T>());
  RR_LAUNCH(k_sliced_gather<T>, P.ntasks, kSliceThreads, slice_smem<T>(P.W), st, P.view(), xq,
            P.psum, stop);
  return RR_OK;
}

}  // namespace

rr_status sliced_build(int64_t n_outer, int64_t n_inner, const int64_t *outer_ptr,
                       const int32_t *inner, SlicedPattern &P, cudaStream_t st) {
  P = SlicedPattern{};
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
    RR_CUDA(cudaMalloc(&P.pw, sizeof(int32_t) * (P.npieces + 1)));
    RR_CUDA(cudaMalloc(&P.slot, sizeof(int32_t) * std::max<int64_t>(1, P.npieces)));
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
    // tasks: about two CTAs per SM in total, split evenly over the slices
    P.tasks_per_slice = std::max<int32_t>(1, (2 * kSMs + P.nb - 1) / P.nb);
    P.ntasks = P.nb * P.tasks_per_slice;
    RR_CUDA(cudaMalloc(&P.task_slice, sizeof(int32_t) * P.ntasks));
    RR_CUDA(cudaMalloc(&P.task_p, sizeof(int32_t) * (P.ntasks + 1)));
    RR_LAUNCH(k_tasks, grid_for(P.ntasks + 1, kThreads), kThreads, 0, st, P.nb,
              P.tasks_per_slice, n_outer, word_off, piece_off, P.pw, P.task_slice, P.task_p);
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
  cudaFree(P.xq);
  P = SlicedPattern{};
}

rr_status sliced_gather(const SlicedPattern &P, const double *x, const SlicedPattern *in,
                        const int32_t *stop, cudaStream_t st, bool fp32) {
  return fp32 ? gather_t<float>(P, x, in, stop, st) : gather_t<double>(P, x, in, stop, st);
}

rr_status sliced_slot_sum(const SlicedPattern &P, double *out, cudaStream_t st) {
  RR_LAUNCH(k_slot_sum, grid_for(P.n_outer, kThreads), kThreads, 0, st, P.n_outer, P.slot_ptr,
            P.psum, out);
  return RR_OK;
}

rr_status sliced_epilogue(const SlicedPattern &P, const CscEpilogue &ep, cudaStream_t st) {
  RR_LAUNCH(k_sliced_epilogue, kVecGrid, kThreads, 0, st, P.n_outer, P.slot_ptr, P.psum, ep);
  return RR_OK;
}

}  // namespace rr
