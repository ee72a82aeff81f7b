// The matrix-free operator of Eq. (1): u = X v (CSR) and X^T u + lambda v
// (transposed copy, CSC), binary X, FP64 vectors. The transposed product is
// cut into pieces of at most kCscChunk nonzeros so the power-law heavy
// columns do not serialise on one warp; it carries the epilogues that the
// PCG iteration needs (residual updates, smoother, dot products), each dot
// reduced in a fixed order so repeated runs give identical bits.
#include "common.cuh"
#include "kernels.h"

namespace rr {

namespace {

// One warp per row; four independent index loads in flight per lane.
__global__ void __launch_bounds__(kThreads) k_csr_spmv(int64_t N, const int64_t *__restrict__ row_ptr,
                                                       const int32_t *__restrict__ col_idx,
                                                       const double *__restrict__ v,
                                                       double *__restrict__ u,
                                                       const int32_t *__restrict__ stop) {
  if (stop && *stop) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < N; r += nwarps) {
    const int64_t b = row_ptr[r], e = row_ptr[r + 1];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int64_t p = b + lane;
    for (; p + 96 < e; p += 128) {
      const int32_t c0 = __ldg(col_idx + p), c1 = __ldg(col_idx + p + 32);
      const int32_t c2 = __ldg(col_idx + p + 64), c3 = __ldg(col_idx + p + 96);
      s0 += __ldg(v + c0);
      s1 += __ldg(v + c1);
      s2 += __ldg(v + c2);
      s3 += __ldg(v + c3);
    }
    for (; p < e; p += 32) s0 += __ldg(v + __ldg(col_idx + p));
    const double s = warp_sum((s0 + s1) + (s2 + s3));
    if (lane == 0) u[r] = s;
  }
}

__device__ __forceinline__ double csc_epilogue(const CscEpilogue &ep, int64_t i, double sum,
                                               double &dot) {
  switch (ep.mode) {
    case CSC_RHS:
      ep.out[i] = sum;
      return 0.0;
    case CSC_APPLY:
      ep.out[i] = sum + ep.lambda * ep.v[i];
      return 0.0;
    case CSC_PRE:
      ep.out[i] = ep.r[i] - (sum + ep.lambda * ep.v[i]);
      return 0.0;
    case CSC_POST: {
      const double r2 = ep.r[i] - (sum + ep.lambda * ep.v[i]);
      const double z = ep.v[i] + ep.omega * r2 / ep.d[i];
      ep.out[i] = z;
      dot += ep.r[i] * z;
      return 0.0;
    }
    case CSC_PCG: {
      const double t = sum + ep.lambda * ep.v[i];
      ep.out[i] = t;
      dot += ep.v[i] * t;
      return 0.0;
    }
    default: {  // CSC_RESID
      const double t = ep.r[i] - (sum + ep.lambda * ep.v[i]);
      ep.out[i] = t;
      dot += t * t;
      return 0.0;
    }
  }
}

// Pass 1: one warp per piece. Single-piece columns finish here.
__global__ void __launch_bounds__(kThreads) k_csc_pieces(int64_t n_items, const CscItem *__restrict__ items,
                                                         const int32_t *__restrict__ row_idx,
                                                         const double *__restrict__ u,
                                                         double *__restrict__ slot_sum,
                                                         CscEpilogue ep) {
  if (ep.stop && *ep.stop) return;
  __shared__ double sm[kWarps + 1];
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double dot = 0.0;
  for (int64_t it = warp; it < n_items; it += nwarps) {
    const CscItem item = items[it];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int64_t p = item.begin + lane;
    for (; p + 96 < item.end; p += 128) {
      const int32_t r0 = __ldg(row_idx + p), r1 = __ldg(row_idx + p + 32);
      const int32_t r2 = __ldg(row_idx + p + 64), r3 = __ldg(row_idx + p + 96);
      s0 += __ldg(u + r0);
      s1 += __ldg(u + r1);
      s2 += __ldg(u + r2);
      s3 += __ldg(u + r3);
    }
    for (; p < item.end; p += 32) s0 += __ldg(u + __ldg(row_idx + p));
    const double s = warp_sum((s0 + s1) + (s2 + s3));
    if (lane == 0) {
      if (item.slot >= 0)
        slot_sum[item.slot] = s;
      else
        csc_epilogue(ep, item.col, s, dot);
    }
  }
  const double tot = block_sum(lane == 0 ? dot : 0.0, sm);
  if (threadIdx.x == 0 && ep.dot_part) ep.dot_part[blockIdx.x] = tot;
}

// Pass 2: one warp per multi-piece column; sums its pieces in order.
__global__ void __launch_bounds__(kThreads) k_csc_heavy(int64_t n_heavy, const int32_t *__restrict__ heavy_col,
                                                        const int32_t *__restrict__ heavy_first,
                                                        const int32_t *__restrict__ heavy_n,
                                                        const double *__restrict__ slot_sum,
                                                        CscEpilogue ep, int part_offset) {
  if (ep.stop && *ep.stop) return;
  __shared__ double sm[kWarps + 1];
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double dot = 0.0;
  for (int64_t h = warp; h < n_heavy; h += nwarps) {
    const int32_t first = heavy_first[h], n = heavy_n[h];
    double s = 0.0;
    for (int q = lane; q < n; q += 32) s += slot_sum[first + q];
    s = warp_sum(s);
    if (lane == 0) csc_epilogue(ep, heavy_col[h], s, dot);
  }
  const double tot = block_sum(lane == 0 ? dot : 0.0, sm);
  if (threadIdx.x == 0 && ep.dot_part) ep.dot_part[part_offset + blockIdx.x] = tot;
}

__global__ void k_plan_counts(int64_t F, const int64_t *__restrict__ col_ptr,
                              int64_t *__restrict__ pieces, int64_t *__restrict__ slots,
                              int64_t *__restrict__ heavy) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < F;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = col_ptr[j + 1] - col_ptr[j];
    const int64_t np = m <= kCscChunk ? 1 : (m + kCscChunk - 1) / kCscChunk;
    pieces[j] = np;
    slots[j] = np > 1 ? np : 0;
    heavy[j] = np > 1 ? 1 : 0;
  }
}

__global__ void k_plan_fill(int64_t F, const int64_t *__restrict__ col_ptr,
                            const int64_t *__restrict__ item_off, const int64_t *__restrict__ slot_off,
                            const int64_t *__restrict__ heavy_off, CscItem *__restrict__ items,
                            int32_t *__restrict__ heavy_col, int32_t *__restrict__ heavy_first,
                            int32_t *__restrict__ heavy_n) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < F;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = col_ptr[j], e = col_ptr[j + 1];
    const int64_t np = item_off[j + 1] - item_off[j];
    for (int64_t q = 0; q < np; ++q) {
      CscItem it;
      it.begin = b + q * kCscChunk;
      it.end = min(e, it.begin + kCscChunk);
      it.col = (int32_t)j;
      it.slot = np > 1 ? (int32_t)(slot_off[j] + q) : -1;
      items[item_off[j] + q] = it;
    }
    if (np > 1) {
      const int64_t h = heavy_off[j];
      heavy_col[h] = (int32_t)j;
      heavy_first[h] = (int32_t)slot_off[j];
      heavy_n[h] = (int32_t)np;
    }
  }
}

constexpr int kPiecesGrid = kSMs * 8;
constexpr int kHeavyGrid = kSMs;

}  // namespace

rr_status csc_plan_build(int64_t F, const int64_t *col_ptr, CscPlan &plan, cudaStream_t st) {
  int64_t *buf = nullptr;
  const int64_t ss = scan_scratch_len(F) + 8;
  RR_CUDA(cudaMalloc(&buf, sizeof(int64_t) * (6 * (F + 1) + ss)));
  int64_t *pieces = buf, *slots = buf + (F + 1), *heavy = buf + 2 * (F + 1);
  int64_t *item_off = buf + 3 * (F + 1), *slot_off = buf + 4 * (F + 1),
          *heavy_off = buf + 5 * (F + 1), *scr = buf + 6 * (F + 1);
  rr_status s = RR_OK;
  int64_t tot[3] = {0, 0, 0};
  do {
    if ((s = [&]() -> rr_status {
           RR_LAUNCH(k_plan_counts, grid_for(F, kThreads), kThreads, 0, st, F, col_ptr, pieces, slots,
                     heavy);
           return RR_OK;
         }()) != RR_OK)
      break;
    if ((s = scan_exclusive(pieces, item_off, F, scr, st)) != RR_OK) break;
    if ((s = scan_exclusive(slots, slot_off, F, scr, st)) != RR_OK) break;
    if ((s = scan_exclusive(heavy, heavy_off, F, scr, st)) != RR_OK) break;
    cudaMemcpyAsync(&tot[0], item_off + F, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&tot[1], slot_off + F, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&tot[2], heavy_off + F, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      rr_set_error("csc_plan_build: synchronise failed");
      s = RR_CUDA_ERROR;
      break;
    }
    plan.n_items = tot[0];
    plan.n_slots = tot[1];
    plan.n_heavy = tot[2];
    if (cudaMalloc(&plan.items, sizeof(CscItem) * std::max<int64_t>(1, plan.n_items)) != cudaSuccess ||
        cudaMalloc(&plan.heavy_col, sizeof(int32_t) * std::max<int64_t>(1, plan.n_heavy)) != cudaSuccess ||
        cudaMalloc(&plan.heavy_first, sizeof(int32_t) * std::max<int64_t>(1, plan.n_heavy)) != cudaSuccess ||
        cudaMalloc(&plan.heavy_n, sizeof(int32_t) * std::max<int64_t>(1, plan.n_heavy)) != cudaSuccess ||
        cudaMalloc(&plan.slot_sum, sizeof(double) * std::max<int64_t>(1, plan.n_slots)) != cudaSuccess) {
      rr_set_error("csc_plan_build: out of device memory");
      s = RR_OOM;
      break;
    }
    s = [&]() -> rr_status {
      RR_LAUNCH(k_plan_fill, grid_for(F, kThreads), kThreads, 0, st, F, col_ptr, item_off, slot_off,
                heavy_off, plan.items, plan.heavy_col, plan.heavy_first, plan.heavy_n);
      return RR_OK;
    }();
    if (s == RR_OK && cudaStreamSynchronize(st) != cudaSuccess) s = RR_CUDA_ERROR;
  } while (false);
  cudaFree(buf);
  return s;
}

void csc_plan_free(CscPlan &plan) {
  cudaFree(plan.items);
  cudaFree(plan.heavy_col);
  cudaFree(plan.heavy_first);
  cudaFree(plan.heavy_n);
  cudaFree(plan.slot_sum);
  plan = CscPlan{};
}

int csc_dot_parts(const CscPlan &plan) {
  (void)plan;
  return kPiecesGrid + kHeavyGrid;
}

rr_status csr_spmv(int64_t N, const int64_t *row_ptr, const int32_t *col_idx, const double *v,
                   double *u, const int32_t *stop, cudaStream_t st) {
  if (N == 0) return RR_OK;
  RR_LAUNCH(k_csr_spmv, grid_for(N, kWarps), kThreads, 0, st, N, row_ptr, col_idx, v, u, stop);
  return RR_OK;
}

rr_status csc_spmv(int64_t F, const int32_t *row_idx, const double *u, const CscPlan &plan,
                   const CscEpilogue &ep, cudaStream_t st) {
  (void)F;
  RR_LAUNCH(k_csc_pieces, kPiecesGrid, kThreads, 0, st, plan.n_items, plan.items, row_idx, u,
            plan.slot_sum, ep);
  RR_LAUNCH(k_csc_heavy, kHeavyGrid, kThreads, 0, st, plan.n_heavy, plan.heavy_col,
            plan.heavy_first, plan.heavy_n, plan.slot_sum, ep, kPiecesGrid);
  return RR_OK;
}

}  // namespace rr
