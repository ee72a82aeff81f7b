// Preconditioner pieces and CG recurrences (FP64).
//  restriction  r_c = P^T r1, r_c[S] = s_S * sum_{i in S} r1[i]   (Eq. (prolong))
//  coarse solve e_c = A_c^{-1} r_c with the explicit inverse of the Cholesky factor
//  prolongation z2 = z1 + P e_c
//  smoother     z = omega D^{-1} r
//  CG           Hestenes-Stiefel recurrences from x_0 = 0, r_0 = b (Algorithm 3's
//               initialisation), stopping on ||r|| <= tol ||b|| (Section 4's residual).
// Every scalar is a fixed-order sum of per-block partials; each consuming block
// recomputes it, so no extra finishing kernel is needed and runs are bitwise
// repeatable. The scalar state lives on the device (PcgScalars); once
// `converged` is set every later kernel of the loop returns at once.
#include "common.cuh"
#include "kernels.h"

namespace rr {

namespace {

// Restriction, pass 1: one warp per work item, an item being a range of at
// most kRestrictItem members of one cluster (large clusters have several);
// the lanes stride over the members with four loads in flight, then a fixed
// shuffle tree.
__global__ void k_restrict_items(const RestrictItem *__restrict__ items, int32_t n_items,
                                 const int32_t *__restrict__ members, const double *__restrict__ r1,
                                 double *__restrict__ item_sum, const int32_t *__restrict__ stop) {
  pdl_wait();
  if (stop && *stop) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = warp; it < n_items; it += nwarps) {
    const RestrictItem w = items[it];
    double acc = 0.0;
    for (int32_t m0 = w.begin + lane; m0 < w.end; m0 += 4 * 32) {
      double t[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int32_t m = m0 + 32 * u;
        t[u] = m < w.end ? r1[members[m]] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) acc += t[u];
    }
    acc = warp_sum(acc);
    if (lane == 0) item_sum[it] = acc;
  }
}

// Restriction, pass 2: r_c[S] = s_S * (the item sums of S), one warp per
// cluster, lanes strided over the items, a fixed shuffle tree.
__global__ void k_restrict_combine(int32_t k, const int32_t *__restrict__ item_ptr,
                                   const double *__restrict__ item_sum,
                                   const double *__restrict__ s, double *__restrict__ rc,
                                   const int32_t *__restrict__ stop) {
  pdl_wait();
  if (stop && *stop) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t S = warp; S < k; S += nwarps) {
    double acc = 0.0;
    for (int32_t q = item_ptr[S] + lane; q < item_ptr[S + 1]; q += 32) acc += item_sum[q];
    acc = warp_sum(acc);
    if (lane == 0) rc[S] = s[S] * acc;
  }
}

// The coarse solve e_c = Ainv r_c with r_c staged in shared memory: r_c from
// the item sums (r_c[S] = s_S * (sum of the item sums of S, in order)), or,
// with item_ptr == nullptr, item_sum itself.
// With item_ptr == nullptr the input vector is item_sum itself (a plain
// mat-vec ec = Ainv x); with scale, ec[S] is multiplied by scale[S].
__global__ void k_coarse_matvec(int32_t k, const double *__restrict__ Ainv,
                                const int32_t *__restrict__ item_ptr,
                                const double *__restrict__ item_sum, const double *__restrict__ s,
                                double *__restrict__ rc_out, double *__restrict__ ec,
                                const int32_t *__restrict__ stop,
                                const double *__restrict__ scale) {
  pdl_wait();
  if (stop && *stop) return;
  extern __shared__ double rcs[];
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    double v;
    if (item_ptr) {
      double acc = 0.0;
      for (int32_t q = item_ptr[i]; q < item_ptr[i + 1]; ++q) acc += item_sum[q];
      v = s[i] * acc;
    } else {
      v = item_sum[i];
    }
    rcs[i] = v;
    if (blockIdx.x == 0 && rc_out) rc_out[i] = v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t S = warp; S < k; S += nwarps) {
    const double *row = Ainv + S * k;
    // four row loads in flight per lane; the four partial sums are added in a fixed order
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int t = lane;
    // eight row loads in flight per lane (issued before the products)
    for (; t + 224 < k; t += 256) {
      double r8[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) r8[u] = row[t + 32 * u];
      a0 += r8[0] * rcs[t];
      a1 += r8[1] * rcs[t + 32];
      a2 += r8[2] * rcs[t + 64];
      a3 += r8[3] * rcs[t + 96];
      a0 += r8[4] * rcs[t + 128];
      a1 += r8[5] * rcs[t + 160];
      a2 += r8[6] * rcs[t + 192];
      a3 += r8[7] * rcs[t + 224];
    }
    for (; t + 96 < k; t += 128) {
      a0 += row[t] * rcs[t];
      a1 += row[t + 32] * rcs[t + 32];
      a2 += row[t + 64] * rcs[t + 64];
      a3 += row[t + 96] * rcs[t + 96];
    }
    for (; t < k; t += 32) a0 += row[t] * rcs[t];
    double acc = (a0 + a1) + (a2 + a3);
    acc = warp_sum(acc);
    if (lane == 0) ec[S] = scale ? acc * scale[S] : acc;
  }
}

// The same coarse step in FP32 (the FP32 inner iterations' preconditioner):
// r_c staged as FP32, Ainv32 (FP32 copy of the FP64 inverse, k padded to a
// multiple of 4 per row: ld) read four entries per load, FP32 products and
// sums, e_c stored in FP64.
__global__ void k_coarse_matvec32(int32_t k, int32_t ld, const float *__restrict__ Ainv32,
                                  const double *__restrict__ rc, double *__restrict__ ec,
                                  const int32_t *__restrict__ stop) {
  pdl_wait();
  if (stop && *stop) return;
  extern __shared__ float rcs32[];
  for (int i = threadIdx.x; i < ld; i += blockDim.x) rcs32[i] = i < k ? (float)rc[i] : 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float4 *x4 = reinterpret_cast<const float4 *>(rcs32);
  for (int64_t S = warp; S < k; S += nwarps) {
    const float4 *row = reinterpret_cast<const float4 *>(Ainv32 + S * ld);
    float a0 = 0.f, a1 = 0.f;
    int t = lane;
    for (; t + 32 < ld / 4; t += 64) {
      const float4 r0 = __ldg(row + t), r1 = __ldg(row + t + 32);
      const float4 v0 = x4[t], v1 = x4[t + 32];
      a0 += r0.x * v0.x + r0.y * v0.y + r0.z * v0.z + r0.w * v0.w;
      a1 += r1.x * v1.x + r1.y * v1.y + r1.z * v1.z + r1.w * v1.w;
    }
    for (; t < ld / 4; t += 32) {
      const float4 r0 = __ldg(row + t), v0 = x4[t];
      a0 += r0.x * v0.x + r0.y * v0.y + r0.z * v0.z + r0.w * v0.w;
    }
    float acc = a0 + a1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) ec[S] = (double)acc;
  }
}

__global__ void k_to_f32_padded(int32_t k, int32_t ld, const double *__restrict__ A,
                                float *__restrict__ A32) {
  const int64_t n = (int64_t)k * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ld, j = e % ld;
    A32[e] = j < k ? (float)A[i * k + j] : 0.f;
  }
}

__global__ void k_restrict_plan(int32_t k, const int64_t *__restrict__ cl_ptr, int32_t item_size,
                                const int32_t *__restrict__ item_ptr, RestrictItem *__restrict__ items) {
  for (int32_t S = blockIdx.x * blockDim.x + threadIdx.x; S < k; S += gridDim.x * blockDim.x) {
    const int64_t b = cl_ptr[S], e = cl_ptr[S + 1];
    int32_t q = item_ptr[S];
    for (int64_t m = b; m < e; m += item_size, ++q)
      items[q] = RestrictItem{(int32_t)m, (int32_t)min(e, m + item_size)};
  }
}

__global__ void k_restrict_counts(int32_t k, const int64_t *__restrict__ cl_ptr, int32_t item_size,
                                  int64_t *__restrict__ cnt) {
  for (int32_t S = blockIdx.x * blockDim.x + threadIdx.x; S < k; S += gridDim.x * blockDim.x)
    cnt[S] = (cl_ptr[S + 1] - cl_ptr[S] + item_size - 1) / item_size;
}

__global__ void k_i64_to_i32(int64_t n, const int64_t *__restrict__ in, int32_t *__restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int32_t)in[i];
}

// z2 = z1 + P e_c (and, if z2_32, its FP32 copy for the next operator apply).
__global__ void k_prolong_add(int64_t F, const int32_t *__restrict__ labels,
                              const double *__restrict__ s, const double *__restrict__ ec,
                              const double *__restrict__ z1, double *__restrict__ z2,
                              float *__restrict__ z2_32, const int32_t *__restrict__ stop) {
  pdl_wait();
  if (stop && *stop) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t l = labels[i];
    const double v = z1[i] + s[l] * ec[l];
    z2[i] = v;
    if (z2_32) z2_32[i] = (float)v;
  }
}

__global__ void k_jacobi(int64_t F, double omega, const double *__restrict__ r,
                         const double *__restrict__ d, double *__restrict__ z,
                         float *__restrict__ z32, double *__restrict__ rz_part,
                         const int32_t *__restrict__ stop) {
  pdl_wait();
  if (stop && *stop) return;
  __shared__ double sm[kWarps + 1];
  double dot = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = d ? omega * r[i] / d[i] : r[i];
    z[i] = zi;
    if (z32) z32[i] = (float)zi;
    dot += r[i] * zi;
  }
  if (rz_part) {
    const double tot = block_sum(dot, sm);
    if (threadIdx.x == 0) rz_part[blockIdx.x] = tot;
  }
}

__global__ void k_pcg_direction(int64_t F, const double *__restrict__ rz_part, int n_rz,
                                const double *__restrict__ z, double *__restrict__ p,
                                float *__restrict__ p32, const PcgScalars *__restrict__ S) {
  pdl_wait();
  if (S->converged) return;
  __shared__ double sm[kWarps + 1];
  const double rho = sum_partials(rz_part, n_rz, sm);
  const double beta = S->first ? 0.0 : rho / S->rho_old;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = S->first ? z[i] : z[i] + beta * p[i];
    p[i] = v;
    if (p32) p32[i] = (float)v;
  }
}

// The update, then (in the block that arrives last) the iteration's scalars:
// rr = ||r||^2 from the blocks' partials (read through L2, in the same fixed
// order as any other sum of partials), rho_old, iter++, convergence and
// finiteness flags, the residual history.
__global__ void k_pcg_update(int64_t F, const double *__restrict__ rz_part, int n_rz,
                             const double *__restrict__ pq_part, int n_pq,
                             const double *__restrict__ p, const double *__restrict__ q,
                             double *__restrict__ w, double *__restrict__ r, double omega,
                             const double *__restrict__ d, double *__restrict__ z1,
                             float *__restrict__ z1_32, double *__restrict__ rr_part,
                             PcgScalars *S, const double *__restrict__ wd,
                             double *__restrict__ history, int32_t hist_cap) {
  pdl_wait();
  if (S->converged) return;
  __shared__ double sm[kWarps + 1];
  __shared__ int32_t last;
  const double rho = sum_partials(rz_part, n_rz, sm);
  const double pq = sum_partials(pq_part, n_pq, sm);
  const double alpha = rho / pq;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x) {
    w[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    acc += ri * ri;
    if (z1) {
      const double zi = wd ? ri * wd[i] : omega * ri / d[i];
      z1[i] = zi;
      if (z1_32) z1_32[i] = (float)zi;
    }
  }
  const double tot = block_sum(acc, sm);
  if (threadIdx.x == 0) {
    rr_part[blockIdx.x] = tot;
    __threadfence();
    last = atomicAdd(&S->arrive, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += __ldcg(&rr_part[i]);
  const double rr = block_sum(v, sm);
  if (threadIdx.x == 0) {
    S->arrive = 0;
    S->rho_old = rho;
    S->rr = rr;
    S->first = 0;
    const int32_t it = S->iter + 1;
    S->iter = it;
    const double rn = sqrt(rr);
    if (history && it <= hist_cap) history[it - 1] = rn / S->bnorm;
    if (!isfinite(rr) || !isfinite(rho)) {
      S->nonfinite = 1;
      S->converged = 1;
    } else if (rn <= S->target) {
      S->converged = 1;
    }
  }
}

__global__ void k_dot_parts(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
                            double *__restrict__ part) {
  pdl_wait();
  __shared__ double sm[kWarps + 1];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += a[i] * b[i];
  const double tot = block_sum(acc, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_pcg_start(const double *__restrict__ bb_part, int n_bb,
                            const double *__restrict__ rr_part, int n_rr, double tol,
                            int32_t set_bnorm, PcgScalars *S) {
  pdl_wait();
  __shared__ double sm[kWarps + 1];
  const double bb = sum_partials(bb_part, n_bb, sm);
  const double rr = sum_partials(rr_part, n_rr, sm);
  if (threadIdx.x == 0) {
    if (set_bnorm) {
      S->bnorm = sqrt(bb);
      S->target = tol * S->bnorm;
      S->iter = 0;
      S->nonfinite = isfinite(bb) ? 0 : 1;
    }
    S->rr = rr;
    S->rho_old = 0.0;
    S->first = 1;
    S->converged = (S->nonfinite || sqrt(rr) <= S->target) ? 1 : 0;
  }
}

// Scalars of a fixed number of plain CG steps run inside another solver's
// iteration: a fresh start (first direction), no stopping target, and stopped
// at once when the outer solver has converged.
__global__ void k_inner_start(PcgScalars *S, const int32_t *__restrict__ outer_converged) {
  pdl_wait();
  if (threadIdx.x == 0) {
    S->rho_old = 0.0;
    S->rr = 0.0;
    S->bnorm = 1.0;
    S->target = 0.0;
    S->iter = 0;
    S->nonfinite = 0;
    S->first = 1;
    S->converged = *outer_converged;
  }
}

__global__ void k_sum_parts(const double *__restrict__ part, int n, double *out) {
  pdl_wait();
  __shared__ double sm[kWarps + 1];
  const double v = sum_partials(part, n, sm);
  if (threadIdx.x == 0) *out = v;
}

__global__ void k_loop_condition(cudaGraphConditionalHandle hc, const PcgScalars *__restrict__ S) {
  pdl_wait();
  if (threadIdx.x == 0)
    cudaGraphSetConditional(hc, (!S->converged && S->iter < S->limit) ? 1u : 0u);
}

__global__ void k_axpby(int64_t n, double a, const double *__restrict__ x, double b,
                        double *__restrict__ y) {
  pdl_wait();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (x ? a * x[i] : 0.0) + (b != 0.0 ? b * y[i] : 0.0);
}

}  // namespace

rr_status restrict_plan(int32_t k, const int64_t *cl_ptr, RestrictPlan &plan, int64_t *scratch,
                        cudaStream_t st, int32_t item_size) {
  // scratch: >= 2 (k + 1) + scan scratch int64
  int64_t *cnt = scratch, *off = scratch + (k + 1), *scr = scratch + 2 * (k + 1);
  RR_LAUNCH(k_restrict_counts, grid_for(k, kThreads), kThreads, 0, st, k, cl_ptr, item_size, cnt);
  RR_TRY(scan_exclusive(cnt, off, k, scr, st));
  int64_t n = 0;
  RR_CUDA(cudaMemcpyAsync(&n, off + k, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  plan.n_items = (int32_t)n;
  plan.k = k;
  RR_CUDA(cudaMalloc(&plan.item_ptr, sizeof(int32_t) * (k + 1)));
  RR_CUDA(cudaMalloc(&plan.items, sizeof(RestrictItem) * std::max<int64_t>(1, n)));
  RR_CUDA(cudaMalloc(&plan.item_sum, sizeof(double) * std::max<int64_t>(1, n)));
  RR_CUDA(cudaMalloc(&plan.rc, sizeof(double) * std::max<int32_t>(1, k)));
  RR_LAUNCH(k_i64_to_i32, grid_for(k + 1, kThreads), kThreads, 0, st, (int64_t)k + 1, off,
            plan.item_ptr);
  RR_LAUNCH(k_restrict_plan, grid_for(k, kThreads), kThreads, 0, st, k, cl_ptr, item_size,
            plan.item_ptr, plan.items);
  RR_CUDA(cudaStreamSynchronize(st));
  return RR_OK;
}

void restrict_free(RestrictPlan &plan) {
  cudaFree(plan.item_ptr);
  cudaFree(plan.items);
  cudaFree(plan.item_sum);
  cudaFree(plan.rc);
  plan = RestrictPlan{};
}

rr_status restrict_clusters(const RestrictPlan &plan, const int32_t *members, const double *r1,
                            const double *s, const int32_t *stop, cudaStream_t st) {
  RR_LAUNCH_PDL(k_restrict_items, grid_for(plan.n_items, kWarps), kThreads, 0, st, plan.items,
                plan.n_items, members, r1, plan.item_sum, stop);
  RR_LAUNCH_PDL(k_restrict_combine, grid_for(plan.k, kWarps), kThreads, 0, st, plan.k,
                plan.item_ptr, plan.item_sum, s, plan.rc, stop);
  return RR_OK;
}

rr_status coarse_matvec(int32_t k, const double *Ainv, const RestrictPlan &plan, const double *s,
                        double *rc, double *ec, const int32_t *stop, cudaStream_t st) {
  const size_t smem = sizeof(double) * (size_t)k;
  static int attr_for = -1;
  if (smem > 48 * 1024 && attr_for < k) {
    RR_CUDA(cudaFuncSetAttribute(k_coarse_matvec, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    attr_for = k;
  }
  (void)s;
  RR_LAUNCH_PDL(k_coarse_matvec, grid_for(k, kWarps), kThreads, smem, st, k, Ainv,
                (const int32_t *)nullptr, (const double *)plan.rc, s, rc, ec, stop,
                (const double *)nullptr);
  return RR_OK;
}

rr_status coarse_to_f32(int32_t k, const double *Ainv, float *Ainv32, cudaStream_t st) {
  const int32_t ld = (k + 3) & ~3;
  RR_LAUNCH(k_to_f32_padded, grid_for((int64_t)k * ld, kThreads), kThreads, 0, st, k, ld, Ainv,
            Ainv32);
  return RR_OK;
}

rr_status coarse_matvec32(int32_t k, const float *Ainv32, const RestrictPlan &plan,
                          const double *s, double *ec, const int32_t *stop, cudaStream_t st) {
  const int32_t ld = (k + 3) & ~3;
  const size_t smem = sizeof(float) * (size_t)ld;
  static int attr_for = -1;
  if (smem > 48 * 1024 && attr_for < k) {
    RR_CUDA(cudaFuncSetAttribute(k_coarse_matvec32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    attr_for = k;
  }
  (void)s;
  RR_LAUNCH_PDL(k_coarse_matvec32, grid_for(k, kWarps), kThreads, smem, st, k, ld, Ainv32,
                (const double *)plan.rc, ec, stop);
  return RR_OK;
}

rr_status coarse_matvec_eigen(int32_t k, const double *Vk, const double *Qt, const double *dvec,
                              const RestrictPlan &plan, const double *s, double *tmp, double *ec,
                              const int32_t *stop, cudaStream_t st) {
  const size_t smem = sizeof(double) * (size_t)k;
  static int attr_for = -1;
  if (smem > 48 * 1024 && attr_for < k) {
    RR_CUDA(cudaFuncSetAttribute(k_coarse_matvec, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    attr_for = k;
  }
  // t = diag(1 / (mu + lambda)) Q^T r_c (rows of Vk are the eigenvectors), then e_c = Q t
  RR_LAUNCH_PDL(k_coarse_matvec, grid_for(k, kWarps), kThreads, smem, st, k, Vk,
                (const int32_t *)nullptr, (const double *)plan.rc, s, (double *)nullptr, tmp, stop,
                dvec);
  RR_LAUNCH_PDL(k_coarse_matvec, grid_for(k, kWarps), kThreads, smem, st, k, Qt,
                (const int32_t *)nullptr, (const double *)tmp, s, (double *)nullptr, ec, stop,
                (const double *)nullptr);
  return RR_OK;
}

rr_status prolong_add(int64_t F, const int32_t *labels, const double *s, const double *ec,
                      const double *z1, double *z2, const int32_t *stop, cudaStream_t st,
                      float *z2_32) {
  RR_LAUNCH_PDL(k_prolong_add, kVecGrid, kThreads, 0, st, F, labels, s, ec, z1, z2, z2_32, stop);
  return RR_OK;
}

rr_status jacobi(int64_t F, double omega, const double *r, const double *d, double *z,
                 double *rz_part, const int32_t *stop, cudaStream_t st, float *z32) {
  RR_LAUNCH_PDL(k_jacobi, kVecGrid, kThreads, 0, st, F, omega, r, d, z, z32, rz_part, stop);
  return RR_OK;
}

rr_status pcg_direction(int64_t F, const double *rz_part, int n_rz, const double *z, double *p,
                        PcgScalars *S, cudaStream_t st, float *p32) {
  RR_LAUNCH_PDL(k_pcg_direction, kVecGrid, kThreads, 0, st, F, rz_part, n_rz, z, p, p32, S);
  return RR_OK;
}

rr_status pcg_update(int64_t F, const double *rz_part, int n_rz, const double *pq_part, int n_pq,
                     const double *p, const double *q, double *w, double *r, double omega,
                     const double *d, double *z1, double *rr_part, PcgScalars *S,
                     cudaStream_t st, float *z1_32, const double *wd, double *history,
                     int32_t hist_cap) {
  RR_LAUNCH_PDL(k_pcg_update, kVecGrid, kThreads, 0, st, F, rz_part, n_rz, pq_part, n_pq, p, q, w, r,
            omega, d, z1, z1_32, rr_part, S, wd, history, hist_cap);
  return RR_OK;
}

rr_status inner_start(PcgScalars *S, const int32_t *outer_converged, cudaStream_t st) {
  RR_LAUNCH_PDL(k_inner_start, 1, 32, 0, st, S, outer_converged);
  return RR_OK;
}

rr_status dot_parts(int64_t n, const double *a, const double *b, double *part, cudaStream_t st) {
  RR_LAUNCH_PDL(k_dot_parts, kVecGrid, kThreads, 0, st, n, a, b, part);
  return RR_OK;
}

rr_status pcg_start(const double *bb_part, int n_bb, const double *rr_part, int n_rr, double tol,
                    int32_t set_bnorm, PcgScalars *S, cudaStream_t st) {
  RR_LAUNCH_PDL(k_pcg_start, 1, kThreads, 0, st, bb_part, n_bb, rr_part, n_rr, tol, set_bnorm, S);
  return RR_OK;
}

rr_status sum_parts(const double *part, int n, double *out, cudaStream_t st) {
  RR_LAUNCH_PDL(k_sum_parts, 1, kThreads, 0, st, part, n, out);
  return RR_OK;
}

rr_status copy_f64(double *dst, const double *src, int64_t n, cudaStream_t st) {
  RR_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  return RR_OK;
}

rr_status loop_condition(cudaGraphConditionalHandle hc, const PcgScalars *S, cudaStream_t st) {
  RR_LAUNCH_PDL(k_loop_condition, 1, 32, 0, st, hc, S);
  return RR_OK;
}

rr_status axpby(int64_t n, double a, const double *x, double b, double *y, cudaStream_t st) {
  RR_LAUNCH_PDL(k_axpby, kVecGrid, kThreads, 0, st, n, a, x, b, y);
  return RR_OK;
}

}  // namespace rr
