// Coarse level of the two-level preconditioner (Section 3.2 and Section 4):
// cluster compaction, the prolongation scale s_S = 1/sqrt(n_S) (Eq. (prolong)),
// the integer counts C = X * onehot(labels), the exact Gram G = C^T C, the
// Galerkin operator A_c = D_s G D_s + lambda I, its Cholesky factor and the
// explicit inverse A_c^{-1} = L^{-T} L^{-1} used by the per-iteration coarse solve.
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rr {

namespace {

__global__ void k_count_labels(int64_t F, const int32_t *__restrict__ labels,
                               unsigned long long *__restrict__ n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&n[labels[i]], 1ULL);
}

// Single block: remap[S] = rank of S among the non-empty clusters (-1 if empty);
// n_out[rank] = n[S]; *k_eff = number of non-empty clusters.
__global__ void k_compact(int32_t k, const int64_t *__restrict__ n, int32_t *__restrict__ remap,
                          int64_t *__restrict__ n_out, int32_t *k_eff) {
  __shared__ int32_t sm[kWarps + 1];
  int32_t carry = 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int32_t b = 0; b < k; b += kThreads) {
    const int32_t s = b + threadIdx.x;
    const int32_t used = (s < k && n[s] > 0) ? 1 : 0;
    int32_t inc = used;
    for (int o = 1; o < 32; o <<= 1) {
      int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    __syncthreads();
    if (lane == 31) sm[warp] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t run = 0;
      for (int w = 0; w < kWarps; ++w) {
        int32_t t = sm[w];
        sm[w] = run;
        run += t;
      }
      sm[kWarps] = run;
    }
    __syncthreads();
    const int32_t ex = carry + sm[warp] + inc - used;
    if (s < k) {
      remap[s] = used ? ex : -1;
      if (used) n_out[ex] = n[s];
    }
    carry += sm[kWarps];
    __syncthreads();
  }
  if (threadIdx.x == 0) *k_eff = carry;
}

__global__ void k_remap_labels(int64_t F, const int32_t *__restrict__ remap,
                               int32_t *__restrict__ labels) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x)
    labels[i] = remap[labels[i]];
}

__global__ void k_prolong_scale(int32_t k, const int64_t *__restrict__ n, double *__restrict__ s) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x)
    s[i] = 1.0 / sqrt((double)n[i]);
}

// C32[S, r] += 1 for every entry (r, j) with label_j = S (exact int32 counts);
// *max_count = the largest count (one atomic per warp).
__global__ void k_coarse_counts(int64_t N, int64_t n_pad, const int64_t *__restrict__ row_ptr,
                                const int32_t *__restrict__ col_idx,
                                const int32_t *__restrict__ labels, int32_t *__restrict__ C32,
                                int32_t *max_count) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t mx = 0;
  for (int64_t r = warp; r < N; r += nwarps) {
    for (int64_t e = row_ptr[r] + lane; e < row_ptr[r + 1]; e += 32) {
      const int64_t S = labels[col_idx[e]];
      const int32_t now = atomicAdd(&C32[S * n_pad + r], 1) + 1;
      mx = max(mx, now);
    }
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0 && mx > 0) atomicMax(max_count, mx);
}

// FP16 copy of the counts for the tensor cores (exact: every count <= 2048).
__global__ void k_counts_to_half(int64_t n, const int32_t *__restrict__ C32,
                                 __half *__restrict__ C16) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    C16[i] = __int2half_rn(C32[i]);
}

// G = C32 C32^T over the lower tile triangle, exact: int32 products of counts
// summed over 32-row steps, steps summed in int64, stored as FP64 (exact below
// 2^53). A step's sum is below 2^31 while every count is below 8192; larger
// counts are reported as unsupported by the caller.
constexpr int kGT = 64;   // output tile
constexpr int kGK = 32;   // rows per step
__global__ void __launch_bounds__(kThreads) k_gram_cc(int32_t k, int64_t n_pad,
                                                      const int32_t *__restrict__ Ct,
                                                      double *__restrict__ G) {
  // blockIdx.x enumerates lower-triangular tile pairs (ti >= tj)
  int64_t t = blockIdx.x;
  int ti = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((int64_t)(ti + 1) * (ti + 2) / 2 <= t) ++ti;
  while ((int64_t)ti * (ti + 1) / 2 > t) --ti;
  const int tj = (int)(t - (int64_t)ti * (ti + 1) / 2);
  const int S0 = ti * kGT, T0 = tj * kGT;
  __shared__ int32_t a[kGK][kGT + 1];
  __shared__ int32_t bsm[kGK][kGT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads, 4 x 4 outputs each
  int64_t acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  for (int64_t r0 = 0; r0 < n_pad; r0 += kGK) {
    for (int idx = threadIdx.x; idx < kGK * kGT; idx += kThreads) {
      const int row = idx / kGK, kk = idx % kGK;   // consecutive threads read consecutive rows r
      const int S = S0 + row, T = T0 + row;
      a[kk][row] = (S < k) ? Ct[(int64_t)S * n_pad + r0 + kk] : 0;
      bsm[kk][row] = (T < k) ? Ct[(int64_t)T * n_pad + r0 + kk] : 0;
    }
    __syncthreads();
    int32_t part[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) part[i][j] = 0;
#pragma unroll 8
    for (int kk = 0; kk < kGK; ++kk) {
      int32_t av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = a[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = bsm[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) part[i][j] += av[i] * bv[j];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += part[i][j];
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int S = S0 + ty * 4 + i, T = T0 + tx * 4 + j;
      if (S < k && T < k && S >= T) {
        G[(int64_t)S * k + T] = (double)acc[i][j];
        G[(int64_t)T * k + S] = (double)acc[i][j];
      }
    }
}

// A_c[S,T] = (G[S,T] s_S) s_T for S >= T, mirrored; + lambda on the diagonal.
__global__ void k_coarse_operator(int32_t k, const double *__restrict__ G,
                                  const double *__restrict__ s, double lambda,
                                  double *__restrict__ Ac) {
  const int64_t kk = (int64_t)k * k;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < kk;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int S = (int)(idx / k), T = (int)(idx % k);
    const int hi = S >= T ? S : T, lo = S >= T ? T : S;
    // explicit roundings: no fused multiply-add, so the value is the
    // correctly rounded product, then the correctly rounded sum
    double v = __dmul_rn(__dmul_rn(G[(int64_t)hi * k + lo], s[hi]), s[lo]);
    if (S == T) v = __dadd_rn(v, lambda);
    Ac[idx] = v;
  }
}

constexpr int kNB = 32;   // Cholesky panel width

// Factors the nb x nb diagonal block at j0 in shared memory (right-looking,
// the block's threads over the entries) and, when Wd is given, writes
// W = L11^{-1} (lower, 32 x 32 row-major, zero elsewhere) there for the panel:
// the same elimination applied to the identity (row j of W divided by L_jj,
// then subtracted L_ij times from every row i > j).
__global__ void k_chol_diag(int32_t k, int32_t j0, double *__restrict__ L, double *__restrict__ Wd,
                            int32_t *err) {
  __shared__ double a[kNB][kNB + 1];
  __shared__ double w[kNB][kNB + 1];
  __shared__ int bad;
  const int nb = min(kNB, k - j0);
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int i = idx / nb, j = idx % nb;
    a[i][j] = L[(int64_t)(j0 + i) * k + j0 + j];
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      const double piv = a[j][j];
      if (!(piv > 0.0)) {
        bad = 1;
        a[j][j] = 1.0;
      } else {
        a[j][j] = sqrt(piv);
      }
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) a[i][j] /= a[j][j];
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
      const int i = idx / nb, m = idx % nb;
      if (i > j && m > j && m <= i) a[i][m] -= a[i][j] * a[m][j];
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int i = idx / nb, j = idx % nb;
    L[(int64_t)(j0 + i) * k + j0 + j] = (j <= i) ? a[i][j] : 0.0;
  }
  if (threadIdx.x == 0 && bad) set_dev_error(err, DEV_NOT_SPD);
  if (!Wd) return;
  for (int idx = threadIdx.x; idx < kNB * kNB; idx += blockDim.x) {
    const int i = idx / kNB, c = idx % kNB;
    w[i][c] = (i == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    for (int c = threadIdx.x; c <= j; c += blockDim.x) w[j][c] /= a[j][j];
    __syncthreads();
    for (int idx = threadIdx.x; idx < kNB * kNB; idx += blockDim.x) {
      const int i = idx / kNB, c = idx % kNB;
      if (i > j && i < nb && c <= j) w[i][c] -= a[i][j] * w[j][c];
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < kNB * kNB; idx += blockDim.x) {
    const int i = idx / kNB, c = idx % kNB;
    Wd[idx] = (i < nb && c < nb && c <= i) ? w[i][c] : 0.0;
  }
}

// Rows below the diagonal block: L21 = A21 L11^{-T} = A21 W^T, a product with
// no dependent chain: one thread per entry of kPanelRows rows, W and the
// block's rows staged in shared memory (each block owns whole rows, read
// before they are overwritten).
constexpr int kPanelRows = 8;
__global__ void __launch_bounds__(kPanelRows * kNB) k_chol_panel(int32_t k, int32_t j0,
                                                                 double *__restrict__ L,
                                                                 const double *__restrict__ Wd) {
  __shared__ double ws[kNB][kNB + 1];
  __shared__ double as[kPanelRows][kNB + 1];
  const int nb = min(kNB, k - j0);
  for (int idx = threadIdx.x; idx < kNB * kNB; idx += blockDim.x)
    ws[idx / kNB][idx % kNB] = Wd[idx];
  const int r = threadIdx.x / kNB, c = threadIdx.x % kNB;
  const int64_t i = (int64_t)j0 + nb + (int64_t)blockIdx.x * kPanelRows + r;
  const bool ok = i < k && c < nb;
  if (ok) as[r][c] = L[i * k + j0 + c];
  __syncthreads();
  if (ok) {
    double s = 0.0;
    for (int m = 0; m <= c; ++m) s += as[r][m] * ws[c][m];
    L[i * k + j0 + c] = s;
  }
}

// Trailing update A22 -= L21 L21^T on lower 32 x 32 tiles.
__global__ void k_chol_update(int32_t k, int32_t j0, double *__restrict__ L) {
  const int nb = min(kNB, k - j0);
  const int base = j0 + nb;
  int64_t t = blockIdx.x;
  int ti = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((int64_t)(ti + 1) * (ti + 2) / 2 <= t) ++ti;
  while ((int64_t)ti * (ti + 1) / 2 > t) --ti;
  const int tj = (int)(t - (int64_t)ti * (ti + 1) / 2);
  const int I0 = base + ti * 32, J0 = base + tj * 32;
  __shared__ double li[32][kNB + 1], lj[32][kNB + 1];
  for (int idx = threadIdx.x; idx < 32 * kNB; idx += blockDim.x) {
    const int r = idx / kNB, c = idx % kNB;
    li[r][c] = (I0 + r < k && c < nb) ? L[(int64_t)(I0 + r) * k + j0 + c] : 0.0;
    lj[r][c] = (J0 + r < k && c < nb) ? L[(int64_t)(J0 + r) * k + j0 + c] : 0.0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
    const int r = idx / 32, c = idx % 32;
    const int i = I0 + r, j = J0 + c;
    if (i < k && j < k && j <= i) {
      double s = 0.0;
#pragma unroll 8
      for (int q = 0; q < kNB; ++q) s += li[r][q] * lj[c][q];
      L[(int64_t)i * k + j] -= s;
    }
  }
}

// LinvT[j][i] = (L^{-1})[i][j] for i >= j: one warp per column j, forward
// substitution with warp-parallel dot products. The column being built sits in
// shared memory (dynamic, one row of k doubles per warp of the block), so each
// step waits on a shared-memory round trip only; written out at the end.
constexpr int kTriWarps = 4;
constexpr int kTriWin = 32;   // row entries per lane held in registers (rows up to 1024 long)
__global__ void __launch_bounds__(32 * kTriWarps) k_tri_inverse(int32_t k,
                                                                const double *__restrict__ L,
                                                                double *__restrict__ LinvT) {
  extern __shared__ double xs_all[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double *x = xs_all + (int64_t)wib * k;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = warp; j < k; j += nwarps) {
    double rwin = 0.0;   // lane l: 1 / L[i0 + l][i0 + l] for the current window of 32 rows
    // the first kTriWin entries of the row being summed (m = j + lane + 32 t), loaded
    // one step ahead, so the step waits on shared memory and arithmetic only
    double cur[kTriWin];
#pragma unroll
    for (int t = 0; t < kTriWin; ++t) cur[t] = 0.0;
    for (int64_t i = j; i < k; ++i) {
      const int step = (int)((i - j) & 31);
      if (step == 0) {   // the divides of the next 32 rows, off the dependent chain
        const int64_t ii = i + lane;
        rwin = ii < k ? 1.0 / L[ii * k + ii] : 0.0;
      }
      double nxt[kTriWin];
      const int64_t i1 = i + 1;
#pragma unroll
      for (int t = 0; t < kTriWin; ++t) {
        const int64_t m = j + lane + 32 * t;
        nxt[t] = (i1 < k && m < i1) ? L[i1 * k + m] : 0.0;
      }
      const double *Li = L + i * k;
      double s0 = 0.0, s1 = 0.0;
#pragma unroll
      for (int t = 0; t < kTriWin; t += 2) {
        if (32 * t >= i - j) break;
        const int64_t m = j + lane + 32 * t;
        if (m < i) s0 += cur[t] * x[m];
        if (m + 32 < i) s1 += cur[t + 1] * x[m + 32];
      }
      for (int64_t m = j + lane + 32 * kTriWin; m < i; m += 32) s0 += Li[m] * x[m];
      const double s = warp_sum(s0 + s1);
      const double ri = __shfl_sync(0xffffffffu, rwin, step);
      if (lane == 0) x[i] = ((i == j ? 1.0 : 0.0) - s) * ri;
      __syncwarp();
#pragma unroll
      for (int t = 0; t < kTriWin; ++t) cur[t] = nxt[t];
    }
    double *out = LinvT + j * k;
    for (int64_t i = j + lane; i < k; i += 32) out[i] = x[i];
    __syncwarp();
  }
}

// Ainv[S][T] = sum_m LinvT[S][m] LinvT[T][m] on lower 32 x 32 tiles, mirrored.
__global__ void k_inverse_product(int32_t k, const double *__restrict__ LinvT,
                                  double *__restrict__ Ainv) {
  int64_t t = blockIdx.x;
  int ti = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((int64_t)(ti + 1) * (ti + 2) / 2 <= t) ++ti;
  while ((int64_t)ti * (ti + 1) / 2 > t) --ti;
  const int tj = (int)(t - (int64_t)ti * (ti + 1) / 2);
  const int S0 = ti * 32, T0 = tj * 32;
  __shared__ double a[32][33], b[32][33];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16, 2 x 2 outputs each
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int m0 = S0 > T0 ? S0 : T0; m0 < k; m0 += 32) {
    for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
      const int r = idx / 32, c = idx % 32;
      const int m = m0 + c;
      a[r][c] = (S0 + r < k && m < k) ? LinvT[(int64_t)(S0 + r) * k + m] : 0.0;
      b[r][c] = (T0 + r < k && m < k) ? LinvT[(int64_t)(T0 + r) * k + m] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int c = 0; c < 32; ++c) {
      const double a0 = a[ty * 2][c], a1 = a[ty * 2 + 1][c];
      const double b0 = b[tx * 2][c], b1 = b[tx * 2 + 1][c];
      acc[0][0] += a0 * b0;
      acc[0][1] += a0 * b1;
      acc[1][0] += a1 * b0;
      acc[1][1] += a1 * b1;
    }
    __syncthreads();
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      const int S = S0 + ty * 2 + i, T = T0 + tx * 2 + j;
      if (S < k && T < k && S >= T) {
        Ainv[(int64_t)S * k + T] = acc[i][j];
        Ainv[(int64_t)T * k + S] = acc[i][j];
      }
    }
}

inline unsigned tri_tiles(int64_t n_tiles) { return (unsigned)(n_tiles * (n_tiles + 1) / 2); }

}  // namespace

rr_status compact_clusters(int64_t F, int32_t k, int32_t *labels, int64_t *n_S, int32_t *remap,
                           int32_t *k_eff_host, cudaStream_t st) {
  // n_S is used as scratch of 2k entries: counts, then the compacted sizes
  int64_t *cnt = n_S + k;
  RR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * k, st));
  RR_LAUNCH(k_count_labels, grid_for(F, kThreads), kThreads, 0, st, F, labels,
            (unsigned long long *)cnt);
  int32_t *keff_dev = remap + k;
  RR_LAUNCH(k_compact, 1, kThreads, 0, st, k, cnt, remap, n_S, keff_dev);
  RR_LAUNCH(k_remap_labels, grid_for(F, kThreads), kThreads, 0, st, F, remap, labels);
  RR_CUDA(cudaMemcpyAsync(k_eff_host, keff_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  return RR_OK;
}

rr_status prolong_scale(int32_t k, const int64_t *n_S, double *s, cudaStream_t st) {
  RR_LAUNCH(k_prolong_scale, grid_for(k, kThreads), kThreads, 0, st, k, n_S, s);
  return RR_OK;
}

rr_status coarse_counts(int64_t N, int64_t n_pad, int32_t k_pad, const int64_t *row_ptr,
                        const int32_t *col_idx, const int32_t *labels, int32_t *C32,
                        int32_t *max_count, cudaStream_t st) {
  RR_CUDA(cudaMemsetAsync(C32, 0, sizeof(int32_t) * (size_t)k_pad * n_pad, st));
  RR_CUDA(cudaMemsetAsync(max_count, 0, sizeof(int32_t), st));
  RR_LAUNCH(k_coarse_counts, grid_for(N, kWarps), kThreads, 0, st, N, n_pad, row_ptr, col_idx,
            labels, C32, max_count);
  return RR_OK;
}

rr_status counts_to_half(int64_t n, const int32_t *C32, void *C16, cudaStream_t st) {
  RR_LAUNCH(k_counts_to_half, grid_for(n, kThreads), kThreads, 0, st, n, C32, (__half *)C16);
  return RR_OK;
}

rr_status gram_exact_cuda_cores(int32_t k, int32_t k_pad, int64_t n_pad, const int32_t *C32,
                                double *G, cudaStream_t st) {
  (void)k_pad;
  const int64_t nt = (k + kGT - 1) / kGT;
  RR_LAUNCH(k_gram_cc, tri_tiles(nt), kThreads, 0, st, k, n_pad, C32, G);
  return RR_OK;
}

rr_status coarse_operator(int32_t k, const double *G, const double *s, double lambda, double *Ac,
                          cudaStream_t st) {
  RR_LAUNCH(k_coarse_operator, grid_for((int64_t)k * k, kThreads), kThreads, 0, st, k, G, s,
            lambda, Ac);
  return RR_OK;
}

rr_status cholesky(int32_t k, double *L, double *scratch, int32_t *err, cudaStream_t st) {
  for (int32_t j0 = 0; j0 < k; j0 += kNB) {
    const int32_t rest = k - j0 - std::min(kNB, k - j0);
    RR_LAUNCH(k_chol_diag, 1, kThreads, 0, st, k, j0, L, rest > 0 ? scratch : nullptr, err);
    if (rest > 0) {
      RR_LAUNCH(k_chol_panel, (unsigned)((rest + kPanelRows - 1) / kPanelRows), kPanelRows * kNB,
                0, st, k, j0, L, scratch);
      const int64_t nt = (rest + 31) / 32;
      RR_LAUNCH(k_chol_update, tri_tiles(nt), kThreads, 0, st, k, j0, L);
    }
  }
  return RR_OK;
}

rr_status chol_inverse(int32_t k, const double *L, double *Linv, double *Ainv, cudaStream_t st) {
  RR_CUDA(cudaMemsetAsync(Linv, 0, sizeof(double) * (size_t)k * k, st));
  // warps per block: as many as their columns fit in 200 KB of shared memory (k <= 16384: >= 1)
  const int tw = (int)std::max<int64_t>(1, std::min<int64_t>(kTriWarps, (200 * 1024) / (8 * (int64_t)k)));
  const size_t tsmem = sizeof(double) * (size_t)tw * k;
  RR_CUDA(cudaFuncSetAttribute(k_tri_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               200 * 1024));
  RR_LAUNCH(k_tri_inverse, (unsigned)((k + tw - 1) / tw), 32 * tw, tsmem, st, k, L, Linv);
  const int64_t nt = (k + 31) / 32;
  RR_LAUNCH(k_inverse_product, tri_tiles(nt), kThreads, 0, st, k, Linv, Ainv);
  return RR_OK;
}

}  // namespace rr
