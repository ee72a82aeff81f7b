// Dense X (N x F, FP32, row-major): the clustering, the coarse level and the
// operator of the two-level method when X is stored densely (the paper's
// dense data sets of Table 1; Section 3.4's k-means++ with the Euclidean
// distance, Section 3.2's Galerkin operator).
//
// k-means (FP64, no fused multiply-add: every product and sum rounded on its
// own, as the oracle computes them): every sum over the N rows is taken in
// blocks of kRowBlock consecutive rows, each block in ascending row order,
// then the block sums in ascending block order; a centroid sums its member
// columns in ascending feature order. The draws follow the binary path
// (SplitMix64, u_t = (x_t >> 11) 2^-53) with the dense rule: first centre
// floor(u_0 F); centre t the first unchosen feature whose running sum of D2
// exceeds u_t * sum(D2) (the last unchosen feature with D2 > 0 if none; the
// lowest unchosen one if every D2 is 0). Lloyd: score(i, S) = ||mu_S||^2 -
// 2 x_i . mu_S, the smallest S on ties, empty clusters skipped.
//
// Operator X^T X v: one pass over X when F is a multiple of 4 and at most
// 8192 (k_dfused): each thread owns the same 4-column groups of every row,
// keeps v and its column sums in registers, and for each tile of R rows loads
// its x values once, forms its share of the R row dots, the block sums them
// (u_r = x_r . v, one barrier per tile), and adds x_ri u_r to its column sums;
// tiles go to the blocks round-robin, so the per-block partials and their
// in-order sum in the epilogue repeat bit for bit. Otherwise two passes: u =
// X v by one warp per row, X^T u by column partial sums over row blocks.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "epilogue.cuh"
#include "kernels.h"

namespace rr {

namespace {

constexpr int kRowBlock = 64;       // k-means row blocks (the oracle's)
constexpr int kColRows = 512;       // rows per block of the X^T u partial sums

__device__ __forceinline__ uint64_t sm64(uint64_t seed, int64_t t) {
  uint64_t z = seed + (uint64_t)(t + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double u53(uint64_t seed, int64_t t) {
  return (double)(sm64(seed, t) >> 11) * 0x1.0p-53;
}

// ---------------------------------------------------------------- seeding

// part[b F + i] = sum over the rows of block b of (x_ri - x_rc)^2, c = centers[t].
__global__ void k_dd2_part(int64_t N, int64_t F, const float *__restrict__ X,
                           const int32_t *__restrict__ centers, int32_t t,
                           double *__restrict__ part) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t b = blockIdx.y;
  if (i >= F) return;
  const int64_t c = centers[t];
  const int64_t r0 = b * kRowBlock, r1 = min(N, r0 + kRowBlock);
  double s = 0.0;
  for (int64_t r = r0; r < r1; ++r) {
    const double d = __dsub_rn((double)X[r * F + i], (double)X[r * F + c]);
    s = __dadd_rn(s, __dmul_rn(d, d));
  }
  part[b * F + i] = s;
}

// d2[i] = min(d2[i], sum of the block parts) (plain assignment in round 0; 0 for the centre).
__global__ void k_dd2_update(int64_t F, int64_t nb, const double *__restrict__ part,
                             const int32_t *__restrict__ centers, int32_t t,
                             double *__restrict__ d2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= F) return;
  double s = 0.0;
  for (int64_t b = 0; b < nb; ++b) s = __dadd_rn(s, part[b * F + i]);
  const double dist = (i == centers[t]) ? 0.0 : s;
  if (t == 0 || dist < d2[i]) d2[i] = dist;
}

// One thread: centre t (t = 0: floor(u_0 F); else the D2-weighted draw).
__global__ void k_dpick(int64_t F, int32_t t, uint64_t seed, const double *__restrict__ d2,
                        int32_t *centers, uint8_t *chosen, int32_t *err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t c = -1;
  if (t == 0) {
    c = (int64_t)floor(u53(seed, 0) * (double)F);
    if (c >= F) c = F - 1;
  } else {
    double total = 0.0;
    for (int64_t i = 0; i < F; ++i) total = __dadd_rn(total, d2[i]);
    if (total == 0.0) {
      for (int64_t i = 0; i < F; ++i)
        if (!chosen[i]) {
          c = i;
          break;
        }
    } else {
      const double thr = __dmul_rn(u53(seed, t), total);
      double cum = 0.0;
      for (int64_t i = 0; i < F; ++i) {
        cum = __dadd_rn(cum, d2[i]);
        if (cum > thr && !chosen[i]) {
          c = i;
          break;
        }
      }
      if (c < 0)
        for (int64_t i = F - 1; i >= 0; --i)
          if (!chosen[i] && d2[i] > 0.0) {
            c = i;
            break;
          }
    }
  }
  if (c < 0) {
    set_dev_error(err, DEV_BAD_INDEX);
    c = 0;
  }
  centers[t] = (int32_t)c;
  chosen[c] = 1;
}

// ---------------------------------------------------------------- Lloyd

__global__ void k_dlabels_init(int64_t F, int32_t k, const int32_t *__restrict__ centers,
                               int32_t *__restrict__ labels) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x)
    labels[i] = -1;
}
__global__ void k_dlabels_centres(int32_t k, const int32_t *__restrict__ centers,
                                  int32_t *__restrict__ labels) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < k; s += gridDim.x * blockDim.x)
    labels[centers[s]] = s;
}

// key[i] = label (k for unassigned features), the column of feature i in the
// cluster-membership pattern (so that its transpose lists members ascending).
__global__ void k_dkeys(int64_t F, int32_t k, const int32_t *__restrict__ labels,
                        int32_t *__restrict__ key) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x)
    key[i] = labels[i] < 0 ? k : labels[i];
}

// out[s N + r] = (sum over the members of s, ascending, of x_r,member) [/ n_s when divide].
__global__ void k_dcolsum(int64_t N, int64_t F, const float *__restrict__ X,
                          const int64_t *__restrict__ cl_ptr, const int32_t *__restrict__ members,
                          int32_t divide, double *__restrict__ out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t s = blockIdx.y;
  if (r >= N) return;
  const int64_t m0 = cl_ptr[s], m1 = cl_ptr[s + 1];
  double acc = 0.0;
  for (int64_t m = m0; m < m1; ++m) acc = __dadd_rn(acc, (double)X[r * F + members[m]]);
  if (divide) acc = (m1 > m0) ? __ddiv_rn(acc, (double)(m1 - m0)) : 0.0;
  out[(int64_t)s * N + r] = acc;
}

// part[s nb + b] = sum over block b of mu_s,r^2.
__global__ void k_dmm_part(int64_t N, int64_t nb, const double *__restrict__ mu,
                           double *__restrict__ part) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t s = blockIdx.y;
  if (b >= nb) return;
  const int64_t r0 = b * kRowBlock, r1 = min(N, r0 + kRowBlock);
  double q = 0.0;
  for (int64_t r = r0; r < r1; ++r) {
    const double m = mu[(int64_t)s * N + r];
    q = __dadd_rn(q, __dmul_rn(m, m));
  }
  part[(int64_t)s * nb + b] = q;
}

__global__ void k_dmm(int32_t k, int64_t nb, const double *__restrict__ part,
                      double *__restrict__ mm) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < k; s += gridDim.x * blockDim.x) {
    double q = 0.0;
    for (int64_t b = 0; b < nb; ++b) q = __dadd_rn(q, part[(int64_t)s * nb + b]);
    mm[s] = q;
  }
}

// The row-block partial dots of the kDotS clusters s0 .. s0 + kDotS - 1:
// part[(b kDotS + j) F + i] = sum over the rows of block b, ascending, of
// x_ri mu_(s0+j),r. One block of threads per (128 columns, row block); the
// block's mu rows are staged in shared memory.
constexpr int kDotS = 8, kDotThreads = 128;
__global__ void __launch_bounds__(kDotThreads) k_ddot_part(int64_t N, int64_t F, int32_t k, int32_t s0,
                                                           const float *__restrict__ X,
                                                           const double *__restrict__ mu,
                                                           double *__restrict__ part) {
  __shared__ double mus[kDotS][kRowBlock];
  const int64_t i = (int64_t)blockIdx.x * kDotThreads + threadIdx.x;
  const int64_t b = blockIdx.y;
  const int64_t r0 = b * kRowBlock;
  const int rn = (int)min((int64_t)kRowBlock, N - r0);
  const int ns = min(kDotS, k - s0);
  for (int e = threadIdx.x; e < kDotS * kRowBlock; e += kDotThreads) {
    const int j = e / kRowBlock, rr = e % kRowBlock;
    mus[j][rr] = (j < ns && rr < rn) ? mu[(int64_t)(s0 + j) * N + r0 + rr] : 0.0;
  }
  __syncthreads();
  if (i >= F) return;
  double p[kDotS];
#pragma unroll
  for (int j = 0; j < kDotS; ++j) p[j] = 0.0;
  for (int rr = 0; rr < rn; ++rr) {
    const double x = (double)X[(r0 + rr) * F + i];
#pragma unroll
    for (int j = 0; j < kDotS; ++j) p[j] = __dadd_rn(p[j], __dmul_rn(x, mus[j][rr]));
  }
#pragma unroll
  for (int j = 0; j < kDotS; ++j) part[(b * kDotS + j) * F + i] = p[j];
}

// dot[(s0 + j) F + i] = the block partials summed in ascending block order.
__global__ void k_ddot_chain(int64_t F, int64_t nb, int32_t ns, int32_t s0,
                             const double *__restrict__ part, double *__restrict__ dot) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)ns * F) return;
  const int64_t j = e / F, i = e % F;
  double t = 0.0;
  for (int64_t b = 0; b < nb; ++b) t = __dadd_rn(t, part[(b * kDotS + j) * F + i]);
  dot[(s0 + j) * F + i] = t;
}

// next label: argmin over non-empty S of mm_S - 2 dot_S,i (first minimum); changes counted.
__global__ void k_dargmin(int64_t F, int32_t k, const int64_t *__restrict__ cl_ptr,
                          const double *__restrict__ mm, const double *__restrict__ dot,
                          int32_t *__restrict__ labels, unsigned long long *changes) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t best = -1;
    double bv = 0.0;
    for (int32_t s = 0; s < k; ++s) {
      if (cl_ptr[s + 1] == cl_ptr[s]) continue;
      const double v = __dsub_rn(mm[s], __dmul_rn(2.0, dot[(int64_t)s * F + i]));
      if (best < 0 || v < bv) {
        best = s;
        bv = v;
      }
    }
    if (best != labels[i]) {
      atomicAdd(changes, 1ull);
      labels[i] = best;
    }
  }
}

// ---------------------------------------------------------------- coarse level, smoother

// G[S, T] = sum_r C[S, r] C[T, r] (C = X onehot, k x N), one block per (S, T <= S), mirrored.
__global__ void k_dgram(int64_t N, int32_t k, const double *__restrict__ C, double *__restrict__ G) {
  __shared__ double sm[kWarps + 1];
  const int32_t S = blockIdx.x, T = blockIdx.y;
  if (T > S) return;
  double acc = 0.0;
  for (int64_t r = threadIdx.x; r < N; r += blockDim.x)
    acc += C[(int64_t)S * N + r] * C[(int64_t)T * N + r];
  const double tot = block_sum(acc, sm);
  if (threadIdx.x == 0) {
    G[(int64_t)S * k + T] = tot;
    G[(int64_t)T * k + S] = tot;
  }
}

// sq[i] = sum_r x_ri^2; rowabs[r] = sum_i |x_ri| (two passes; rowabs first).
__global__ void k_drowabs(int64_t N, int64_t F, const float *__restrict__ X, double *__restrict__ ra) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < N; r += nwarps) {
    double s = 0.0;
    for (int64_t i = lane; i < F; i += 32) s += fabs((double)X[r * F + i]);
    s = warp_sum(s);
    if (lane == 0) ra[r] = s;
  }
}
// per column and block of kColRows rows: part[(2 b) F + i] = sum x^2,
// part[(2 b + 1) F + i] = sum |x_ri| ra[r]  (sum_j |(X^T X)_ij| <= gs[i]).
__global__ void k_dcolstats_part(int64_t N, int64_t F, const float *__restrict__ X,
                                 const double *__restrict__ ra, double *__restrict__ part) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t b = blockIdx.y;
  if (i >= F) return;
  const int64_t r0 = b * kColRows, r1 = min(N, r0 + kColRows);
  double a = 0.0, g = 0.0;
  for (int64_t r = r0; r < r1; ++r) {
    const double x = (double)X[r * F + i];
    a += x * x;
    g += fabs(x) * ra[r];
  }
  part[(2 * b) * F + i] = a;
  part[(2 * b + 1) * F + i] = g;
}
__global__ void k_dcolstats(int64_t F, int64_t nb, const double *__restrict__ part,
                            double *__restrict__ sq, double *__restrict__ gs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= F) return;
  double a = 0.0, g = 0.0;
  for (int64_t b = 0; b < nb; ++b) {
    a += part[(2 * b) * F + i];
    g += part[(2 * b + 1) * F + i];
  }
  sq[i] = a;
  gs[i] = g;
}

// d_i = sq_i + lambda; max over i of (gs_i + lambda) / d_i through the ordered bits.
__global__ void k_djacobi(int64_t F, double lambda, const double *__restrict__ sq,
                          const double *__restrict__ gs, double *__restrict__ d,
                          unsigned long long *__restrict__ max_bits) {
  unsigned long long best = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double di = sq[i] + lambda;
    d[i] = di;
    const double ratio = (gs[i] + lambda) / di;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(ratio);
    best = bits > best ? bits : best;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, best, o);
    best = t > best ? t : best;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(max_bits, best);
}

// ---------------------------------------------------------------- operator

// u[r] = x_r . v (one warp per row), accumulation in T; v staged in shared memory as T.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dxv(int64_t N, int64_t F, const float *__restrict__ X,
                                                  const double *__restrict__ v,
                                                  double *__restrict__ u,
                                                  const int32_t *__restrict__ stop) {
  pdl_wait();
  if (stop && *stop) return;
  extern __shared__ unsigned char dsm[];
  T *vs = reinterpret_cast<T *>(dsm);
  for (int64_t i = threadIdx.x; i < F; i += blockDim.x) vs[i] = (T)v[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < N; r += nwarps) {
    const float *xr = X + r * F;
    T acc = 0;
    for (int64_t i = lane; i < F; i += 32) acc += (T)xr[i] * vs[i];
    double s = (double)acc;
    s = warp_sum(s);
    if (lane == 0) u[r] = s;
  }
}

// part[b F + i] = sum over the rows of block b of x_ri u_r (accumulation in T).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dxtu(int64_t N, int64_t F, const float *__restrict__ X,
                                                   const double *__restrict__ u,
                                                   double *__restrict__ part,
                                                   const int32_t *__restrict__ stop) {
  pdl_wait();
  if (stop && *stop) return;
  __shared__ T us[kColRows];
  const int64_t r0 = (int64_t)blockIdx.y * kColRows;
  const int rn = (int)min((int64_t)kColRows, N - r0);
  for (int e = threadIdx.x; e < rn; e += blockDim.x) us[e] = (T)u[r0 + e];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= F) return;
  T acc = 0;
  for (int rr = 0; rr < rn; ++rr) acc += (T)X[(r0 + rr) * F + i] * us[rr];
  part[(int64_t)blockIdx.y * F + i] = (double)acc;
}

// One pass of X^T X v (see the file header). R rows per tile, G 4-column
// groups per thread (columns 4 (tid + 256 g) .. +3); every product and sum,
// the row dots' reductions included, in T (FP32 here keeps the FP64 pipe,
// a small fraction of the FP32 rate on this part, out of the loop);
// part[blockIdx.x * F + i] receives the block's sum for column i.
template <typename T, int R, int G>
__global__ void __launch_bounds__(kThreads) k_dfused(int64_t N, int64_t F, const float *__restrict__ X,
                                                     const double *__restrict__ v,
                                                     double *__restrict__ part,
                                                     const int32_t *__restrict__ stop) {
  pdl_wait();
  if (stop && *stop) return;
  __shared__ T red[2][R][kWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t F4 = F >> 2;
  const float4 *X4 = reinterpret_cast<const float4 *>(X);
  T vr[G][4], acc[G][4];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int64_t c4 = tid + (int64_t)g * kThreads;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      vr[g][j] = c4 < F4 ? (T)v[4 * c4 + j] : (T)0;
      acc[g][j] = (T)0;
    }
  }
  const int64_t n_tiles = (N + R - 1) / R;
  int par = 0;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t r0 = tile * R;
    float4 x[R][G];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int64_t c4 = tid + (int64_t)g * kThreads;
        x[r][g] = (r0 + r < N && c4 < F4) ? __ldcs(X4 + (r0 + r) * F4 + c4)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    T pr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      T sdot = (T)0;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        sdot += (T)x[r][g].x * vr[g][0];
        sdot += (T)x[r][g].y * vr[g][1];
        sdot += (T)x[r][g].z * vr[g][2];
        sdot += (T)x[r][g].w * vr[g][3];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sdot += __shfl_xor_sync(0xffffffffu, sdot, o);
      pr[r] = sdot;
    }
    if (lane == 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) red[par][r][warp] = pr[r];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      T u = (T)0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) u += red[par][r][w];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        acc[g][0] += (T)x[r][g].x * u;
        acc[g][1] += (T)x[r][g].y * u;
        acc[g][2] += (T)x[r][g].z * u;
        acc[g][3] += (T)x[r][g].w * u;
      }
    }
    par ^= 1;
  }
  double *out = part + (int64_t)blockIdx.x * F;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int64_t c4 = tid + (int64_t)g * kThreads;
    if (c4 < F4) {
#pragma unroll
      for (int j = 0; j < 4; ++j) out[4 * c4 + j] = (double)acc[g][j];
    }
  }
}

// t_i = sum of the nb row-block partials of column i, then the epilogue;
// kVecGrid partial dots. A block takes 32 columns at a time: warp g sums the
// partials b = g, g + 8, ... (four loads in flight), warp 0 adds the eight
// warp sums in order, so the bits do not depend on the launch.
__global__ void __launch_bounds__(kThreads) k_depi(int64_t F, int64_t nb,
                                                   const double *__restrict__ part, CscEpilogue ep) {
  pdl_wait();
  if (ep.stop && *ep.stop) return;
  __shared__ double red[kWarps][33];
  __shared__ double sm[kWarps + 1];
  const int c = threadIdx.x & 31, g = threadIdx.x >> 5;
  double dot = 0.0;
  for (int64_t c0 = (int64_t)blockIdx.x * 32; c0 < F; c0 += (int64_t)gridDim.x * 32) {
    const int64_t i = c0 + c;
    double s = 0.0;
    if (i < F) {
      int64_t b = g;
      for (; b + 3 * kWarps < nb; b += 4 * kWarps) {
        const double a0 = part[b * F + i], a1 = part[(b + kWarps) * F + i];
        const double a2 = part[(b + 2 * kWarps) * F + i], a3 = part[(b + 3 * kWarps) * F + i];
        s += a0;
        s += a1;
        s += a2;
        s += a3;
      }
      for (; b < nb; b += kWarps) s += part[b * F + i];
    }
    red[g][c] = s;
    __syncthreads();
    if (g == 0 && i < F) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) t += red[w][c];
      epilogue(ep, i, t, dot);
    }
    __syncthreads();
  }
  const double tot = block_sum(dot, sm);
  if (threadIdx.x == 0 && ep.dot_part) ep.dot_part[blockIdx.x] = tot;
}

}  // namespace

rr_status dense_kmeanspp(int64_t N, int64_t F, const float *X, int32_t k, uint64_t seed,
                         int32_t *centers, double *d2, uint8_t *chosen, double *part, int32_t *err,
                         cudaStream_t st) {
  const int64_t nb = (N + kRowBlock - 1) / kRowBlock;
  RR_CUDA(cudaMemsetAsync(chosen, 0, F, st));
  RR_LAUNCH(k_dpick, 1, 32, 0, st, F, 0, seed, d2, centers, chosen, err);
  const dim3 g((unsigned)((F + kThreads - 1) / kThreads), (unsigned)nb);
  for (int32_t t = 0; t < k; ++t) {
    RR_LAUNCH(k_dd2_part, g, kThreads, 0, st, N, F, X, centers, t, part);
    RR_LAUNCH(k_dd2_update, (unsigned)((F + kThreads - 1) / kThreads), kThreads, 0, st, F, nb, part,
              centers, t, d2);
    if (t + 1 < k) RR_LAUNCH(k_dpick, 1, 32, 0, st, F, t + 1, seed, d2, centers, chosen, err);
  }
  return RR_OK;
}

rr_status dense_lloyd(int64_t N, int64_t F, const float *X, int32_t k, const int32_t *centers,
                      int32_t max_iter, int32_t *labels, DenseKmeansScratch &w, int32_t *iters,
                      cudaStream_t st) {
  const int64_t nb = (N + kRowBlock - 1) / kRowBlock;
  RR_LAUNCH(k_dlabels_init, grid_for(F, kThreads), kThreads, 0, st, F, k, centers, labels);
  RR_LAUNCH(k_dlabels_centres, grid_for(k, kThreads), kThreads, 0, st, k, centers, labels);
  unsigned long long changes = 0;
  int32_t it = 0;
  while (it < max_iter) {
    ++it;
    // members of every cluster, ascending (unassigned features under key k)
    RR_LAUNCH(k_dkeys, grid_for(F, kThreads), kThreads, 0, st, F, k, labels, w.key);
    RR_TRY(transpose_pattern(F, k + 1, F, w.iota, w.key, w.cl_ptr, w.members, w.counts, w.cursor,
                             w.tmp, w.scan_scratch, st));
    RR_LAUNCH(k_dcolsum, dim3((unsigned)((N + kThreads - 1) / kThreads), (unsigned)k), kThreads, 0,
              st, N, F, X, w.cl_ptr, w.members, 1, w.mu);
    RR_LAUNCH(k_dmm_part, dim3((unsigned)((nb + kThreads - 1) / kThreads), (unsigned)k), kThreads,
              0, st, N, nb, w.mu, w.part);
    RR_LAUNCH(k_dmm, 1, 64, 0, st, k, nb, w.part, w.mm);
    for (int32_t s0 = 0; s0 < k; s0 += kDotS) {
      RR_LAUNCH(k_ddot_part, dim3((unsigned)((F + kDotThreads - 1) / kDotThreads), (unsigned)nb),
                kDotThreads, 0, st, N, F, k, s0, X, w.mu, w.dpart);
      const int32_t ns = std::min(kDotS, k - s0);
      RR_LAUNCH(k_ddot_chain, grid_for((int64_t)ns * F, kThreads), kThreads, 0, st, F, nb, ns, s0,
                w.dpart, w.dot);
    }
    RR_CUDA(cudaMemsetAsync(w.changes, 0, sizeof(unsigned long long), st));
    RR_LAUNCH(k_dargmin, grid_for(F, kThreads), kThreads, 0, st, F, k, w.cl_ptr, w.mm, w.dot,
              labels, w.changes);
    RR_CUDA(cudaMemcpyAsync(&changes, w.changes, sizeof(changes), cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    if (changes == 0) break;
  }
  *iters = it;
  return RR_OK;
}

rr_status dense_coarse_gram(int64_t N, int64_t F, const float *X, int32_t k_eff,
                            const int64_t *cl_ptr, const int32_t *members, double *C, double *G,
                            cudaStream_t st) {
  RR_LAUNCH(k_dcolsum, dim3((unsigned)((N + kThreads - 1) / kThreads), (unsigned)k_eff), kThreads,
            0, st, N, F, X, cl_ptr, members, 0, C);
  RR_LAUNCH(k_dgram, dim3((unsigned)k_eff, (unsigned)k_eff), kThreads, 0, st, N, k_eff, C, G);
  return RR_OK;
}

rr_status dense_colstats(int64_t N, int64_t F, const float *X, double *rowabs, double *part,
                         double *sq, double *gs, cudaStream_t st) {
  const int64_t nb = dense_col_blocks(N);
  RR_LAUNCH(k_drowabs, grid_for(N, kWarps), kThreads, 0, st, N, F, X, rowabs);
  RR_LAUNCH(k_dcolstats_part, dim3((unsigned)((F + kThreads - 1) / kThreads), (unsigned)nb),
            kThreads, 0, st, N, F, X, rowabs, part);
  RR_LAUNCH(k_dcolstats, (unsigned)((F + kThreads - 1) / kThreads), kThreads, 0, st, F, nb, part,
            sq, gs);
  return RR_OK;
}

int64_t dense_dot_part_len(int64_t N, int64_t F) {
  return ((N + kRowBlock - 1) / kRowBlock) * kDotS * F;
}

rr_status dense_jacobi(int64_t F, double lambda, const double *sq, const double *gs, double *d,
                       unsigned long long *max_bits, cudaStream_t st) {
  RR_LAUNCH(k_djacobi, grid_for(F, kThreads), kThreads, 0, st, F, lambda, sq, gs, d, max_bits);
  return RR_OK;
}

int64_t dense_col_blocks(int64_t N) { return (N + kColRows - 1) / kColRows; }

rr_status dense_matvec(int64_t N, int64_t F, const float *X, const double *v, double *u,
                       const int32_t *stop, bool fp32, cudaStream_t st) {
  const size_t smem = (fp32 ? sizeof(float) : sizeof(double)) * (size_t)F;
  if (smem > 200 * 1024) {
    rr_set_error("dense operator: F = %lld is above the shared-memory staging limit",
                 (long long)F);
    return RR_UNSUPPORTED;
  }
  static bool attr = false;
  if (!attr) {
    RR_CUDA(cudaFuncSetAttribute(k_dxv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    RR_CUDA(cudaFuncSetAttribute(k_dxv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  if (fp32)
    RR_LAUNCH_PDL(k_dxv<float>, grid_for(N, kWarps), kThreads, smem, st, N, F, X, v, u, stop);
  else
    RR_LAUNCH_PDL(k_dxv<double>, grid_for(N, kWarps), kThreads, smem, st, N, F, X, v, u, stop);
  return RR_OK;
}

rr_status dense_transposed(int64_t N, int64_t F, const float *X, const double *u, double *part,
                           const CscEpilogue &ep, bool fp32, cudaStream_t st) {
  const int64_t nb = dense_col_blocks(N);
  const dim3 g((unsigned)((F + kThreads - 1) / kThreads), (unsigned)nb);
  if (fp32)
    RR_LAUNCH_PDL(k_dxtu<float>, g, kThreads, 0, st, N, F, X, u, part, ep.stop);
  else
    RR_LAUNCH_PDL(k_dxtu<double>, g, kThreads, 0, st, N, F, X, u, part, ep.stop);
  RR_LAUNCH_PDL(k_depi, kVecGrid, kThreads, 0, st, F, nb, part, ep);
  return RR_OK;
}

namespace {

// 4-column groups per thread for F columns (0: no one-pass kernel for this F).
int fused_groups(int64_t F) {
  if (F % 4 != 0) return 0;
  const int64_t g = (F / 4 + kThreads - 1) / kThreads;
  return g <= 1 ? 1 : g <= 2 ? 2 : g <= 4 ? 4 : g <= 8 ? 8 : 0;
}

// Blocks of the one-pass kernel: all that fit on the device at once.
template <typename T, int R, int G>
int fused_grid() {
  static int grid = 0;
  if (grid == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfused<T, R, G>, kThreads, 0) !=
            cudaSuccess)
      return 0;
    grid = std::max(1, sms * std::max(1, per_sm));
  }
  return grid;
}

// The (T, R, G) instantiation for 4-column groups G: R rows per tile keep the
// x values of a tile at <= 64 registers (FP32) or the accumulators and v
// within the register file (FP64).
template <typename Fn>
rr_status with_fused(int G, bool fp32, Fn &&fn) {
  if (fp32) {
    switch (G) {
      case 1: return fn(std::integral_constant<int, 0>{});
      case 2: return fn(std::integral_constant<int, 1>{});
      case 4: return fn(std::integral_constant<int, 2>{});
      default: return fn(std::integral_constant<int, 3>{});
    }
  }
  switch (G) {
    case 1: return fn(std::integral_constant<int, 4>{});
    case 2: return fn(std::integral_constant<int, 5>{});
    case 4: return fn(std::integral_constant<int, 6>{});
    default: return fn(std::integral_constant<int, 7>{});
  }
}
template <int V> struct Fused;
template <> struct Fused<0> { using T = float; static constexpr int R = 4, G = 1; };
template <> struct Fused<1> { using T = float; static constexpr int R = 4, G = 2; };
template <> struct Fused<2> { using T = float; static constexpr int R = 4, G = 4; };
template <> struct Fused<3> { using T = float; static constexpr int R = 2, G = 8; };
template <> struct Fused<4> { using T = double; static constexpr int R = 4, G = 1; };
template <> struct Fused<5> { using T = double; static constexpr int R = 4, G = 2; };
template <> struct Fused<6> { using T = double; static constexpr int R = 2, G = 4; };
template <> struct Fused<7> { using T = double; static constexpr int R = 1, G = 8; };

}  // namespace

int64_t dense_part_rows(int64_t N, int64_t F) {
  int64_t rows = dense_col_blocks(N);
  const int G = fused_groups(F);
  if (G == 0) return rows;
  for (bool fp32 : {true, false}) {
    int grid = 0;
    with_fused(G, fp32, [&](auto v) -> rr_status {
      using C = Fused<decltype(v)::value>;
      grid = fused_grid<typename C::T, C::R, C::G>();
      return RR_OK;
    });
    rows = std::max<int64_t>(rows, grid);
  }
  return rows;
}

rr_status dense_operator(int64_t N, int64_t F, const float *X, const double *v, double *u,
                         double *part, const CscEpilogue &ep, bool fp32, cudaStream_t st) {
  const int G = fused_groups(F);
  if (G == 0) {
    RR_TRY(dense_matvec(N, F, X, v, u, ep.stop, fp32, st));
    return dense_transposed(N, F, X, u, part, ep, fp32, st);
  }
  return with_fused(G, fp32, [&](auto tag) -> rr_status {
    using C = Fused<decltype(tag)::value>;
    const int grid = fused_grid<typename C::T, C::R, C::G>();
    if (grid == 0) {
      rr_set_error("dense operator: occupancy query failed");
      return RR_CUDA_ERROR;
    }
    RR_LAUNCH_PDL((k_dfused<typename C::T, C::R, C::G>), grid, kThreads, 0, st, N, F, X, v, part,
                  ep.stop);
    RR_LAUNCH_PDL(k_depi, kVecGrid, kThreads, 0, st, F, (int64_t)grid, part, ep);
    return RR_OK;
  });
}

}  // namespace rr
