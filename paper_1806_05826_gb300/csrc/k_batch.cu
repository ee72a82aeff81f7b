// Batched two-level PCG: many targets y_j and many regularisation weights
// lambda_l over one X. Section 2 states the problem for several right-hand
// sides and several weights; the hierarchy of Section 3 (the clustering, P and
// the exact Gram of the coarse level) depends on X only, so every system shares
// it, and only the coarse factor (A_c + lambda I, Eq. (Galerkin) with the
// weight on the diagonal), the Jacobi diagonal and the damping change with
// lambda.
//
// Layout: the systems are the columns of F x ld row-major blocks (ld a
// multiple of 64). Slab s is the column range [64 s, 64 s + 64). The operator
// apply is two sparse-times-dense passes over X's pattern:
//   pass 1  U[r, :] = sum_{i in row r} V[i, :]        (one warp per row)
//   pass 2  Z[i, :] = sum_{r in column i} U[r, :]      (one warp per chunk of a column)
// where a warp covers one slab, lane l the columns 2l and 2l+1, so every index
// of the pattern fetches one 256-byte (FP32) or 512-byte (FP64) row segment.
// The grid's y dimension walks the slabs in order, so one slab's V and U
// (25.6 MB and 51 MB at 100,000 x 200,000 and FP32) are what the L2 holds at
// a time. Inner iterations gather FP32 copies of the vectors with FP32
// accumulation; CG vectors, dot products, norms, the coarse level (the
// Cholesky factors and the coarse products) and the true residual stay FP64, the true
// residual restarting CG on the correction (iterative refinement) until it
// meets the tolerance. Each system keeps its own CG scalars and stops on its
// own residual (Section 4's relative residual); finished slabs are skipped.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "handle.h"
#include "kernels.h"

namespace rr {

constexpr int kSlab = 64;            // systems per slab
constexpr int kBEpiBlocks = 304;     // feature chunks of the vector kernels (fixed: deterministic partials)
constexpr int64_t kUnitRows = 256;   // pass-2 chunk: at most this many rows of one column per
                                     // warp (FP32 sums over <= 256 terms, as the single-system
                                     // pieces; chunks are added in FP64)

struct BatchCol {   // CG state of one system
  double lambda, omega;
  double rho, rho_old, beta, pq, alpha, rr, bnorm, target, true_rr;
  int32_t conv, first, iters, nonfinite;
};
struct BatchGlobal {
  int32_t iter, limit, any_active, rounds;   // rounds: refinement rounds run by the graph
};

enum BEpiMode : int32_t { BEPI_PRE = 0, BEPI_POST = 1, BEPI_PCG = 2, BEPI_RESID = 3 };
struct BEpi {
  int32_t mode;
  const double *x;   // z1 (PRE), z2 (POST), p (PCG), w (RESID)
  const double *r;   // r (PRE, POST), b (RESID)
  double *out;       // r1 (PRE), z (POST), q (PCG), rt (RESID)
  double *part;      // [kBEpiBlocks][ld] partial dots: <r,z> (POST), <p,q> (PCG), ||rt||^2 (RESID)
};
enum BFinMode : int32_t { BFIN_BNORM = 0, BFIN_RZ = 1, BFIN_PQ = 2, BFIN_RR = 3, BFIN_TRUE = 4 };

// The SpMM variant: C columns per lane (slabs of 32 C systems), UNROLL row
// segments in flight per warp. Every variant sums every column in the same
// order, so the choice changes the speed only.
struct SpmmConfig {
  int32_t C = 2, unroll = 8;
};

struct BatchState {
  int32_t cap_ld = 0, cap_lam = 0;     // workspace capacity (columns, weights)
  int32_t k = 0;
  int64_t n_units2 = 0;
  int64_t *ubeg2 = nullptr, *uend2 = nullptr, *uptr2 = nullptr;
  double *b = nullptr, *w = nullptr, *r = nullptr, *r1 = nullptr, *z1 = nullptr, *z2 = nullptr,
         *z = nullptr, *p = nullptr, *q = nullptr, *rt = nullptr, *part = nullptr, *ip = nullptr,
         *U64 = nullptr, *Zp64 = nullptr;
  float *V = nullptr, *U = nullptr, *Zp = nullptr;
  double *rcB = nullptr, *ecB = nullptr, *AinvB = nullptr;   // coarse level (FP64)
  double *Ac = nullptr, *Lw = nullptr, *Linv = nullptr, *Ainv = nullptr, *lam_dev = nullptr,
         *omega_dev = nullptr;
  unsigned long long *max_bits = nullptr;
  BatchCol *col = nullptr, *col_host = nullptr;
  BatchGlobal *g = nullptr, *g_host = nullptr;
  int32_t *slab_active = nullptr, *slab_host = nullptr, *flag = nullptr, *flag_host = nullptr;
  int32_t *state = nullptr, *restarts = nullptr;      // [ld] refinement state on the device
  int32_t *state_host = nullptr, *restarts_host = nullptr;
  cudaStream_t cs = nullptr;
  SpmmConfig spmm;                     // the FP32 SpMM variant in use (autotuned)
  double spmm_ms = 0.0;                // its time for one apply (both passes, all slabs)
  DevArena mem;
};

namespace {

// C consecutive values of T loaded and stored together (C = 1, 2 or 4).
template <class T, int C>
struct Pack {
  T v[C];
};
template <class T, int C>
__device__ __forceinline__ Pack<T, C> load_pack(const T *p) {
  Pack<T, C> r;
  if constexpr (C == 4 && sizeof(T) == 4) {
    const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
  } else if constexpr (C == 2 && sizeof(T) == 4) {
    const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
    r.v[0] = t.x; r.v[1] = t.y;
  } else if constexpr (C == 2 && sizeof(T) == 8) {
    const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
    r.v[0] = t.x; r.v[1] = t.y;
  } else {
#pragma unroll
    for (int q = 0; q < C; ++q) r.v[q] = __ldg(p + q);
  }
  return r;
}

// ---------------------------------------------------------------- sparse x dense passes

// out[u, slab] = sum over the indices of unit u of V[index, slab]. Units are
// [ubeg[u], uend[u]) ranges of idx (rows of the CSR for pass 1, column chunks
// of the CSC for pass 2). A slab is 32 C columns (lane l holds columns
// C l .. C l + C - 1); grid.y walks the slabs. The 32 indices of a step are
// loaded once, coalesced, and broadcast by shuffles; UNROLL row segments are
// in flight per warp. Every column is summed in index order, whatever C and
// UNROLL (deterministic, and the same bits for every variant the autotuner
// may pick). A slab runs when one of the 64-column activity flags it covers
// is set (slab_active: per 64 columns; null = all).
template <class T, int UNROLL, int C>
__global__ void __launch_bounds__(kThreads) k_bspmm(int64_t n_units, const int64_t *__restrict__ ubeg,
                                                    const int64_t *__restrict__ uend,
                                                    const int32_t *__restrict__ idx,
                                                    const T *__restrict__ V, int64_t ldv,
                                                    T *__restrict__ out, int64_t ldo,
                                                    const int32_t *__restrict__ slab_active) {
  pdl_wait();
  constexpr int W = 32 * C;
  const int64_t col0 = (int64_t)blockIdx.y * W;
  if (slab_active) {
    bool any = false;
    for (int64_t s = col0 / kSlab; s <= (col0 + W - 1) / kSlab; ++s) any |= slab_active[s] != 0;
    if (!any) return;
  }
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const T *Vs = V + col0 + C * lane;
  for (int64_t u = warp; u < n_units; u += nwarps) {
    const int64_t b = ubeg[u], e = uend[u];
    T a[C];
#pragma unroll
    for (int q = 0; q < C; ++q) a[q] = 0;
    for (int64_t p0 = b; p0 < e; p0 += 32) {
      const int cnt = (int)min((int64_t)32, e - p0);
      const int32_t mine = lane < cnt ? __ldg(idx + p0 + lane) : 0;
      int j = 0;
      for (; j + UNROLL <= cnt; j += UNROLL) {
        Pack<T, C> t[UNROLL];
#pragma unroll
        for (int s = 0; s < UNROLL; ++s) {
          const int32_t i = __shfl_sync(0xffffffffu, mine, j + s);
          t[s] = load_pack<T, C>(Vs + (int64_t)i * ldv);
        }
#pragma unroll
        for (int s = 0; s < UNROLL; ++s)
#pragma unroll
          for (int q = 0; q < C; ++q) a[q] += t[s].v[q];
      }
      for (; j < cnt; ++j) {
        const int32_t i = __shfl_sync(0xffffffffu, mine, j);
        const Pack<T, C> t = load_pack<T, C>(Vs + (int64_t)i * ldv);
#pragma unroll
        for (int q = 0; q < C; ++q) a[q] += t.v[q];
      }
    }
    T *o = out + u * ldo + col0 + C * lane;
#pragma unroll
    for (int q = 0; q < C; ++q) o[q] = a[q];
  }
}

// ---------------------------------------------------------------- vector kernels
// Block = 64 columns (tx) x 4 feature lanes (ty); blockIdx.y = slab; blockIdx.x
// = one of kBEpiBlocks contiguous feature chunks. Partial dots per (chunk,
// column) are reduced over ty in a fixed order.

__device__ __forceinline__ void chunk_of(int64_t F, int64_t &f0, int64_t &f1) {
  f0 = F * (int64_t)blockIdx.x / gridDim.x;
  f1 = F * (int64_t)(blockIdx.x + 1) / gridDim.x;
}

__device__ __forceinline__ void write_part(double *part, int64_t ld, int64_t c, bool valid,
                                           double v) {
  __shared__ double red[4][kSlab];
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  red[ty][tx] = v;
  __syncthreads();
  if (ty == 0 && valid)
    part[(int64_t)blockIdx.x * ld + c] = ((red[0][tx] + red[1][tx]) + red[2][tx]) + red[3][tx];
}

__device__ __forceinline__ double jacobi_d(const int64_t *col_ptr, int64_t f, double lam) {
  return (double)(col_ptr[f + 1] - col_ptr[f]) + lam;
}

// After pass 2: Z = sum of the unit partials of each feature, then the mode's
// update (the batched counterpart of the single-system epilogue).
template <class T>
__global__ void __launch_bounds__(kThreads) k_bepi(int64_t F, int32_t S, int64_t ld,
                                                   const int64_t *__restrict__ uptr,
                                                   const T *__restrict__ Zp,
                                                   const int64_t *__restrict__ col_ptr,
                                                   const BatchCol *__restrict__ col, BEpi ep) {
  pdl_wait();
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int64_t c = (int64_t)blockIdx.y * kSlab + tx;
  const bool valid = c < S;
  const bool active = valid && (ep.mode == BEPI_RESID || !col[c].conv);
  const double lam = valid ? col[c].lambda : 0.0, om = valid ? col[c].omega : 0.0;
  int64_t f0, f1;
  chunk_of(F, f0, f1);
  double dot = 0.0;
  if (active) {
    for (int64_t f = f0 + ty; f < f1; f += 4) {
      double t = 0.0;
      for (int64_t u = uptr[f]; u < uptr[f + 1]; ++u) t += (double)Zp[u * ld + c];
      const int64_t o = f * ld + c;
      const double x = ep.x[o];
      t += lam * x;
      switch (ep.mode) {
        case BEPI_PRE:
          ep.out[o] = ep.r[o] - t;
          break;
        case BEPI_POST: {
          const double rr = ep.r[o];
          const double zz = x + om * (rr - t) / jacobi_d(col_ptr, f, lam);
          ep.out[o] = zz;
          dot += rr * zz;
          break;
        }
        case BEPI_PCG:
          ep.out[o] = t;
          dot += x * t;
          break;
        default: {
          const double rt = ep.r[o] - t;
          ep.out[o] = rt;
          dot += rt * rt;
          break;
        }
      }
    }
  }
  if (ep.part) write_part(ep.part, ld, c, valid, dot);
}

// b = X^T y_(c mod nrhs) from the RHS pass's unit partials (ld_y columns);
// w = 0; r = b; z1 = omega D^-1 r; V = fp32(z1); partial ||b||^2.
__global__ void __launch_bounds__(kThreads) k_bstart(int64_t F, int32_t S, int32_t nrhs, int64_t ld,
                                                     const int64_t *__restrict__ uptr,
                                                     const double *__restrict__ Zy, int64_t ldy,
                                                     const int64_t *__restrict__ col_ptr,
                                                     const BatchCol *__restrict__ col,
                                                     double *__restrict__ b, double *__restrict__ w,
                                                     double *__restrict__ r, double *__restrict__ z1,
                                                     float *__restrict__ V, double *__restrict__ part) {
  pdl_wait();
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int64_t c = (int64_t)blockIdx.y * kSlab + tx;
  const bool valid = c < S;
  const double lam = valid ? col[c].lambda : 0.0, om = valid ? col[c].omega : 0.0;
  const int64_t j = valid ? c % nrhs : 0;
  int64_t f0, f1;
  chunk_of(F, f0, f1);
  double dot = 0.0;
  for (int64_t f = f0 + ty; f < f1; f += 4) {
    const int64_t o = f * ld + c;
    if (valid) {
      double t = 0.0;
      for (int64_t u = uptr[f]; u < uptr[f + 1]; ++u) t += Zy[u * ldy + j];
      const double zz = om * t / jacobi_d(col_ptr, f, lam);
      b[o] = t;
      w[o] = 0.0;
      r[o] = t;
      z1[o] = zz;
      V[o] = (float)zz;
      dot += t * t;
    } else {
      b[o] = 0.0;
      w[o] = 0.0;
      r[o] = 0.0;
      z1[o] = 0.0;
      V[o] = 0.0f;
    }
  }
  write_part(part, ld, c, valid, dot);
}

// Restart of flagged systems on the true residual: r = rt; z1 = omega D^-1 r; V = fp32(z1).
__global__ void __launch_bounds__(kThreads) k_brestart(int64_t F, int32_t S, int64_t ld,
                                                       const int32_t *__restrict__ flag,
                                                       const int64_t *__restrict__ col_ptr,
                                                       const BatchCol *__restrict__ col,
                                                       const double *__restrict__ rt,
                                                       double *__restrict__ r, double *__restrict__ z1,
                                                       float *__restrict__ V) {
  pdl_wait();
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int64_t c = (int64_t)blockIdx.y * kSlab + tx;
  if (c >= S || !flag[c]) return;
  const double lam = col[c].lambda, om = col[c].omega;
  int64_t f0, f1;
  chunk_of(F, f0, f1);
  for (int64_t f = f0 + ty; f < f1; f += 4) {
    const int64_t o = f * ld + c;
    const double rr = rt[o];
    const double zz = om * rr / jacobi_d(col_ptr, f, lam);
    r[o] = rr;
    z1[o] = zz;
    V[o] = (float)zz;
  }
}

// Restriction, pass 1: item partials ip[item, c] = sum over the item's members
// of r1[member, c] (items: ranges of at most kRestrictItemBatch members of one cluster).
__global__ void __launch_bounds__(kThreads) k_brestrict(const RestrictItem *__restrict__ items,
                                                        int32_t n_items, int32_t S, int64_t ld,
                                                        const int32_t *__restrict__ members,
                                                        const double *__restrict__ r1,
                                                        const BatchCol *__restrict__ col,
                                                        double *__restrict__ ip) {
  pdl_wait();
  __shared__ double red[4][kSlab];
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int64_t c = (int64_t)blockIdx.y * kSlab + tx;
  const bool active = c < S && !col[c].conv;
  for (int32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
    const RestrictItem w = items[it];
    double acc = 0.0;
    if (active)
      for (int32_t m = w.begin + ty; m < w.end; m += 4) acc += r1[(int64_t)members[m] * ld + c];
    red[ty][tx] = acc;
    __syncthreads();
    if (ty == 0 && active) ip[(int64_t)it * ld + c] = ((red[0][tx] + red[1][tx]) + red[2][tx]) + red[3][tx];
    __syncthreads();
  }
}

// Restriction, pass 2: rc[S, c] = s_S * (item partials of S, in order).
__global__ void __launch_bounds__(kThreads) k_bcombine(int32_t k, int32_t kpad, int32_t S, int64_t ld,
                                                       const int32_t *__restrict__ item_ptr,
                                                       const double *__restrict__ ip,
                                                       const double *__restrict__ s,
                                                       const BatchCol *__restrict__ col,
                                                       double *__restrict__ rc) {
  pdl_wait();
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int64_t c = (int64_t)blockIdx.y * kSlab + tx;
  const bool active = c < S && !col[c].conv;
  for (int32_t cl = blockIdx.x * 4 + ty; cl < kpad; cl += gridDim.x * 4) {
    double acc = 0.0;
    if (active && cl < k) {
      for (int32_t q = item_ptr[cl]; q < item_ptr[cl + 1]; ++q) acc += ip[(int64_t)q * ld + c];
      acc *= s[cl];
    }
    rc[(int64_t)cl * ld + c] = acc;
  }
}

// Restriction of the remaining error e - z1 = (wref - w) - z1 (rr_harvest's
// targets), item partials as k_brestrict.
__global__ void __launch_bounds__(kThreads) k_brestrict_err(const RestrictItem *__restrict__ items,
                                                            int32_t n_items, int32_t S, int64_t ld,
                                                            const int32_t *__restrict__ members,
                                                            const double *__restrict__ wref,
                                                            const double *__restrict__ w,
                                                            const double *__restrict__ z1,
                                                            const BatchCol *__restrict__ col,
                                                            double *__restrict__ ip) {
  pdl_wait();
  __shared__ double red[4][kSlab];
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int64_t c = (int64_t)blockIdx.y * kSlab + tx;
  const bool active = c < S && !col[c].conv;
  for (int32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
    const RestrictItem q = items[it];
    double acc = 0.0;
    if (active)
      for (int32_t m = q.begin + ty; m < q.end; m += 4) {
        const int64_t o = (int64_t)members[m] * ld + c;
        acc += (wref[o] - w[o]) - z1[o];
      }
    red[ty][tx] = acc;
    __syncthreads();
    if (ty == 0 && active) ip[(int64_t)it * ld + c] = ((red[0][tx] + red[1][tx]) + red[2][tx]) + red[3][tx];
    __syncthreads();
  }
}

// One block per system c still iterating: its pair (r_c, P^T (e - z1)) into
// slot iter * S + c (FP32 rows of k).
__global__ void k_bharvest(int32_t S, int64_t ld, int32_t k, const double *__restrict__ rc,
                           const double *__restrict__ rcE, const BatchCol *__restrict__ col,
                           const BatchGlobal *__restrict__ g, float *__restrict__ Xs,
                           float *__restrict__ Ts, int64_t *__restrict__ valid, int64_t slots) {
  pdl_wait();
  const int64_t c = blockIdx.x;
  if (c >= S || col[c].conv) return;
  const int64_t slot = (int64_t)g->iter * S + c;
  if (slot >= slots) return;
  for (int32_t q = threadIdx.x; q < k; q += blockDim.x) {
    Xs[slot * k + q] = (float)rc[(int64_t)q * ld + c];
    Ts[slot * k + q] = (float)rcE[(int64_t)q * ld + c];
  }
  if (threadIdx.x == 0) valid[slot] = 1;
}

// Compaction of the written slots, in slot order (pos = exclusive scan of valid).
__global__ void k_bcompact(int64_t slots, int32_t k, const int64_t *__restrict__ valid,
                           const int64_t *__restrict__ pos, const float *__restrict__ Xs,
                           const float *__restrict__ Ts, float *__restrict__ Xp,
                           float *__restrict__ Tp, int64_t max_pairs) {
  for (int64_t sl = blockIdx.x; sl < slots; sl += gridDim.x) {
    if (!valid[sl] || pos[sl] >= max_pairs) continue;
    const int64_t d = pos[sl];
    for (int32_t q = threadIdx.x; q < k; q += blockDim.x) {
      Xp[d * k + q] = Xs[sl * k + q];
      Tp[d * k + q] = Ts[sl * k + q];
    }
  }
}

// Coarse solve e_c = A_c(lambda_c)^-1 r_c for every system in FP64 (as in the
// single-system path): a 64 x 64 output tile per block (coarse rows x
// systems), K in steps of 16 through shared memory, 4 x 4 outputs per thread.
// Column c takes the inverse of its weight, l(c) = c / nrhs; a tile whose
// systems span several weights makes one pass per weight with the other
// columns masked.
constexpr int kCT = 64, kCK = 16;
__global__ void __launch_bounds__(kThreads) k_bcoarse(int32_t k, int32_t kpad, int32_t S, int32_t nrhs,
                                                      int64_t ld, const double *__restrict__ Ainv,
                                                      const double *__restrict__ rc,
                                                      const BatchCol *__restrict__ col,
                                                      double *__restrict__ ec) {
  pdl_wait();
  __shared__ double As[kCK][kCT + 2];
  __shared__ double Bs[kCK][kCT + 2];
  const int i0 = blockIdx.x * kCT;
  const int64_t c0 = (int64_t)blockIdx.y * kCT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t clast = (c0 + kCT < (int64_t)S ? c0 + kCT : (int64_t)S) - 1;
  double acc[4][4] = {};
  if (c0 < S) {
    const int32_t l0 = (int32_t)(c0 / nrhs), l1 = (int32_t)(clast / nrhs);
    for (int32_t l = l0; l <= l1; ++l) {
      const double *A = Ainv + (int64_t)l * kpad * kpad;
      for (int m0 = 0; m0 < kpad; m0 += kCK) {
        // A^T chunk: As[m][i] = A[i0 + i][m0 + m]; 1024 values, 4 per thread
        for (int e = threadIdx.x; e < kCK * kCT; e += kThreads) {
          const int i = e / kCK, m = e % kCK;
          As[m][i] = A[(int64_t)(i0 + i) * kpad + m0 + m];
        }
        for (int e = threadIdx.x; e < kCK * kCT; e += kThreads) {
          const int m = e / kCT, cc = e % kCT;
          const int64_t c = c0 + cc;
          const bool use = c < S && (int32_t)(c / nrhs) == l && !col[c].conv;
          Bs[m][cc] = use ? rc[(int64_t)(m0 + m) * ld + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < kCK; ++m) {
          double a[4], bb[4];
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            a[x] = As[m][ty * 4 + x];
            bb[x] = Bs[m][tx * 4 + x];
          }
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], bb[y], acc[x][y]);
        }
        __syncthreads();
      }
    }
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int i = i0 + ty * 4 + x;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t c = c0 + tx * 4 + y;
      if (i < kpad && c < ld) ec[(int64_t)i * ld + c] = acc[x][y];
    }
  }
  (void)k;
}

// Prolongation z2 = z1 + P e_c, z2[i] = z1[i] + s_l(i) e_c[l(i)]; V = fp32(z2).
__global__ void __launch_bounds__(kThreads) k_bprolong(int64_t F, int32_t S, int64_t ld,
                                                       const int32_t *__restrict__ labels,
                                                       const double *__restrict__ s,
                                                       const double *__restrict__ ec,
                                                       const BatchCol *__restrict__ col,
                                                       const double *__restrict__ z1,
                                                       double *__restrict__ z2, float *__restrict__ V) {
  pdl_wait();
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int64_t c = (int64_t)blockIdx.y * kSlab + tx;
  if (c >= S || col[c].conv) return;
  int64_t f0, f1;
  chunk_of(F, f0, f1);
  for (int64_t f = f0 + ty; f < f1; f += 4) {
    const int32_t l = labels[f];
    const int64_t o = f * ld + c;
    const double v = z1[o] + s[l] * ec[(int64_t)l * ld + c];
    z2[o] = v;
    V[o] = (float)v;
  }
}

// p = z + beta p (p = z on a (re)start); V = fp32(p).
__global__ void __launch_bounds__(kThreads) k_bdirection(int64_t F, int32_t S, int64_t ld,
                                                         const BatchCol *__restrict__ col,
                                                         const double *__restrict__ z,
                                                         double *__restrict__ p, float *__restrict__ V) {
  pdl_wait();
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int64_t c = (int64_t)blockIdx.y * kSlab + tx;
  if (c >= S || col[c].conv) return;
  const bool first = col[c].first;
  const double beta = col[c].beta;
  int64_t f0, f1;
  chunk_of(F, f0, f1);
  for (int64_t f = f0 + ty; f < f1; f += 4) {
    const int64_t o = f * ld + c;
    const double v = first ? z[o] : z[o] + beta * p[o];
    p[o] = v;
    V[o] = (float)v;
  }
}

// w += alpha p; r -= alpha q; z1 = omega D^-1 r; V = fp32(z1); partial ||r||^2.
// Block (0,0) also clears the activity flags that the finishing kernel sets again.
__global__ void __launch_bounds__(kThreads) k_bupdate(int64_t F, int32_t S, int64_t ld,
                                                      const int64_t *__restrict__ col_ptr,
                                                      const BatchCol *__restrict__ col,
                                                      const double *__restrict__ p,
                                                      const double *__restrict__ q,
                                                      double *__restrict__ w, double *__restrict__ r,
                                                      double *__restrict__ z1, float *__restrict__ V,
                                                      double *__restrict__ part, BatchGlobal *g,
                                                      int32_t *slab_active, int32_t n_slabs) {
  pdl_wait();
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    g->any_active = 0;
    for (int s = 0; s < n_slabs; ++s) slab_active[s] = 0;
  }
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int64_t c = (int64_t)blockIdx.y * kSlab + tx;
  const bool active = c < S && !col[c].conv;
  double dot = 0.0;
  if (active) {
    const double alpha = col[c].alpha, lam = col[c].lambda, om = col[c].omega;
    int64_t f0, f1;
    chunk_of(F, f0, f1);
    for (int64_t f = f0 + ty; f < f1; f += 4) {
      const int64_t o = f * ld + c;
      w[o] += alpha * p[o];
      const double rr = r[o] - alpha * q[o];
      r[o] = rr;
      dot += rr * rr;
      const double zz = om * rr / jacobi_d(col_ptr, f, lam);
      z1[o] = zz;
      V[o] = (float)zz;
    }
  }
  write_part(part, ld, c, c < S, dot);
}

// Per-system scalars from the partial dots (fixed order), one block per slab.
__global__ void __launch_bounds__(kThreads) k_bfinish(int32_t mode, int32_t S, int64_t ld,
                                                      const double *__restrict__ part, int32_t nb,
                                                      double tol, BatchCol *col, BatchGlobal *g,
                                                      int32_t *slab_active) {
  pdl_wait();
  __shared__ double red[4][kSlab];
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int64_t c = (int64_t)blockIdx.x * kSlab + tx;
  double v = 0.0;
  if (c < S)
    for (int32_t b = ty; b < nb; b += 4) v += part[(int64_t)b * ld + c];
  red[ty][tx] = v;
  __syncthreads();
  if (mode == BFIN_RR && blockIdx.x == 0 && threadIdx.x == 0) g->iter += 1;
  if (ty != 0 || c >= S) return;
  const double sum = ((red[0][tx] + red[1][tx]) + red[2][tx]) + red[3][tx];
  BatchCol &C = col[c];
  switch (mode) {
    case BFIN_BNORM: {
      C.bnorm = sqrt(sum);
      C.target = tol * C.bnorm;
      C.rr = sum;
      C.rho_old = 0.0;
      C.first = 1;
      C.iters = 0;
      C.nonfinite = isfinite(sum) ? 0 : 1;
      C.conv = (C.nonfinite || C.bnorm == 0.0) ? 1 : 0;
      if (!C.conv) {
        atomicOr(&slab_active[blockIdx.x], 1);
        atomicOr(&g->any_active, 1);
      }
      break;
    }
    case BFIN_RZ:
      if (C.conv) break;
      C.rho = sum;
      C.beta = C.first ? 0.0 : sum / C.rho_old;
      break;
    case BFIN_PQ:
      if (C.conv) break;
      C.pq = sum;
      C.alpha = C.rho / sum;
      if (!isfinite(C.alpha)) {
        C.nonfinite = 1;
        C.conv = 1;
      }
      break;
    case BFIN_RR:
      if (C.conv) break;
      C.rr = sum;
      C.rho_old = C.rho;
      C.first = 0;
      C.iters += 1;
      if (!isfinite(sum) || !isfinite(C.rho)) {
        C.nonfinite = 1;
        C.conv = 1;
      } else if (sqrt(sum) <= C.target) {
        C.conv = 1;
      } else {
        atomicOr(&slab_active[blockIdx.x], 1);
        atomicOr(&g->any_active, 1);
      }
      break;
    default:   // BFIN_TRUE
      C.true_rr = sum;
      break;
  }
}

__global__ void k_bloop_condition(cudaGraphConditionalHandle hc, const BatchGlobal *__restrict__ g) {
  pdl_wait();
  if (threadIdx.x == 0) cudaGraphSetConditional(hc, (g->any_active && g->iter < g->limit) ? 1u : 0u);
}

// ---- iterative refinement on the device (the rules of the host-driven loop)

__global__ void k_brefine_clear(BatchGlobal *g, int32_t *slab_active, int32_t n_slabs) {
  pdl_wait();
  if (threadIdx.x == 0) g->any_active = 0;
  for (int32_t s = threadIdx.x; s < n_slabs; s += blockDim.x) slab_active[s] = 0;
}

// After a true residual: a system is done when ||b - A w|| meets its target;
// it has failed on a non-finite value or at the iteration or restart cap;
// otherwise it restarts CG from w on the true residual with a fresh direction
// (flag[c] = 1, its slab and the loop marked active). state: 0 running, 1
// done, 2 failed.
__global__ void k_brefine(int32_t S, BatchCol *col, int32_t *state, int32_t *restarts,
                          int32_t max_restarts, int32_t max_iter, BatchGlobal *g, int32_t *flag,
                          int32_t *slab_active) {
  pdl_wait();
  const int32_t iter = g->iter;
  for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < S; c += gridDim.x * blockDim.x) {
    flag[c] = 0;
    if (state[c] != 0) continue;
    BatchCol &C = col[c];
    if (C.nonfinite || !isfinite(C.true_rr)) {
      state[c] = 2;
      continue;
    }
    if (sqrt(C.true_rr) <= C.target) {
      state[c] = 1;
      continue;
    }
    if (iter >= max_iter || restarts[c] >= max_restarts) {
      state[c] = 2;
      continue;
    }
    restarts[c] += 1;
    C.conv = 0;
    C.first = 1;
    C.rr = C.true_rr;
    flag[c] = 1;
    atomicOr(&slab_active[c / kSlab], 1);
    atomicOr(&g->any_active, 1);
  }
}

// End of a refinement round: another round while a system restarted.
__global__ void k_bround_condition(cudaGraphConditionalHandle outer, BatchGlobal *g) {
  pdl_wait();
  if (threadIdx.x == 0) {
    g->rounds += 1;
    cudaGraphSetConditional(outer, g->any_active ? 1u : 0u);
  }
}

// Y (nrhs targets of length N, target j at Y + j N) -> Yr (N x ldy row-major, zero padding).
__global__ void k_btranspose_in(int64_t N, int32_t nrhs, int64_t ldy, const double *__restrict__ Y,
                                double *__restrict__ Yr) {
  __shared__ double t[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int j = j0 + y;
    const int64_t r = r0 + threadIdx.x;
    t[y][threadIdx.x] = (j < nrhs && r < N) ? Y[(int64_t)j * N + r] : 0.0;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t r = r0 + y;
    const int j = j0 + threadIdx.x;
    if (r < N && j < ldy) Yr[r * ldy + j] = t[threadIdx.x][y];
  }
}

// w (F x ld row-major) -> W (system c at W + c F), c < S.
__global__ void k_btranspose_out(int64_t F, int32_t S, int64_t ld, const double *__restrict__ w,
                                 double *__restrict__ W) {
  __shared__ double t[32][33];
  const int64_t f0 = (int64_t)blockIdx.x * 32;
  const int64_t c0 = (int64_t)blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t f = f0 + y, c = c0 + threadIdx.x;
    t[y][threadIdx.x] = (f < F && c < S) ? w[f * ld + c] : 0.0;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t c = c0 + y, f = f0 + threadIdx.x;
    if (c < S && f < F) W[c * F + f] = t[threadIdx.x][y];
  }
}

// Damping per weight: omega_l = 1 / max_i (gsum_i + lambda_l) / (colnnz_i + lambda_l)
// (the Gershgorin bound of the single-system setup), through the order-preserving
// bits of positive doubles.
__global__ void k_bomega_max(int64_t F, int32_t nlam, const double *__restrict__ lam,
                             const int64_t *__restrict__ col_ptr, const int64_t *__restrict__ gsum,
                             unsigned long long *__restrict__ max_bits) {
  for (int32_t l = 0; l < nlam; ++l) {
    unsigned long long best = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
         i += (int64_t)gridDim.x * blockDim.x) {
      const double di = (double)(col_ptr[i + 1] - col_ptr[i]) + lam[l];
      const double ratio = ((double)gsum[i] + lam[l]) / di;
      const unsigned long long bits = (unsigned long long)__double_as_longlong(ratio);
      best = bits > best ? bits : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long t = __shfl_xor_sync(0xffffffffu, best, o);
      best = t > best ? t : best;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&max_bits[l], best);
  }
}

__global__ void k_bomega(int32_t nlam, const unsigned long long *__restrict__ max_bits,
                         double *__restrict__ omega) {
  for (int32_t l = threadIdx.x; l < nlam; l += blockDim.x)
    omega[l] = 1.0 / __longlong_as_double((long long)max_bits[l]);
}

// The k x k inverse into a kpad x kpad block (zero padding).
__global__ void k_binv_pad(int32_t k, int32_t kpad, const double *__restrict__ Ainv,
                           double *__restrict__ out) {
  const int64_t n = (int64_t)kpad * kpad;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / kpad, j = e % kpad;
    out[e] = (i < k && j < k) ? Ainv[i * k + j] : 0.0;
  }
}

// ---------------------------------------------------------------- host side

inline int64_t round_up64(int64_t a) { return (a + kSlab - 1) / kSlab * kSlab; }

template <class T, int U, int C>
rr_status launch_bspmm_v(int64_t n_units, const int64_t *ubeg, const int64_t *uend,
                         const int32_t *idx, const T *V, int64_t ldv, T *out, int64_t ldo,
                         int64_t ld, const int32_t *slab_active, cudaStream_t st) {
  const dim3 grid((unsigned)grid_for(n_units, kWarps), (unsigned)(ld / (32 * C)));
  RR_LAUNCH_PDL((k_bspmm<T, U, C>), grid, kThreads, 0, st, n_units, ubeg, uend, idx, V, ldv, out,
                ldo, slab_active);
  return RR_OK;
}

// ld columns (a multiple of 64; of 128 when C = 4) of V through the pattern.
template <class T>
rr_status launch_bspmm(int64_t n_units, const int64_t *ubeg, const int64_t *uend, const int32_t *idx,
                       const T *V, int64_t ldv, T *out, int64_t ldo, int64_t ld,
                       const int32_t *slab_active, cudaStream_t st,
                       SpmmConfig cfg = SpmmConfig{2, sizeof(T) == 4 ? 8 : 4}) {
#define RR_BSPMM(U_, C_)                                                                    \
  if (cfg.unroll == U_ && cfg.C == C_)                                                      \
    return launch_bspmm_v<T, U_, C_>(n_units, ubeg, uend, idx, V, ldv, out, ldo, ld,        \
                                     slab_active, st);
  RR_BSPMM(4, 1) RR_BSPMM(4, 2) RR_BSPMM(8, 1) RR_BSPMM(8, 2)
  if constexpr (sizeof(T) == 4) {
    RR_BSPMM(4, 4) RR_BSPMM(8, 4)
  }
#undef RR_BSPMM
  rr_set_error("batched SpMM: no variant with %d columns per lane, unroll %d", cfg.C, cfg.unroll);
  return RR_UNSUPPORTED;
}

// Training-pair capture of rr_harvest (see include/rr.h): slot it * S + c
// holds the pair of system c at iteration it.
struct Harvest {
  const double *wref;   // [F x ld] the reference solutions
  double *ipE, *rcE;    // restriction of e - z1 (item partials, coarse)
  float *Xs, *Ts;       // [slots x k]
  int64_t *valid;       // [slots] 1 where a pair was written
  int64_t slots;
};

struct BatchRun {
  rr_handle *h;
  BatchState *B;
  int32_t S, nrhs, nlam, n_slabs;
  int64_t ld;
  double tol;
  const Harvest *hv;
};

// The operator's two passes on the FP32 stage V; result partials in Zp.
rr_status bapply_f32(const BatchRun &R, cudaStream_t st) {
  rr_handle *h = R.h;
  BatchState *B = R.B;
  RR_TRY(launch_bspmm<float>(h->N, h->row_ptr, h->row_ptr + 1, h->col_idx, B->V, R.ld, B->U, R.ld,
                             R.ld, B->slab_active, st, B->spmm));
  RR_TRY(launch_bspmm<float>(B->n_units2, B->ubeg2, B->uend2, h->row_idx, B->U, R.ld, B->Zp, R.ld,
                             R.ld, B->slab_active, st, B->spmm));
  return RR_OK;
}

rr_status bepilogue_f32(const BatchRun &R, const BEpi &ep, cudaStream_t st) {
  const dim3 grid(kBEpiBlocks, (unsigned)R.n_slabs);
  RR_LAUNCH_PDL(k_bepi<float>, grid, kThreads, 0, st, R.h->F, R.S, R.ld, R.B->uptr2, R.B->Zp,
            R.h->col_ptr, R.B->col, ep);
  return RR_OK;
}

rr_status bfinish(const BatchRun &R, int32_t mode, cudaStream_t st) {
  RR_LAUNCH_PDL(k_bfinish, (unsigned)R.n_slabs, kThreads, 0, st, mode, R.S, R.ld, R.B->part,
            kBEpiBlocks, R.tol, R.B->col, R.B->g, R.B->slab_active);
  return RR_OK;
}

// One batched PCG iteration (the single-system iteration, column by column).
rr_status biteration(const BatchRun &R, cudaStream_t st) {
  rr_handle *h = R.h;
  BatchState *B = R.B;
  const int64_t F = h->F;
  const dim3 vgrid(kBEpiBlocks, (unsigned)R.n_slabs);
  const int32_t kpad = (int32_t)round_up64(B->k);
  // pre-smoothing: z1 (staged in V by the previous update); r1 = r - A z1
  RR_TRY(bapply_f32(R, st));
  RR_TRY(bepilogue_f32(R, BEpi{BEPI_PRE, B->z1, B->r, B->r1, nullptr}, st));
  // coarse correction: r_c = P^T r1; e_c = A_c^-1 r_c; z2 = z1 + P e_c
  const RestrictPlan &pl = h->bplan;
  RR_LAUNCH_PDL(k_brestrict, dim3((unsigned)std::max(1, std::min(pl.n_items, kSMs * 4)), (unsigned)R.n_slabs),
            kThreads, 0, st, pl.items, pl.n_items, R.S, R.ld, h->members, B->r1, B->col, B->ip);
  RR_LAUNCH_PDL(k_bcombine, dim3((unsigned)((kpad + 3) / 4), (unsigned)R.n_slabs), kThreads, 0, st,
            B->k, kpad, R.S, R.ld, pl.item_ptr, B->ip, h->s, B->col, B->rcB);
  if (R.hv) {
    const Harvest &hv = *R.hv;
    RR_LAUNCH_PDL(k_brestrict_err, dim3((unsigned)std::max(1, std::min(pl.n_items, kSMs * 4)), (unsigned)R.n_slabs),
              kThreads, 0, st, pl.items, pl.n_items, R.S, R.ld, h->members, hv.wref, B->w, B->z1,
              B->col, hv.ipE);
    RR_LAUNCH_PDL(k_bcombine, dim3((unsigned)((kpad + 3) / 4), (unsigned)R.n_slabs), kThreads, 0, st,
              B->k, kpad, R.S, R.ld, pl.item_ptr, hv.ipE, h->s, B->col, hv.rcE);
    RR_LAUNCH_PDL(k_bharvest, (unsigned)R.S, kThreads, 0, st, R.S, R.ld, B->k, B->rcB, hv.rcE, B->col,
              B->g, hv.Xs, hv.Ts, hv.valid, hv.slots);
  }
  RR_LAUNCH_PDL(k_bcoarse, dim3((unsigned)(kpad / kCT), (unsigned)R.n_slabs), kThreads, 0, st, B->k,
            kpad, R.S, R.nrhs, R.ld, B->AinvB, B->rcB, B->col, B->ecB);
  RR_LAUNCH_PDL(k_bprolong, vgrid, kThreads, 0, st, F, R.S, R.ld, h->labels, h->s, B->ecB, B->col,
            B->z1, B->z2, B->V);
  // post-smoothing: r2 = r - A z2; z = z2 + omega D^-1 r2; <r, z>
  RR_TRY(bapply_f32(R, st));
  RR_TRY(bepilogue_f32(R, BEpi{BEPI_POST, B->z2, B->r, B->z, B->part}, st));
  RR_TRY(bfinish(R, BFIN_RZ, st));
  // direction and q = A p; <p, q>
  RR_LAUNCH_PDL(k_bdirection, vgrid, kThreads, 0, st, F, R.S, R.ld, B->col, B->z, B->p, B->V);
  RR_TRY(bapply_f32(R, st));
  RR_TRY(bepilogue_f32(R, BEpi{BEPI_PCG, B->p, nullptr, B->q, B->part}, st));
  RR_TRY(bfinish(R, BFIN_PQ, st));
  // update; ||r||^2; stopping test
  RR_LAUNCH_PDL(k_bupdate, vgrid, kThreads, 0, st, F, R.S, R.ld, h->col_ptr, B->col, B->p, B->q, B->w,
            B->r, B->z1, B->V, B->part, B->g, B->slab_active, R.n_slabs);
  RR_TRY(bfinish(R, BFIN_RR, st));
  return RR_OK;
}

// FP64 true residual rt = b - A w of every system, ||rt||^2 into col[c].true_rr.
rr_status btrue_residual(const BatchRun &R, cudaStream_t st) {
  rr_handle *h = R.h;
  BatchState *B = R.B;
  RR_TRY(launch_bspmm<double>(h->N, h->row_ptr, h->row_ptr + 1, h->col_idx, B->w, R.ld, B->U64,
                              R.ld, R.ld, nullptr, st));
  RR_TRY(launch_bspmm<double>(B->n_units2, B->ubeg2, B->uend2, h->row_idx, B->U64, R.ld, B->Zp64,
                              R.ld, R.ld, nullptr, st));
  const dim3 grid(kBEpiBlocks, (unsigned)R.n_slabs);
  RR_LAUNCH_PDL(k_bepi<double>, grid, kThreads, 0, st, h->F, R.S, R.ld, B->uptr2, B->Zp64, h->col_ptr,
            B->col, BEpi{BEPI_RESID, B->w, B->b, B->rt, B->part});
  RR_TRY(bfinish(R, BFIN_TRUE, st));
  return RR_OK;
}

// Pass-2 units: each column of the CSC cut into chunks of at most kUnitRows rows.
rr_status build_units(rr_handle *h, BatchState *B) {
  const int64_t F = h->F;
  std::vector<int64_t> cp(F + 1);
  RR_CUDA(cudaMemcpyAsync(cp.data(), h->col_ptr, sizeof(int64_t) * (F + 1), cudaMemcpyDeviceToHost, h->st));
  RR_CUDA(cudaStreamSynchronize(h->st));
  std::vector<int64_t> ub, ue, up(F + 1);
  for (int64_t f = 0; f < F; ++f) {
    up[f] = (int64_t)ub.size();
    for (int64_t b = cp[f]; b < cp[f + 1]; b += kUnitRows) {
      ub.push_back(b);
      ue.push_back(std::min(cp[f + 1], b + kUnitRows));
    }
  }
  up[F] = (int64_t)ub.size();
  B->n_units2 = (int64_t)ub.size();
  RR_TRY(B->mem.alloc(&B->ubeg2, ub.size()));
  RR_TRY(B->mem.alloc(&B->uend2, ue.size()));
  RR_TRY(B->mem.alloc(&B->uptr2, F + 1));
  if (!ub.empty()) {
    RR_CUDA(cudaMemcpyAsync(B->ubeg2, ub.data(), sizeof(int64_t) * ub.size(), cudaMemcpyHostToDevice, h->st));
    RR_CUDA(cudaMemcpyAsync(B->uend2, ue.data(), sizeof(int64_t) * ue.size(), cudaMemcpyHostToDevice, h->st));
  }
  RR_CUDA(cudaMemcpyAsync(B->uptr2, up.data(), sizeof(int64_t) * (F + 1), cudaMemcpyHostToDevice, h->st));
  RR_CUDA(cudaStreamSynchronize(h->st));
  return RR_OK;
}

rr_status batch_reserve(rr_handle *h, int64_t ld, int32_t nlam) {
  BatchState *B = h->batch;
  if (B && B->cap_ld >= ld && B->cap_lam >= nlam) return RR_OK;
  if (B) {
    batch_free(B);
    h->batch = nullptr;
  }
  B = new BatchState();
  h->batch = B;
  const int64_t F = h->F, N = h->N;
  const int32_t k = h->k_eff;
  const int64_t kpad = round_up64(k);
  B->k = k;
  B->cap_ld = (int32_t)ld;
  B->cap_lam = nlam;
  RR_TRY(build_units(h, B));
  const size_t fv = (size_t)F * ld;
  double **vecs[] = {&B->b, &B->w, &B->r, &B->r1, &B->z1, &B->z2, &B->z, &B->p, &B->q, &B->rt};
  for (double **v : vecs) RR_TRY(B->mem.alloc(v, fv));
  RR_TRY(B->mem.alloc(&B->part, (size_t)kBEpiBlocks * ld));
  RR_TRY(B->mem.alloc(&B->ip, (size_t)std::max(1, h->bplan.n_items) * ld));
  RR_TRY(B->mem.alloc(&B->U64, (size_t)N * ld));
  RR_TRY(B->mem.alloc(&B->Zp64, (size_t)std::max<int64_t>(1, B->n_units2) * ld));
  RR_TRY(B->mem.alloc(&B->V, fv));
  RR_TRY(B->mem.alloc(&B->U, (size_t)N * ld));
  RR_TRY(B->mem.alloc(&B->Zp, (size_t)std::max<int64_t>(1, B->n_units2) * ld));
  RR_TRY(B->mem.alloc(&B->rcB, (size_t)kpad * ld));
  RR_TRY(B->mem.alloc(&B->ecB, (size_t)kpad * ld));
  RR_TRY(B->mem.alloc(&B->AinvB, (size_t)nlam * kpad * kpad));
  const size_t kk = (size_t)k * k;
  RR_TRY(B->mem.alloc(&B->Ac, kk));
  RR_TRY(B->mem.alloc(&B->Lw, kk));
  RR_TRY(B->mem.alloc(&B->Linv, kk));
  RR_TRY(B->mem.alloc(&B->Ainv, kk));
  RR_TRY(B->mem.alloc(&B->lam_dev, nlam));
  RR_TRY(B->mem.alloc(&B->omega_dev, nlam));
  RR_TRY(B->mem.alloc(&B->max_bits, nlam));
  RR_TRY(B->mem.alloc(&B->col, ld));
  RR_TRY(B->mem.alloc(&B->g, 1));
  RR_TRY(B->mem.alloc(&B->slab_active, ld / kSlab));
  RR_TRY(B->mem.alloc(&B->flag, ld));
  RR_TRY(B->mem.alloc(&B->state, ld));
  RR_TRY(B->mem.alloc(&B->restarts, ld));
  RR_CUDA(cudaMallocHost(&B->state_host, sizeof(int32_t) * ld));
  RR_CUDA(cudaMallocHost(&B->restarts_host, sizeof(int32_t) * ld));
  RR_CUDA(cudaMallocHost(&B->col_host, sizeof(BatchCol) * ld));
  RR_CUDA(cudaMallocHost(&B->g_host, sizeof(BatchGlobal)));
  RR_CUDA(cudaMallocHost(&B->slab_host, sizeof(int32_t) * (ld / kSlab)));
  RR_CUDA(cudaMallocHost(&B->flag_host, sizeof(int32_t) * ld));
  RR_CUDA(cudaStreamCreateWithFlags(&B->cs, cudaStreamNonBlocking));
  return RR_OK;
}

// Coarse inverse and damping of every weight.
rr_status batch_factors(rr_handle *h, BatchState *B, int32_t nlam, const double *lambdas,
                        double *omega_host) {
  cudaStream_t st = h->st;
  const int32_t k = h->k_eff;
  const int32_t kpad = (int32_t)round_up64(k);
  for (int32_t l = 0; l < nlam; ++l) {
    if (h->mu) {   // the handle's eigendecomposition, reused for every weight
      RR_TRY(eig_inverse(k, h->mu, h->Qv, lambdas[l], B->Ainv, st));
    } else {
      RR_TRY(coarse_operator(k, h->G, h->s, lambdas[l], B->Ac, st));
      RR_CUDA(cudaMemcpyAsync(B->Lw, B->Ac, sizeof(double) * (size_t)k * k, cudaMemcpyDeviceToDevice, st));
      RR_TRY(cholesky(k, B->Lw, B->Linv, h->err, st));
      RR_TRY(chol_inverse(k, B->Lw, B->Linv, B->Ainv, st));
    }
    RR_LAUNCH(k_binv_pad, grid_for((int64_t)kpad * kpad, kThreads), kThreads, 0, st, k, kpad,
              B->Ainv, B->AinvB + (size_t)l * kpad * kpad);
  }
  RR_CUDA(cudaMemcpyAsync(B->lam_dev, lambdas, sizeof(double) * nlam, cudaMemcpyHostToDevice, st));
  RR_CUDA(cudaMemsetAsync(B->max_bits, 0, sizeof(unsigned long long) * nlam, st));
  RR_LAUNCH(k_bomega_max, grid_for(h->F, kThreads), kThreads, 0, st, h->F, nlam, B->lam_dev,
            h->col_ptr, h->gsum, B->max_bits);
  RR_LAUNCH(k_bomega, 1, 32, 0, st, nlam, B->max_bits, B->omega_dev);
  RR_CUDA(cudaMemcpyAsync(omega_host, B->omega_dev, sizeof(double) * nlam, cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  int32_t e = 0;
  RR_CUDA(cudaMemcpy(&e, h->err, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (e != DEV_OK) {
    RR_CUDA(cudaMemset(h->err, 0, sizeof(int32_t)));
    rr_set_error("rr_solve_batch: coarse Cholesky failed (device error %d)", e);
    return e == DEV_NOT_SPD ? RR_NOT_SPD : RR_CUDA_ERROR;
  }
  return RR_OK;
}

// The iteration loop as one graph with a conditional while node (built once per
// batched solve, launched once per refinement round).
struct LoopGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t body_kernels = 0;
  ~LoopGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (g) cudaGraphDestroy(g);
  }
};

rr_status build_loop(const BatchRun &R, LoopGraph &L) {
  BatchState *B = R.B;
  RR_CUDA(cudaGraphCreate(&L.g, 0));
  cudaGraphConditionalHandle hc;
  RR_CUDA(cudaGraphConditionalHandleCreate(&hc, L.g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hc;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  RR_CUDA(cudaGraphAddNode(&node, L.g, nullptr, nullptr, 0, &cp));
  RR_CUDA(cudaStreamBeginCaptureToGraph(B->cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal));
  const int64_t l0 = rr_launch_counter;
  rr_status s = biteration(R, B->cs);
  if (s == RR_OK) {
    k_bloop_condition<<<1, 32, 0, B->cs>>>(hc, B->g);
    ++rr_launch_counter;
  }
  L.body_kernels = rr_launch_counter - l0;   // recorded, not launched
  rr_launch_counter = l0;
  cudaGraph_t cap = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(B->cs, &cap);
  if (s != RR_OK || ec != cudaSuccess) {
    cudaGraphDestroy(L.g);
    L.g = nullptr;
    cudaGetLastError();
    if (s != RR_OK) return s;
    rr_set_error("batched loop capture failed: %s", cudaGetErrorString(ec));
    return RR_CUDA_ERROR;
  }
  RR_CUDA(cudaGraphInstantiate(&L.exec, L.g, 0));
  return RR_OK;
}

// The whole batched solve as one graph: an outer conditional while node (one
// refinement round per run) whose body is the iteration loop (an inner
// conditional while node, the single-level loop's body) followed by the FP64
// true residual of every system, the refinement decisions (k_brefine), the
// restarts and the two loop conditions. One launch runs every round; the
// host reads the systems' state once at the end.
struct SolveGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t body_kernels = 0, round_kernels = 0;
  ~SolveGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (g) cudaGraphDestroy(g);
  }
};

rr_status build_solve_graph(const BatchRun &R, SolveGraph &L) {
  BatchState *B = R.B;
  rr_handle *h = R.h;
  cudaStream_t cs = B->cs;
  const int64_t l0 = rr_launch_counter;
  RR_CUDA(cudaGraphCreate(&L.g, 0));
  cudaGraphConditionalHandle ho, hi;
  RR_CUDA(cudaGraphConditionalHandleCreate(&ho, L.g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams op{};
  op.type = cudaGraphNodeTypeConditional;
  op.conditional.handle = ho;
  op.conditional.type = cudaGraphCondTypeWhile;
  op.conditional.size = 1;
  cudaGraphNode_t onode, inode;
  RR_CUDA(cudaGraphAddNode(&onode, L.g, nullptr, nullptr, 0, &op));
  cudaGraph_t obody = op.conditional.phGraph_out[0];
  RR_CUDA(cudaGraphConditionalHandleCreate(&hi, obody, 1, cudaGraphCondAssignDefault));
  auto fail = [&](rr_status s, cudaError_t ec) -> rr_status {
    cudaGraphDestroy(L.g);
    L.g = nullptr;
    cudaGetLastError();
    rr_launch_counter = l0;
    if (s != RR_OK) return s;
    rr_set_error("batched solve graph capture failed: %s", cudaGetErrorString(ec));
    return RR_CUDA_ERROR;
  };
  // a round starts by setting the loop's condition (the loop runs while a
  // system is active and below the limit, as the host-driven form)
  RR_CUDA(cudaStreamBeginCaptureToGraph(cs, obody, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal));
  k_bloop_condition<<<1, 32, 0, cs>>>(hi, B->g);
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t *deps = nullptr;
  size_t ndeps = 0;
  cudaError_t ec = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
  std::vector<cudaGraphNode_t> first(deps, deps + (ec == cudaSuccess ? ndeps : 0));
  cudaGraph_t cap = nullptr;
  const cudaError_t ec2 = cudaStreamEndCapture(cs, &cap);
  if (ec != cudaSuccess || ec2 != cudaSuccess || first.size() != 1)
    return fail(RR_OK, ec != cudaSuccess ? ec : ec2 != cudaSuccess ? ec2 : cudaErrorUnknown);
  cudaGraphNodeParams ip{};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = hi;
  ip.conditional.type = cudaGraphCondTypeWhile;
  ip.conditional.size = 1;
  RR_CUDA(cudaGraphAddNode(&inode, obody, first.data(), nullptr, 1, &ip));
  // the iteration loop
  RR_CUDA(cudaStreamBeginCaptureToGraph(cs, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal));
  int64_t c0 = rr_launch_counter;
  rr_status s = biteration(R, cs);
  if (s == RR_OK) {
    k_bloop_condition<<<1, 32, 0, cs>>>(hi, B->g);
    ++rr_launch_counter;
  }
  L.body_kernels = rr_launch_counter - c0;
  ec = cudaStreamEndCapture(cs, &cap);
  if (s != RR_OK || ec != cudaSuccess) return fail(s, ec);
  // the end of a round, after the loop
  RR_CUDA(cudaStreamBeginCaptureToGraph(cs, obody, &inode, nullptr, 1,
                                        cudaStreamCaptureModeThreadLocal));
  c0 = rr_launch_counter;
  s = btrue_residual(R, cs);
  if (s == RR_OK) {
    k_brefine_clear<<<1, 256, 0, cs>>>(B->g, B->slab_active, R.n_slabs);
    k_brefine<<<(unsigned)((R.S + 255) / 256), 256, 0, cs>>>(
        R.S, B->col, B->state, B->restarts, h->opt.max_restarts, h->opt.max_iter, B->g, B->flag,
        B->slab_active);
    rr_launch_counter += 2;
    const dim3 vgrid(kBEpiBlocks, (unsigned)R.n_slabs);
    k_brestart<<<vgrid, kThreads, 0, cs>>>(h->F, R.S, R.ld, B->flag, h->col_ptr, B->col, B->rt,
                                           B->r, B->z1, B->V);
    k_bround_condition<<<1, 32, 0, cs>>>(ho, B->g);
    rr_launch_counter += 3;   // with the loop condition set at the start of the round
    if (cudaGetLastError() != cudaSuccess) s = RR_CUDA_ERROR;
  }
  L.round_kernels = rr_launch_counter - c0;
  ec = cudaStreamEndCapture(cs, &cap);
  if (s != RR_OK || ec != cudaSuccess) return fail(s, ec);
  rr_launch_counter = l0;   // recorded, not launched
  RR_CUDA(cudaGraphInstantiate(&L.exec, L.g, 0));
  return RR_OK;
}

// The fastest SpMM variant for this pattern and batch width: every candidate
// (columns per lane x row segments in flight) timed on the operator's two
// FP32 passes over all slabs, once per (N, F, nnz, ld) in the process.
rr_status batch_autotune(const BatchRun &R, cudaStream_t st) {
  static std::mutex mu;
  static std::map<std::array<int64_t, 4>, std::pair<SpmmConfig, double>> cache;
  rr_handle *h = R.h;
  BatchState *B = R.B;
  const std::array<int64_t, 4> key{h->N, h->F, h->nnz, R.ld};
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      B->spmm = it->second.first;
      B->spmm_ms = it->second.second;
      return RR_OK;
    }
  }
  std::vector<SpmmConfig> cands;
  for (int32_t c : {1, 2, 4})
    for (int32_t u : {4, 8})
      if (c < 4 || R.ld % 128 == 0) cands.push_back(SpmmConfig{c, u});
  cudaEvent_t e0, e1;
  RR_CUDA(cudaEventCreate(&e0));
  RR_CUDA(cudaEventCreate(&e1));
  SpmmConfig best = B->spmm;
  float best_ms = 0.f;
  rr_status s = RR_OK;
  for (const SpmmConfig &c : cands) {
    float t = 0.f;
    for (int rep = 0; rep < 3 && s == RR_OK; ++rep) {
      if (cudaEventRecord(e0, st) != cudaSuccess) s = RR_CUDA_ERROR;
      if (s == RR_OK)
        s = launch_bspmm<float>(h->N, h->row_ptr, h->row_ptr + 1, h->col_idx, B->V, R.ld, B->U,
                                R.ld, R.ld, nullptr, st, c);
      if (s == RR_OK)
        s = launch_bspmm<float>(B->n_units2, B->ubeg2, B->uend2, h->row_idx, B->U, R.ld, B->Zp,
                                R.ld, R.ld, nullptr, st, c);
      float ms = 0.f;
      if (s == RR_OK && (cudaEventRecord(e1, st) != cudaSuccess ||
                         cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        s = RR_CUDA_ERROR;
      if (rep == 1 || (rep > 1 && ms < t)) t = ms;   // the first run is a warm-up
    }
    if (s != RR_OK) break;
    if (best_ms == 0.f || t < best_ms) {
      best_ms = t;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  RR_TRY(s);
  B->spmm = best;
  B->spmm_ms = best_ms;
  std::lock_guard<std::mutex> lock(mu);
  cache[key] = {best, (double)best_ms};
  return RR_OK;
}

// Runs batched iterations until every system has stopped or the limit.
rr_status brun(const BatchRun &R, LoopGraph *L, int32_t check_every) {
  BatchState *B = R.B;
  cudaStream_t st = R.h->st;
  if (!L) {
    for (;;) {
      for (int32_t i = 0; i < std::max(1, check_every); ++i) RR_TRY(biteration(R, st));
      RR_CUDA(cudaMemcpyAsync(B->g_host, B->g, sizeof(BatchGlobal), cudaMemcpyDeviceToHost, st));
      RR_CUDA(cudaStreamSynchronize(st));
      if (!B->g_host->any_active || B->g_host->iter >= B->g_host->limit) return RR_OK;
    }
  }
  const int32_t it0 = B->g_host->iter;
  RR_CUDA(cudaGraphLaunch(L->exec, st));
  RR_CUDA(cudaMemcpyAsync(B->g_host, B->g, sizeof(BatchGlobal), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  rr_launch_counter += L->body_kernels * std::max<int64_t>(1, B->g_host->iter - it0);
  return RR_OK;
}

}  // namespace

void batch_free(BatchState *B) {
  if (!B) return;
  if (B->cs) cudaStreamDestroy(B->cs);
  B->mem.free_all();
  if (B->col_host) cudaFreeHost(B->col_host);
  if (B->g_host) cudaFreeHost(B->g_host);
  if (B->slab_host) cudaFreeHost(B->slab_host);
  if (B->flag_host) cudaFreeHost(B->flag_host);
  if (B->state_host) cudaFreeHost(B->state_host);
  if (B->restarts_host) cudaFreeHost(B->restarts_host);
  delete B;
}

}  // namespace rr

extern "C" rr_status rr_solve_batch(rr_handle *h, int32_t nrhs, const double *Y, int32_t nlam,
                                    const double *lambdas, double *W, double tol, rr_info *infos) {
  if (h && h->ready && !h->fork_of && cudaEventSynchronize(h->ready) != cudaSuccess) {
    rr_set_error("%s", cudaGetErrorString(cudaGetLastError()));
    return RR_CUDA_ERROR;
  }
  NvtxRange nvtx_range("rr_solve_batch");
  using namespace rr;
  if (!h || !Y || !W || !lambdas || nrhs < 1 || nlam < 1 || !(tol > 0.0 && tol < 1.0)) {
    rr_set_error("rr_solve_batch: NULL pointer, nrhs or nlam < 1, or tol not in (0, 1)");
    return RR_INVALID_ARG;
  }
  if ((int64_t)nrhs * nlam > (int64_t)1 << 20) {
    rr_set_error("rr_solve_batch: more than 2^20 systems");
    return RR_INVALID_ARG;
  }
  if (h->fork_of) {
    rr_set_error("rr_solve_batch: not supported on a handle from rr_fork_lambda");
    return RR_UNSUPPORTED;
  }
  if (h->dense) {
    rr_set_error("rr_solve_batch: the batched engine takes binary X only");
    return RR_UNSUPPORTED;
  }
  for (int32_t l = 0; l < nlam; ++l)
    if (!(lambdas[l] > 0.0) || !isfinite(lambdas[l])) {
      rr_set_error("rr_solve_batch: every lambda must be positive and finite");
      return RR_INVALID_ARG;
    }
  if (h->opt.solver != RR_SOLVER_TWOLEVEL) {
    rr_set_error("rr_solve_batch: the handle's solver must be RR_SOLVER_TWOLEVEL");
    return RR_UNSUPPORTED;
  }
  cudaStream_t st = h->st;
  struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  RR_CUDA(cudaEventCreate(&ev.a));
  RR_CUDA(cudaEventCreate(&ev.b));
  RR_CUDA(cudaEventRecord(ev.a, st));
  const int64_t launches0 = rr_launch_counter;
  const int32_t S = nrhs * nlam;
  const int64_t ld = round_up64(S);
  RR_TRY(batch_reserve(h, ld, nlam));
  BatchState *B = h->batch;
  const int64_t F = h->F, N = h->N;
  const int32_t n_slabs = (int32_t)(ld / kSlab);
  BatchRun R{h, B, S, nrhs, nlam, n_slabs, ld, tol, nullptr};

  std::vector<double> omega(nlam);
  RR_TRY(batch_factors(h, B, nlam, lambdas, omega.data()));
  // per-system weights
  for (int64_t c = 0; c < ld; ++c) {
    BatchCol C{};
    if (c < S) {
      C.lambda = lambdas[c / nrhs];
      C.omega = omega[c / nrhs];
    }
    C.conv = 1;
    B->col_host[c] = C;
  }
  RR_CUDA(cudaMemcpyAsync(B->col, B->col_host, sizeof(BatchCol) * ld, cudaMemcpyHostToDevice, st));
  // b = X^T y_j through the FP64 pass 2 on the targets (ld_y columns), then the start state
  const int64_t ldy = round_up64(nrhs);
  const dim3 tgrid((unsigned)((N + 31) / 32), (unsigned)(ldy / 32));
  RR_LAUNCH(k_btranspose_in, tgrid, dim3(32, 8), 0, st, N, nrhs, ldy, Y, B->U64);
  RR_TRY(launch_bspmm<double>(B->n_units2, B->ubeg2, B->uend2, h->row_idx, B->U64, ldy, B->Zp64,
                              ldy, ldy, nullptr, st));
  const dim3 vgrid(kBEpiBlocks, (unsigned)n_slabs);
  RR_LAUNCH_PDL(k_bstart, vgrid, kThreads, 0, st, F, S, nrhs, ld, B->uptr2, B->Zp64, ldy, h->col_ptr,
            B->col, B->b, B->w, B->r, B->z1, B->V, B->part);
  BatchGlobal G0{0, h->opt.max_iter, 0, 0};
  *B->g_host = G0;
  RR_CUDA(cudaMemcpyAsync(B->g, B->g_host, sizeof(BatchGlobal), cudaMemcpyHostToDevice, st));
  RR_CUDA(cudaMemsetAsync(B->slab_active, 0, sizeof(int32_t) * n_slabs, st));
  RR_TRY(bfinish(R, BFIN_BNORM, st));

  RR_CUDA(cudaMemcpyAsync(B->g_host, B->g, sizeof(BatchGlobal), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));

  RR_TRY(batch_autotune(R, st));
  std::vector<int32_t> restarts(S, 0), state(S, 0);   // state: 0 running, 1 done, 2 failed
  rr_status result = RR_OK;
  if (h->opt.use_graphs) {
    // every refinement round in one graph launch; the state is read once at the end
    RR_CUDA(cudaMemsetAsync(B->state, 0, sizeof(int32_t) * S, st));
    RR_CUDA(cudaMemsetAsync(B->restarts, 0, sizeof(int32_t) * S, st));
    SolveGraph graph;
    RR_TRY(build_solve_graph(R, graph));
    RR_CUDA(cudaGraphLaunch(graph.exec, st));
    RR_CUDA(cudaMemcpyAsync(B->col_host, B->col, sizeof(BatchCol) * ld, cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaMemcpyAsync(B->g_host, B->g, sizeof(BatchGlobal), cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaMemcpyAsync(B->state_host, B->state, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaMemcpyAsync(B->restarts_host, B->restarts, sizeof(int32_t) * S,
                            cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    rr_launch_counter += 1 + graph.body_kernels * (int64_t)B->g_host->iter +
                         graph.round_kernels * (int64_t)B->g_host->rounds;
    for (int32_t c = 0; c < S; ++c) {
      state[c] = B->state_host[c];
      restarts[c] = B->restarts_host[c];
    }
  } else {
    for (;;) {
      if (B->g_host->any_active) RR_TRY(brun(R, nullptr, h->opt.check_every));
      RR_TRY(btrue_residual(R, st));
      RR_CUDA(cudaMemcpyAsync(B->col_host, B->col, sizeof(BatchCol) * ld, cudaMemcpyDeviceToHost, st));
      RR_CUDA(cudaMemcpyAsync(B->g_host, B->g, sizeof(BatchGlobal), cudaMemcpyDeviceToHost, st));
      RR_CUDA(cudaStreamSynchronize(st));
      bool any = false;
      for (int64_t s = 0; s < n_slabs; ++s) B->slab_host[s] = 0;
      for (int32_t c = 0; c < S; ++c) {
        BatchCol &C = B->col_host[c];
        B->flag_host[c] = 0;
        if (state[c] != 0) continue;
        if (C.nonfinite || !isfinite(C.true_rr)) {
          state[c] = 2;
          continue;
        }
        if (sqrt(C.true_rr) <= C.target) {
          state[c] = 1;
          continue;
        }
        if (B->g_host->iter >= h->opt.max_iter || restarts[c] >= h->opt.max_restarts) {
          state[c] = 2;
          continue;
        }
        // refinement: continue from w on the true residual with a fresh direction
        ++restarts[c];
        C.conv = 0;
        C.first = 1;
        C.rr = C.true_rr;
        B->flag_host[c] = 1;
        B->slab_host[c / kSlab] = 1;
        any = true;
      }
      if (!any) break;
      RR_CUDA(cudaMemcpyAsync(B->col, B->col_host, sizeof(BatchCol) * ld, cudaMemcpyHostToDevice, st));
      RR_CUDA(cudaMemcpyAsync(B->flag, B->flag_host, sizeof(int32_t) * S, cudaMemcpyHostToDevice, st));
      RR_CUDA(cudaMemcpyAsync(B->slab_active, B->slab_host, sizeof(int32_t) * n_slabs,
                              cudaMemcpyHostToDevice, st));
      B->g_host->any_active = 1;
      RR_CUDA(cudaMemcpyAsync(B->g, B->g_host, sizeof(BatchGlobal), cudaMemcpyHostToDevice, st));
      RR_LAUNCH_PDL(k_brestart, vgrid, kThreads, 0, st, F, S, ld, B->flag, h->col_ptr, B->col,
                    B->rt, B->r, B->z1, B->V);
    }
  }
  const dim3 ogrid((unsigned)((F + 31) / 32), (unsigned)((S + 31) / 32));
  RR_LAUNCH(k_btranspose_out, ogrid, dim3(32, 8), 0, st, F, S, ld, B->w, W);
  RR_CUDA(cudaEventRecord(ev.b, st));
  RR_CUDA(cudaEventSynchronize(ev.b));
  float ms = 0.f;
  RR_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
  const int64_t launches = rr_launch_counter - launches0;
  for (int32_t c = 0; c < S; ++c) {
    const BatchCol &C = B->col_host[c];
    if (state[c] == 2) result = C.nonfinite ? RR_NONFINITE : RR_NOT_CONVERGED;
    if (!infos) continue;
    rr_info &I = infos[c];
    memset(&I, 0, sizeof I);
    I.iters = C.iters;
    I.restarts = restarts[c];
    I.k_eff = h->k_eff;
    I.kmeans_iters = h->kmeans_iters;
    I.rel_res = C.bnorm > 0 ? sqrt(C.rr) / C.bnorm : 0.0;
    I.true_rel_res = C.bnorm > 0 ? sqrt(C.true_rr) / C.bnorm : 0.0;
    I.omega = C.omega;
    I.setup_ms = h->setup_ms;
    I.solve_ms = ms;
    I.gram_tensor_cores = h->gram_on_tensor_cores ? 1 : 0;
    I.launches = launches;
  }
  if (result == RR_NOT_CONVERGED) rr_set_error("rr_solve_batch: some systems did not reach tol");
  if (result == RR_NONFINITE) rr_set_error("rr_solve_batch: non-finite values in some systems");
  return result;
}

extern "C" rr_status rr_harvest(rr_handle *h, int32_t nrhs, const double *Y, double lambda,
                                const double *Wref, double tol, int32_t max_iter, float *Xp,
                                float *Tp, int64_t max_pairs, int64_t *n_pairs) {
  if (h && h->fork_of) {
    rr_set_error("rr_harvest: not supported on a handle from rr_fork_lambda");
    return RR_UNSUPPORTED;
  }
  if (h && h->ready && !h->fork_of && cudaEventSynchronize(h->ready) != cudaSuccess) {
    rr_set_error("%s", cudaGetErrorString(cudaGetLastError()));
    return RR_CUDA_ERROR;
  }
  NvtxRange nvtx_range("rr_harvest");
  using namespace rr;
  if (!h || !Y || !Wref || !Xp || !Tp || !n_pairs || nrhs < 1 || max_iter < 1 || max_pairs < 1 ||
      !(lambda > 0.0) || !isfinite(lambda) || !(tol > 0.0 && tol < 1.0)) {
    rr_set_error("rr_harvest: NULL pointer or bad sizes / lambda");
    return RR_INVALID_ARG;
  }
  if (nrhs > (1 << 16) || (int64_t)max_iter * nrhs > ((int64_t)1 << 31)) {
    rr_set_error("rr_harvest: nrhs * max_iter too large");
    return RR_INVALID_ARG;
  }
  if (h->dense) {
    rr_set_error("rr_harvest: binary X only");
    return RR_UNSUPPORTED;
  }
  if (h->opt.solver != RR_SOLVER_TWOLEVEL) {
    rr_set_error("rr_harvest: the handle's solver must be RR_SOLVER_TWOLEVEL");
    return RR_UNSUPPORTED;
  }
  *n_pairs = 0;
  cudaStream_t st = h->st;
  const int32_t S = nrhs;
  const int64_t ld = round_up64(S);
  RR_TRY(batch_reserve(h, ld, 1));
  BatchState *B = h->batch;
  const int64_t F = h->F, N = h->N;
  const int32_t k = h->k_eff;
  const int64_t kpad = round_up64(k);
  const int32_t n_slabs = (int32_t)(ld / kSlab);
  double omega = 0.0;
  RR_TRY(batch_factors(h, B, 1, &lambda, &omega));
  for (int64_t c = 0; c < ld; ++c) {
    BatchCol C{};
    if (c < S) {
      C.lambda = lambda;
      C.omega = omega;
    }
    C.conv = 1;
    B->col_host[c] = C;
  }
  RR_CUDA(cudaMemcpyAsync(B->col, B->col_host, sizeof(BatchCol) * ld, cudaMemcpyHostToDevice, st));

  // work space of the capture (freed on return)
  DevArena tmp;
  struct Guard {
    DevArena &a;
    ~Guard() { a.free_all(); }
  } guard{tmp};
  const int64_t slots = (int64_t)max_iter * S;
  Harvest hv{};
  double *wrefT = nullptr;
  int64_t *pos = nullptr, *scr = nullptr;
  RR_TRY(tmp.alloc(&wrefT, (size_t)F * ld));
  RR_TRY(tmp.alloc(&hv.ipE, (size_t)std::max(1, h->bplan.n_items) * ld));
  RR_TRY(tmp.alloc(&hv.rcE, (size_t)kpad * ld));
  RR_TRY(tmp.alloc(&hv.Xs, (size_t)slots * k));
  RR_TRY(tmp.alloc(&hv.Ts, (size_t)slots * k));
  RR_TRY(tmp.alloc(&hv.valid, (size_t)slots));
  RR_TRY(tmp.alloc(&pos, (size_t)slots + 1));
  RR_TRY(tmp.alloc(&scr, (size_t)scan_scratch_len(slots)));
  RR_CUDA(cudaMemsetAsync(hv.valid, 0, sizeof(int64_t) * slots, st));
  hv.wref = wrefT;
  hv.slots = slots;
  const dim3 tw((unsigned)((F + 31) / 32), (unsigned)(ld / 32));
  RR_LAUNCH(k_btranspose_in, tw, dim3(32, 8), 0, st, F, S, ld, Wref, wrefT);

  BatchRun R{h, B, S, nrhs, 1, n_slabs, ld, tol, &hv};
  const int64_t ldy = round_up64(nrhs);
  const dim3 tgrid((unsigned)((N + 31) / 32), (unsigned)(ldy / 32));
  RR_LAUNCH(k_btranspose_in, tgrid, dim3(32, 8), 0, st, N, nrhs, ldy, Y, B->U64);
  RR_TRY(launch_bspmm<double>(B->n_units2, B->ubeg2, B->uend2, h->row_idx, B->U64, ldy, B->Zp64,
                              ldy, ldy, nullptr, st));
  const dim3 vgrid(kBEpiBlocks, (unsigned)n_slabs);
  RR_LAUNCH_PDL(k_bstart, vgrid, kThreads, 0, st, F, S, nrhs, ld, B->uptr2, B->Zp64, ldy, h->col_ptr,
            B->col, B->b, B->w, B->r, B->z1, B->V, B->part);
  BatchGlobal G0{0, max_iter, 0, 0};
  *B->g_host = G0;
  RR_CUDA(cudaMemcpyAsync(B->g, B->g_host, sizeof(BatchGlobal), cudaMemcpyHostToDevice, st));
  RR_CUDA(cudaMemsetAsync(B->slab_active, 0, sizeof(int32_t) * n_slabs, st));
  RR_TRY(bfinish(R, BFIN_BNORM, st));
  RR_CUDA(cudaMemcpyAsync(B->g_host, B->g, sizeof(BatchGlobal), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  if (B->g_host->any_active) {
    RR_TRY(batch_autotune(R, st));
    LoopGraph graph;
    if (h->opt.use_graphs) RR_TRY(build_loop(R, graph));
    RR_TRY(brun(R, h->opt.use_graphs ? &graph : nullptr, h->opt.check_every));
  }
  RR_TRY(scan_exclusive(hv.valid, pos, slots, scr, st));
  RR_LAUNCH(k_bcompact, grid_for(slots, 1), kThreads, 0, st, slots, k, hv.valid, pos, hv.Xs, hv.Ts,
            Xp, Tp, max_pairs);
  int64_t total = 0;
  RR_CUDA(cudaMemcpyAsync(&total, pos + slots, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  *n_pairs = std::min(total, max_pairs);
  return RR_OK;
}

extern "C" rr_status rr_query_batch(const rr_handle *h, int32_t *slab_width, int32_t *unroll,
                                    double *apply_ms) {
  if (!h) {
    rr_set_error("rr_query_batch: NULL handle");
    return RR_INVALID_ARG;
  }
  if (!h->batch) {
    rr_set_error("rr_query_batch: no batched solve has run on this handle");
    return RR_INVALID_ARG;
  }
  if (slab_width) *slab_width = 32 * h->batch->spmm.C;
  if (unroll) *unroll = h->batch->spmm.unroll;
  if (apply_ms) *apply_ms = h->batch->spmm_ms;
  return RR_OK;
}
