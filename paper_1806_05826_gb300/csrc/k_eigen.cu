// The coarse solve by eigendecomposition, reused across lambda (Section 4:
// the Cholesky factor has to be recomputed for every beta, a decomposition of
// the coarse matrix X_c can be reused). With G_s = X_c^T X_c = D_s G D_s =
// Q diag(mu) Q^T, every coarse inverse is
//
//   A_c(lambda)^{-1} = Q diag(1 / (mu + lambda)) Q^T,
//
// applied in the solve loop as Q (diag(1 / (mu + lambda)) (Q^T r_c)), two
// mat-vecs, so a lambda change only rescales a vector (eig_dvec); the batched
// solve forms Q diag(1 / (mu + lambda)) Q^T once per weight (eig_inverse).
// Either replaces a Cholesky factorisation, its triangular inverse and their
// product.
//
// The eigendecomposition is the parallel cyclic Jacobi method: each sweep is
// n - 1 rounds of n / 2 disjoint plane rotations (the round-robin tournament
// ordering, n = k rounded up to even, a padding index with a zero row when k
// is odd), every pair (p, q) meeting once per sweep. In a round every
// rotation's angle is computed from the matrix before the round (k_jac_angles:
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), tau = (a_qq - a_pp) / (2 a_pq),
// c = 1 / sqrt(1 + t^2), s = t c); the rotations then act on A as
// A <- J^T A J 2 x 2 block by 2 x 2 block (block (m1, m2): the rows of pair m1
// and the columns of pair m2; each block read and written by one thread, the
// upper one mirrored into the lower so A stays exactly symmetric, the diagonal
// blocks by the stable formulas a_pp - t a_pq, a_qq + t a_pq, 0), and on the
// eigenvector rows Vt <- J^T Vt (Vt = Q^T, rows contiguous). Sweeps run until
// the off-diagonal Frobenius norm is at most 1e-15 times A's. Fixed order of
// every operation: identical bits on every run.
#include <math.h>

#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace rr {

namespace {

struct JacPair {
  int32_t p, q;
  double c, s, t;
};

__device__ __forceinline__ int32_t jac_player(int32_t pos, int32_t r, int32_t n) {
  return pos == 0 ? 0 : ((pos - 1 + r) % (n - 1)) + 1;
}

// the round's rotations, from A before the round
__global__ void k_jac_angles(int32_t n, int32_t r, const double *__restrict__ A,
                             JacPair *__restrict__ pairs) {
  for (int32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < n / 2;
       m += gridDim.x * blockDim.x) {
    int32_t p = jac_player(m, r, n), q = jac_player(n - 1 - m, r, n);
    if (p > q) {
      const int32_t x = p;
      p = q;
      q = x;
    }
    const double apq = A[(int64_t)p * n + q];
    double t = 0.0;
    if (apq != 0.0) {
      const double tau = (A[(int64_t)q * n + q] - A[(int64_t)p * n + p]) / (2.0 * apq);
      t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
    }
    const double c = 1.0 / sqrt(1.0 + t * t);
    pairs[m] = JacPair{p, q, c, t * c, t};
  }
}

// A <- J^T A J over the upper 2 x 2 blocks (mirrored), and Vt <- J^T Vt:
// threads [0, nb) take blocks (m1 <= m2), threads [nb, nb + n/2 * n) the
// eigenvector rows (pair m, column i).
__global__ void k_jac_rotate(int32_t n, const JacPair *__restrict__ pairs, double *__restrict__ A,
                             double *__restrict__ Vt) {
  const int64_t h = n / 2;
  const int64_t nb = h * (h + 1) / 2;
  const int64_t total = nb + h * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < nb) {
      // upper block index e -> (m1, m2), m1 <= m2, row by row
      int64_t m1 = (int64_t)((2.0 * h + 1.0 - sqrt((2.0 * h + 1.0) * (2.0 * h + 1.0) - 8.0 * e)) / 2.0);
      while (m1 > 0 && m1 * (2 * h - m1 + 1) / 2 > e) --m1;
      while ((m1 + 1) * (2 * h - m1) / 2 <= e) ++m1;
      const int64_t m2 = m1 + (e - m1 * (2 * h - m1 + 1) / 2);
      const JacPair a = pairs[m1], b = pairs[m2];
      if (m1 == m2) {
        const int64_t pp = (int64_t)a.p * n + a.p, qq = (int64_t)a.q * n + a.q;
        const int64_t pq = (int64_t)a.p * n + a.q, qp = (int64_t)a.q * n + a.p;
        const double apq = A[pq];
        A[pp] = A[pp] - a.t * apq;
        A[qq] = A[qq] + a.t * apq;
        A[pq] = 0.0;
        A[qp] = 0.0;
      } else {
        const double b00 = A[(int64_t)a.p * n + b.p], b01 = A[(int64_t)a.p * n + b.q];
        const double b10 = A[(int64_t)a.q * n + b.p], b11 = A[(int64_t)a.q * n + b.q];
        const double t00 = a.c * b00 - a.s * b10, t01 = a.c * b01 - a.s * b11;
        const double t10 = a.s * b00 + a.c * b10, t11 = a.s * b01 + a.c * b11;
        const double r00 = b.c * t00 - b.s * t01, r01 = b.s * t00 + b.c * t01;
        const double r10 = b.c * t10 - b.s * t11, r11 = b.s * t10 + b.c * t11;
        A[(int64_t)a.p * n + b.p] = r00;
        A[(int64_t)a.p * n + b.q] = r01;
        A[(int64_t)a.q * n + b.p] = r10;
        A[(int64_t)a.q * n + b.q] = r11;
        A[(int64_t)b.p * n + a.p] = r00;
        A[(int64_t)b.q * n + a.p] = r01;
        A[(int64_t)b.p * n + a.q] = r10;
        A[(int64_t)b.q * n + a.q] = r11;
      }
    } else {
      const int64_t f = e - nb;
      const int64_t m = f / n, i = f % n;
      const JacPair a = pairs[m];
      const double vp = Vt[(int64_t)a.p * n + i], vq = Vt[(int64_t)a.q * n + i];
      Vt[(int64_t)a.p * n + i] = a.c * vp - a.s * vq;
      Vt[(int64_t)a.q * n + i] = a.s * vp + a.c * vq;
    }
  }
}

// per-block sums of the off-diagonal squares (fixed order), then one block
// adds them: off^2 into out[0]
__global__ void k_jac_off_parts(int32_t n, const double *__restrict__ A, double *__restrict__ part) {
  __shared__ double sm[kWarps + 1];
  const int64_t nn = (int64_t)n * n;
  double acc = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    if (i != j) acc += A[e] * A[e];
  }
  const double tot = block_sum(acc, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_jac_off_sum(int32_t nparts, const double *__restrict__ part, double *out) {
  __shared__ double sm[kWarps + 1];
  const double tot = sum_partials(part, nparts, sm);
  if (threadIdx.x == 0) out[0] = tot;
}

// A (n x n, zero padding) <- G_s (k x k); Vt <- I
__global__ void k_jac_init(int32_t k, int32_t n, const double *__restrict__ Gs,
                           double *__restrict__ A, double *__restrict__ Vt) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    A[e] = (i < k && j < k) ? Gs[i * k + j] : 0.0;
    Vt[e] = i == j ? 1.0 : 0.0;
  }
}

// mu[e] = A[e][e]; Q (k x k, row i = component i) from Vt's first k rows
__global__ void k_jac_out(int32_t k, int32_t n, const double *__restrict__ A,
                          const double *__restrict__ Vt, double *__restrict__ mu,
                          double *__restrict__ Vk) {
  const int64_t kk = (int64_t)k * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < kk;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / k, i = e % k;
    Vk[e] = Vt[r * n + i];   // eigenvector r, component i
    if (i == 0) mu[r] = A[r * n + r];
  }
}

// Ainv = Vk^T diag(1 / (mu + lambda)) Vk (Vk: eigenvector rows): 64 x 64
// output tiles, K (the eigen index) in steps of 16 through shared memory, 4 x 4
// outputs per thread; lower tiles only, mirrored (Ainv exactly symmetric).
constexpr int kET = 64, kEK = 16;
__global__ void __launch_bounds__(kThreads) k_eig_inverse(int32_t k, const double *__restrict__ mu,
                                                         const double *__restrict__ Vk, double lambda,
                                                         double *__restrict__ Ainv) {
  __shared__ double As[kEK][kET + 2];
  __shared__ double Bs[kEK][kET + 2];
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (tj > ti) return;
  const int i0 = ti * kET, j0 = tj * kET;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int e0 = 0; e0 < k; e0 += kEK) {
    for (int q = threadIdx.x; q < kEK * kET; q += kThreads) {
      const int e = q / kET, c = q % kET;
      const int ee = e0 + e;
      const double d = ee < k ? 1.0 / (mu[ee] + lambda) : 0.0;
      As[e][c] = (ee < k && i0 + c < k) ? Vk[(int64_t)ee * k + i0 + c] * d : 0.0;
      Bs[e][c] = (ee < k && j0 + c < k) ? Vk[(int64_t)ee * k + j0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kEK; ++e) {
      double a[4], b[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        a[x] = As[e][ty * 4 + x];
        b[x] = Bs[e][tx * 4 + x];
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int i = i0 + ty * 4 + x, j = j0 + tx * 4 + y;
      if (i < k && j < k && j <= i) {
        Ainv[(int64_t)i * k + j] = acc[x][y];
        Ainv[(int64_t)j * k + i] = acc[x][y];
      }
    }
}

}  // namespace

// The eigendecomposition of G_s = coarse_operator(G, s, lambda = 0): mu[k]
// and Vk (k x k, row e = eigenvector e). Sweeps (each one graph launch of its
// n - 1 rounds) until off(A) <= 1e-15 ||A||_F or 60 sweeps.
rr_status coarse_eigen(int32_t k, const double *G, const double *s, double *mu, double *Vk,
                       int32_t *sweeps_out, cudaStream_t st) {
  const int32_t n = k + (k & 1);
  const int64_t nn = (int64_t)n * n;
  double *A = nullptr, *Vt = nullptr, *Gs = nullptr, *part = nullptr, *off = nullptr;
  JacPair *pairs = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaStream_t cs = nullptr;
  const int nparts = kSMs * 2;
  rr_status s_ = RR_OK;
  auto run = [&]() -> rr_status {
    RR_CUDA(cudaMalloc(&A, sizeof(double) * nn));
    RR_CUDA(cudaMalloc(&Vt, sizeof(double) * nn));
    RR_CUDA(cudaMalloc(&Gs, sizeof(double) * (size_t)k * k));
    RR_CUDA(cudaMalloc(&part, sizeof(double) * nparts));
    RR_CUDA(cudaMalloc(&off, sizeof(double) * 2));
    RR_CUDA(cudaMalloc(&pairs, sizeof(JacPair) * (n / 2 + 1) * (size_t)(n - 1)));
    RR_TRY(coarse_operator(k, G, s, 0.0, Gs, st));
    RR_LAUNCH(k_jac_init, grid_for(nn, kThreads), kThreads, 0, st, k, n, Gs, A, Vt);
    // ||A||_F^2 - off^2 = sum of the diagonal squares; the norm itself once, directly
    RR_LAUNCH(k_jac_off_parts, nparts, kThreads, 0, st, n, A, part);
    RR_LAUNCH(k_jac_off_sum, 1, kThreads, 0, st, nparts, part, off);
    double off0 = 0.0;
    RR_CUDA(cudaMemcpyAsync(&off0, off, sizeof(double), cudaMemcpyDeviceToHost, st));
    std::vector<double> gs((size_t)k * k);
    RR_CUDA(cudaMemcpyAsync(gs.data(), Gs, sizeof(double) * gs.size(), cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    double norm2 = 0.0;
    for (double v : gs) norm2 += v * v;
    const double target = 1e-15 * sqrt(norm2);
    int32_t sweeps = 0;
    if (n >= 2 && sqrt(off0) > target) {
      // one sweep as a graph: n - 1 rounds of (angles, rotations), then off^2
      RR_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      RR_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      const int64_t h = n / 2;
      const int64_t work = h * (h + 1) / 2 + h * n;
      const int64_t l0 = rr_launch_counter;
      rr_status cs_ = RR_OK;
      for (int32_t r = 0; r < n - 1 && cs_ == RR_OK; ++r) {
        JacPair *pr = pairs + (size_t)r * (n / 2 + 1);
        k_jac_angles<<<(unsigned)((h + 127) / 128), 128, 0, cs>>>(n, r, A, pr);
        k_jac_rotate<<<grid_for(work, kThreads), kThreads, 0, cs>>>(n, pr, A, Vt);
        if (cudaGetLastError() != cudaSuccess) cs_ = RR_CUDA_ERROR;
      }
      k_jac_off_parts<<<nparts, kThreads, 0, cs>>>(n, A, part);
      k_jac_off_sum<<<1, kThreads, 0, cs>>>(nparts, part, off);
      const int64_t per_sweep = 2 * (int64_t)(n - 1) + 2;
      rr_launch_counter = l0;
      cudaGraph_t cap = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(cs, &cap);
      if (cs_ != RR_OK || ec != cudaSuccess) {
        if (cap) cudaGraphDestroy(cap);
        rr_set_error("coarse_eigen: sweep capture failed");
        return RR_CUDA_ERROR;
      }
      g = cap;
      RR_CUDA(cudaGraphInstantiate(&ge, g, 0));
      for (sweeps = 1; sweeps <= 60; ++sweeps) {
        RR_CUDA(cudaGraphLaunch(ge, st));
        rr_launch_counter += per_sweep;
        double o = 0.0;
        RR_CUDA(cudaMemcpyAsync(&o, off, sizeof(double), cudaMemcpyDeviceToHost, st));
        RR_CUDA(cudaStreamSynchronize(st));
        if (!(sqrt(o) > target)) break;   // converged (a NaN also stops)
      }
      if (sweeps > 60) {
        rr_set_error("coarse_eigen: no convergence in 60 sweeps");
        return RR_NOT_CONVERGED;
      }
    }
    RR_LAUNCH(k_jac_out, grid_for((int64_t)k * k, kThreads), kThreads, 0, st, k, n, A, Vt, mu, Vk);
    RR_CUDA(cudaStreamSynchronize(st));
    if (sweeps_out) *sweeps_out = sweeps;
    return RR_OK;
  };
  s_ = run();
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  if (cs) cudaStreamDestroy(cs);
  cudaFree(A);
  cudaFree(Vt);
  cudaFree(Gs);
  cudaFree(part);
  cudaFree(off);
  cudaFree(pairs);
  return s_;
}

namespace {
__global__ void k_eig_transpose(int32_t k, const double *__restrict__ Vk, double *__restrict__ Qt) {
  const int64_t kk = (int64_t)k * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < kk;
       e += (int64_t)gridDim.x * blockDim.x)
    Qt[e] = Vk[(e % k) * k + e / k];
}
__global__ void k_eig_dvec(int32_t k, const double *__restrict__ mu, double lambda,
                           double *__restrict__ d) {
  for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < k; e += gridDim.x * blockDim.x)
    d[e] = 1.0 / (mu[e] + lambda);
}
}  // namespace

rr_status eig_transpose(int32_t k, const double *Vk, double *Qt, cudaStream_t st) {
  RR_LAUNCH(k_eig_transpose, grid_for((int64_t)k * k, kThreads), kThreads, 0, st, k, Vk, Qt);
  return RR_OK;
}

rr_status eig_dvec(int32_t k, const double *mu, double lambda, double *d, cudaStream_t st) {
  RR_LAUNCH(k_eig_dvec, grid_for(k, kThreads), kThreads, 0, st, k, mu, lambda, d);
  return RR_OK;
}

rr_status eig_inverse(int32_t k, const double *mu, const double *Vk, double lambda, double *Ainv,
                      cudaStream_t st) {
  const unsigned t = (unsigned)((k + kET - 1) / kET);
  RR_LAUNCH(k_eig_inverse, dim3(t, t), kThreads, 0, st, k, mu, Vk, lambda, Ainv);
  return RR_OK;
}

}  // namespace rr
