// C ABI of the two-level preconditioned CG solver (include/rr.h): handle
// life cycle, setup orchestration and the solve loop. All arithmetic runs in
// the kernels of this directory; this file only sequences them on the
// handle's stream and moves status words to the host.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "handle.h"
#include "kernels.h"

static thread_local char g_err[1024] = "";
thread_local int64_t rr_launch_counter = 0;

void rr_set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

namespace {

using rr::kThreads;

// d_i = ||x_i||^2 + lambda (column nnz for binary X); ratio_i = (sum_j |A_ij|) / d_i
// with sum_j |(X^T X)_ij| = gsum_i (an exact integer). The maximum ratio is
// kept through the order-preserving bit pattern of positive doubles.
__global__ void k_jacobi_setup(int64_t F, double lambda, const int64_t *__restrict__ col_ptr,
                               const int64_t *__restrict__ gsum, double *__restrict__ d,
                               unsigned long long *__restrict__ max_bits) {
  unsigned long long best = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double di = (double)(col_ptr[i + 1] - col_ptr[i]) + lambda;
    d[i] = di;
    const double ratio = ((double)gsum[i] + lambda) / di;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(ratio);
    best = bits > best ? bits : best;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, best, o);
    best = t > best ? t : best;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(max_bits, best);
}

// n_S[S] = number of features labelled S (counts: the order of the atomics does not matter).
__global__ void k_dense_sizes(int64_t F, const int32_t *__restrict__ labels, int64_t *n_S, int32_t k) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t l = labels[i];
    if (l >= 0 && l < k) atomicAdd((unsigned long long *)&n_S[l], 1ull);
  }
}

__global__ void k_omega(const unsigned long long *max_bits, double *omega_out) {
  if (threadIdx.x == 0) *omega_out = 1.0 / __longlong_as_double((long long)*max_bits);
}

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

}  // namespace


namespace {

rr_status check_dev_error(rr_handle *h, const char *where) {
  RR_CUDA(cudaMemcpyAsync(h->err_host, h->err, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st));
  RR_CUDA(cudaStreamSynchronize(h->st));
  const int32_t e = *h->err_host;
  if (e == rr::DEV_OK) return RR_OK;
  RR_CUDA(cudaMemsetAsync(h->err, 0, sizeof(int32_t), h->st));
  switch (e) {
    case rr::DEV_BAD_INDEX:
      rr_set_error("%s: CSR indices not strictly increasing or out of range", where);
      return RR_INVALID_ARG;
    case rr::DEV_NOT_SPD:
      rr_set_error("%s: coarse Cholesky met a pivot <= 0", where);
      return RR_NOT_SPD;
    case rr::DEV_COUNT_OVERFLOW:
      rr_set_error("%s: a row holds more than 2048 features of one cluster", where);
      return RR_UNSUPPORTED;
    case rr::DEV_TIMEOUT:
      rr_set_error("%s: a bounded device wait expired", where);
      return RR_TIMEOUT;
    default:
      rr_set_error("%s: device error %d", where, e);
      return RR_CUDA_ERROR;
  }
}

// Coarse operator, its factor and inverse, Jacobi diagonal and damping at lambda.
// The eigendecomposition of the lambda-free coarse operator (RR_COARSE_EIGEN),
// once per clustering.
rr_status coarse_eigen_setup(rr_handle *h) {
  if (h->opt.coarse != RR_COARSE_EIGEN) return RR_OK;
  const int32_t k = h->k_eff;
  RR_TRY(h->mem.alloc(&h->mu, k));
  RR_TRY(h->mem.alloc(&h->Qv, (int64_t)k * k));
  RR_TRY(h->mem.alloc(&h->Qt, (int64_t)k * k));
  RR_TRY(h->mem.alloc(&h->dvec, k));
  RR_TRY(h->mem.alloc(&h->ec_tmp, k));
  RR_TRY(rr::coarse_eigen(k, h->G, h->s, h->mu, h->Qv, &h->eig_sweeps, h->st));
  return rr::eig_transpose(k, h->Qv, h->Qt, h->st);
}

// e_c = A_c^-1 P^T r1 (restriction item sums already in the plan): the
// explicit inverse, or the eigendecomposition's two mat-vecs.
rr_status coarse_step(rr_handle *h, const int32_t *stop, cudaStream_t st, bool fp32) {
  if (fp32 && h->Ainv32 && !h->mu)   // the FP32 inner iterations' coarse step
    return rr::coarse_matvec32(h->k_eff, h->Ainv32, h->rplan, h->s, h->ec, stop, st);
  if (h->mu)
    return rr::coarse_matvec_eigen(h->k_eff, h->Qv, h->Qt, h->dvec, h->rplan, h->s, h->ec_tmp,
                                   h->ec, stop, st);
  return rr::coarse_matvec(h->k_eff, h->Ainv, h->rplan, h->s, nullptr, h->ec, stop, st);
}

rr_status build_lambda(rr_handle *h, double lambda) {
  cudaStream_t st = h->st;
  const int32_t k = h->k_eff;
  RR_TRY(rr::coarse_operator(k, h->G, h->s, lambda, h->Ac, st));
  if (h->mu) {   // A_c^-1 = Q diag(1 / (mu + lambda)) Q^T, applied as two mat-vecs
    RR_TRY(rr::eig_dvec(k, h->mu, lambda, h->dvec, st));
  } else {
    RR_CUDA(cudaMemcpyAsync(h->Lw, h->Ac, sizeof(double) * (size_t)k * k, cudaMemcpyDeviceToDevice, st));
    RR_TRY(rr::cholesky(k, h->Lw, h->Linv, h->err, st));
    RR_TRY(rr::chol_inverse(k, h->Lw, h->Linv, h->Ainv, st));
    if (h->Ainv32) RR_TRY(rr::coarse_to_f32(k, h->Ainv, h->Ainv32, st));
  }
  RR_CUDA(cudaMemsetAsync(h->max_bits, 0, sizeof(unsigned long long), st));
  if (h->dense) {
    RR_TRY(rr::dense_jacobi(h->F, lambda, h->dsq, h->dgs, h->d, h->max_bits, st));
  } else {
    RR_LAUNCH(k_jacobi_setup, rr::grid_for(h->F, kThreads), kThreads, 0, st, h->F, lambda,
              h->col_ptr, h->gsum, h->d, h->max_bits);
  }
  RR_LAUNCH(k_omega, 1, 32, 0, st, h->max_bits, h->omega_dev);
  double om = 0.0;
  RR_CUDA(cudaMemcpyAsync(&om, h->omega_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  RR_TRY(check_dev_error(h, "coarse factor"));
  h->omega = om;
  h->lambda = lambda;
  RR_TRY(rr::split_set_wd(h->split, h->omega, h->d, st));
  return RR_OK;
}

// The smoother at lambda (d, omega read back, and omega/d of the split form);
// the coarse level is left to start_coarse_factor.
rr_status build_smoother(rr_handle *h, double lambda) {
  cudaStream_t st = h->st;
  RR_CUDA(cudaMemsetAsync(h->max_bits, 0, sizeof(unsigned long long), st));
  RR_LAUNCH(k_jacobi_setup, rr::grid_for(h->F, kThreads), kThreads, 0, st, h->F, lambda,
            h->col_ptr, h->gsum, h->d, h->max_bits);
  RR_LAUNCH(k_omega, 1, 32, 0, st, h->max_bits, h->omega_dev);
  double om = 0.0;
  RR_CUDA(cudaMemcpyAsync(&om, h->omega_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  h->omega = om;
  h->lambda = lambda;
  return RR_OK;
}

// The coarse operator, factor and inverse at lambda (the same operations as
// build_lambda), left running on the handle's factor stream behind h->ready.
// Every later call that uses the coarse level waits for it (wait_coarse); a
// non-positive pivot is reported by the first of them that checks the error
// word (a solve).
rr_status start_coarse_factor(rr_handle *h, double lambda) {
  RR_CUDA(cudaStreamCreateWithFlags(&h->fst, cudaStreamNonBlocking));
  RR_CUDA(cudaEventCreateWithFlags(&h->ready, cudaEventDisableTiming));
  cudaStream_t st = h->fst;
  const int32_t k = h->k_eff;
  RR_TRY(rr::coarse_operator(k, h->G, h->s, lambda, h->Ac, st));
  if (h->mu) {
    RR_TRY(rr::eig_dvec(k, h->mu, lambda, h->dvec, st));
  } else {
    RR_CUDA(cudaMemcpyAsync(h->Lw, h->Ac, sizeof(double) * (size_t)k * k, cudaMemcpyDeviceToDevice, st));
    RR_TRY(rr::cholesky(k, h->Lw, h->Linv, h->err, st));
    RR_TRY(rr::chol_inverse(k, h->Lw, h->Linv, h->Ainv, st));
    if (h->Ainv32) RR_TRY(rr::coarse_to_f32(k, h->Ainv, h->Ainv32, st));
  }
  RR_CUDA(cudaEventRecord(h->ready, st));
  return RR_OK;
}

// Orders st after the coarse factor rr_setup left running (no host wait).
rr_status wait_coarse(const rr_handle *h, cudaStream_t st) {
  if (h->ready && !h->fork_of) RR_CUDA(cudaStreamWaitEvent(st, h->ready, 0));
  return RR_OK;
}

// The same, on the host: before a call rebuilds or swaps the coarse buffers.
rr_status wait_coarse_host(const rr_handle *h) {
  if (h->ready && !h->fork_of) RR_CUDA(cudaEventSynchronize(h->ready));
  return RR_OK;
}

// The coarse inverse and the smoother at lambda into a prepared slot, on the
// prepare stream (the Cholesky form; the same operations as build_lambda).
rr_status prepare_one(rr_handle *h, rr_handle::Prepared &P, double lambda) {
  cudaStream_t st = h->prep_st;
  const int32_t k = h->k_eff;
  const int64_t kk = (int64_t)k * k;
  DevArena &m = h->mem;
  if (!P.Ainv) {
    RR_TRY(m.alloc(&P.Ainv, kk));
    if (h->Ainv32) RR_TRY(m.alloc(&P.Ainv32, (int64_t)k * ((k + 3) & ~3)));
    RR_TRY(m.alloc(&P.d, h->F));
    RR_TRY(m.alloc(&P.omega_dev, 1));
    RR_TRY(m.alloc(&P.max_bits, 1));
    RR_CUDA(cudaEventCreateWithFlags(&P.done, cudaEventDisableTiming));
  }
  P.valid = false;
  RR_TRY(rr::coarse_operator(k, h->G, h->s, lambda, h->prep_Ac, st));
  RR_CUDA(cudaMemcpyAsync(h->prep_Lw, h->prep_Ac, sizeof(double) * kk, cudaMemcpyDeviceToDevice, st));
  RR_TRY(rr::cholesky(k, h->prep_Lw, h->prep_Linv, h->err, st));
  RR_TRY(rr::chol_inverse(k, h->prep_Lw, h->prep_Linv, P.Ainv, st));
  if (P.Ainv32) RR_TRY(rr::coarse_to_f32(k, P.Ainv, P.Ainv32, st));
  RR_CUDA(cudaMemsetAsync(P.max_bits, 0, sizeof(unsigned long long), st));
  if (h->dense) {
    RR_TRY(rr::dense_jacobi(h->F, lambda, h->dsq, h->dgs, P.d, P.max_bits, st));
  } else {
    RR_LAUNCH(k_jacobi_setup, rr::grid_for(h->F, kThreads), kThreads, 0, st, h->F, lambda,
              h->col_ptr, h->gsum, P.d, P.max_bits);
  }
  RR_LAUNCH(k_omega, 1, 32, 0, st, P.max_bits, P.omega_dev);
  RR_CUDA(cudaEventRecord(P.done, st));
  P.lambda = lambda;
  P.valid = true;
  return RR_OK;
}

// rr_set_lambda's fast path: a prepared slot for exactly this lambda is swapped
// in (its buffers and the handle's trade places); returns false if none.
rr_status install_prepared(rr_handle *h, double lambda, bool *found) {
  *found = false;
  for (auto &P : h->prep) {
    if (!P.valid || P.lambda != lambda) continue;
    RR_CUDA(cudaEventSynchronize(P.done));
    RR_TRY(check_dev_error(h, "prepared coarse factor"));
    double om = 0.0;
    RR_CUDA(cudaMemcpyAsync(&om, P.omega_dev, sizeof(double), cudaMemcpyDeviceToHost, h->prep_st));
    RR_CUDA(cudaStreamSynchronize(h->prep_st));
    std::swap(h->Ainv, P.Ainv);
    std::swap(h->Ainv32, P.Ainv32);
    std::swap(h->d, P.d);
    std::swap(h->omega_dev, P.omega_dev);
    std::swap(h->max_bits, P.max_bits);
    P.valid = false;
    RR_TRY(rr::coarse_operator(h->k_eff, h->G, h->s, lambda, h->Ac, h->st));
    h->omega = om;
    h->lambda = lambda;
    RR_TRY(rr::split_set_wd(h->split, h->omega, h->d, h->st));
    *found = true;
    return RR_OK;
  }
  return RR_OK;
}

// Solve vectors, partial-dot buffers, scalars and the capture stream.
rr_status alloc_solve_workspace(rr_handle *h) {
  DevArena &m = h->mem;
  const int64_t N = h->N, F = h->F;
  const int32_t k_eff = h->k_eff;
  h->n_parts = rr::kVecGrid;
  for (double **v : {&h->b, &h->r, &h->z1, &h->z2, &h->z, &h->p, &h->q, &h->r1, &h->rt, &h->w_int})
    RR_TRY(m.alloc(v, F));
  RR_TRY(m.alloc(&h->u, std::max<int64_t>(N, 1)));
  RR_TRY(m.alloc(&h->rc, k_eff));
  RR_TRY(m.alloc(&h->ec, k_eff));
  for (double **v : {&h->part_rz, &h->part_pq, &h->part_rr, &h->part_bb})
    RR_TRY(m.alloc(v, h->n_parts));
  RR_TRY(m.alloc(&h->scal, 4));
  RR_TRY(m.alloc(&h->S, 1));
  RR_CUDA(cudaMemsetAsync(h->S, 0, sizeof(rr::PcgScalars), h->st));
  RR_CUDA(cudaMallocHost(&h->S_host, sizeof(rr::PcgScalars)));
  RR_CUDA(cudaMallocHost(&h->scal_host, 4 * sizeof(double)));
  RR_CUDA(cudaMallocHost(&h->limit_host, sizeof(int32_t)));
  RR_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  h->hist_cap = h->opt.max_iter;
  RR_TRY(m.alloc(&h->history, h->hist_cap));
  return RR_OK;
}

// Setup for dense X: k-means++ and Lloyd in FP64 (k_dense.cu), member lists,
// the coarse Gram of X onehot, the smoother's statistics, the factor.
rr_status setup_impl_dense(rr_handle *h, const rr_matrix *X, double lambda, int32_t k) {
  cudaStream_t st = h->st;
  DevArena &m = h->mem;
  auto t_last = std::chrono::steady_clock::now();
  static const char *const kPhaseNames[8] = {
      "rr_setup: copy and validate", "rr_setup: CSC build", "rr_setup: clustering (seeding)",
      "rr_setup: clustering (Lloyd)", "rr_setup: clusters", "rr_setup: coarse Gram",
      "rr_setup: coarse factor", "rr_setup: patterns and workspace"};
  NvtxPhases ranges;
  ranges.next(kPhaseNames[0]);
  auto phase = [&](int i) -> rr_status {
    RR_CUDA(cudaStreamSynchronize(st));
    const auto now = std::chrono::steady_clock::now();
    h->phase_ms[i] += std::chrono::duration<double, std::milli>(now - t_last).count();
    t_last = now;
    if (i + 1 < 8) ranges.next(kPhaseNames[i + 1]);
    return RR_OK;
  };
  const int64_t N = X->n_rows, F = X->n_cols;
  if (N * F >= (1LL << 34) || F > 25600 || N > 65535LL * 64) {
    rr_set_error("rr_setup: dense X needs N*F < 2^34, F <= 25600 and N <= 4194240");
    return RR_UNSUPPORTED;
  }
  h->dense = true;
  h->N = N;
  h->F = F;
  h->nnz = N * F;
  h->k_req = k;
  RR_TRY(m.alloc(&h->err, 1));
  RR_CUDA(cudaMallocHost(&h->err_host, sizeof(int32_t)));
  RR_CUDA(cudaMemsetAsync(h->err, 0, sizeof(int32_t), st));
  RR_TRY(m.alloc(&h->Xd, N * F));
  RR_CUDA(cudaMemcpyAsync(h->Xd, X->values, sizeof(float) * (size_t)(N * F),
                          X->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  RR_TRY(phase(0));
  RR_TRY(phase(1));
  // ---- k-means++ and Lloyd (FP64, blocked row sums)
  const int64_t nb = (N + 63) / 64;
  RR_TRY(m.alloc(&h->centers, k));
  RR_TRY(m.alloc(&h->labels, F));
  RR_TRY(m.alloc(&h->n_S, 2 * (int64_t)k));
  if (h->opt.init_centers) {
    std::vector<char> seen(F, 0);
    for (int32_t s = 0; s < k; ++s) {
      const int32_t c = h->opt.init_centers[s];
      if (c < 0 || c >= F || seen[c]) {
        rr_set_error("init_centers[%d] = %d is out of range or repeated", s, c);
        return RR_INVALID_ARG;
      }
      seen[c] = 1;
    }
    RR_CUDA(cudaMemcpyAsync(h->centers, h->opt.init_centers, sizeof(int32_t) * k,
                            cudaMemcpyHostToDevice, st));
  } else {
    double *d2 = nullptr, *part = nullptr;
    uint8_t *chosen = nullptr;
    RR_TRY(m.alloc(&d2, F));
    RR_TRY(m.alloc(&chosen, F));
    RR_TRY(m.alloc(&part, nb * F));
    RR_TRY(rr::dense_kmeanspp(N, F, h->Xd, k, h->opt.seed, h->centers, d2, chosen, part, h->err, st));
    RR_TRY(check_dev_error(h, "k-means++"));
    m.release(d2);
    m.release(chosen);
    m.release(part);
  }
  RR_TRY(phase(2));
  rr::DenseKmeansScratch w{};
  RR_TRY(m.alloc(&w.key, F));
  RR_TRY(m.alloc(&w.iota, F + 1));
  RR_TRY(m.alloc(&w.cl_ptr, k + 2));
  RR_TRY(m.alloc(&w.members, F));
  RR_TRY(m.alloc(&w.counts, k + 2));
  RR_TRY(m.alloc(&w.cursor, k + 2));
  RR_TRY(m.alloc(&w.tmp, F));
  RR_TRY(m.alloc(&w.scan_scratch, rr::scan_scratch_len(k + 2) + 8));
  RR_TRY(m.alloc(&w.mu, (int64_t)k * N));
  RR_TRY(m.alloc(&w.part, (int64_t)k * nb));
  RR_TRY(m.alloc(&w.mm, k));
  RR_TRY(m.alloc(&w.dot, (int64_t)k * F));
  RR_TRY(m.alloc(&w.dpart, rr::dense_dot_part_len(N, F)));
  RR_TRY(m.alloc(&w.changes, 1));
  RR_TRY(rr::iota_i64(w.iota, F + 1, st));
  int32_t iters = 0;
  RR_TRY(rr::dense_lloyd(N, F, h->Xd, k, h->centers, h->opt.kmeans_max_iter, h->labels, w, &iters, st));
  h->kmeans_iters = iters;
  // cluster sizes of the final labels
  RR_CUDA(cudaMemsetAsync(h->n_S, 0, sizeof(int64_t) * 2 * (size_t)k, st));
  RR_LAUNCH(k_dense_sizes, rr::grid_for(F, kThreads), kThreads, 0, st, F, h->labels, h->n_S, k);
  m.release(w.mu);
  m.release(w.part);
  m.release(w.dot);
  m.release(w.dpart);
  RR_TRY(phase(3));
  // ---- compaction, member lists, prolongation scale
  int32_t *remap = nullptr;
  RR_TRY(m.alloc(&remap, k + 1));
  int32_t k_eff = 0;
  RR_TRY(rr::compact_clusters(F, k, h->labels, h->n_S, remap, &k_eff, st));
  h->k_eff = k_eff;
  RR_TRY(m.alloc(&h->cl_ptr, k_eff + 1));
  RR_TRY(m.alloc(&h->members, F));
  const int64_t big = std::max<int64_t>(F, k_eff) + 1;
  int64_t *scratch64 = nullptr;
  RR_TRY(m.alloc(&scratch64, 2 * big + rr::scan_scratch_len(big) + 256));
  RR_TRY(rr::transpose_pattern(F, k_eff, F, w.iota, h->labels, h->cl_ptr, h->members, scratch64,
                               scratch64 + big, w.tmp, scratch64 + 2 * big, st));
  RR_TRY(m.alloc(&h->s, k_eff));
  RR_TRY(rr::prolong_scale(k_eff, h->n_S, h->s, st));
  RR_TRY(rr::restrict_plan(k_eff, h->cl_ptr, h->rplan, scratch64, st));
  RR_TRY(rr::restrict_plan(k_eff, h->cl_ptr, h->bplan, scratch64, st, rr::kRestrictItemBatch));
  RR_TRY(phase(4));
  // ---- coarse Gram G = (X onehot)^T (X onehot) (FP64), smoother statistics
  double *C = nullptr, *rowabs = nullptr;
  RR_TRY(m.alloc(&C, (int64_t)k_eff * N));
  RR_TRY(m.alloc(&h->G, (int64_t)k_eff * k_eff));
  RR_TRY(rr::dense_coarse_gram(N, F, h->Xd, k_eff, h->cl_ptr, h->members, C, h->G, st));
  RR_TRY(m.alloc(&rowabs, N));
  RR_TRY(m.alloc(&h->dsq, F));
  RR_TRY(m.alloc(&h->dgs, F));
  double *cs_part = nullptr;
  RR_TRY(m.alloc(&cs_part, 2 * rr::dense_col_blocks(N) * F));
  RR_TRY(rr::dense_colstats(N, F, h->Xd, rowabs, cs_part, h->dsq, h->dgs, st));
  RR_TRY(phase(5));
  const int64_t kk = (int64_t)k_eff * k_eff;
  RR_TRY(m.alloc(&h->Ac, kk));
  RR_TRY(m.alloc(&h->Lw, kk));
  RR_TRY(m.alloc(&h->Linv, kk));
  RR_TRY(m.alloc(&h->Ainv, kk));
  RR_TRY(m.alloc(&h->d, F));
  RR_TRY(m.alloc(&h->omega_dev, 1));
  RR_TRY(m.alloc(&h->max_bits, 1));
  RR_TRY(coarse_eigen_setup(h));
  if (h->opt.precision == RR_PREC_MIXED && !h->mu)
    RR_TRY(m.alloc(&h->Ainv32, (int64_t)k_eff * ((k_eff + 3) & ~3)));
  RR_TRY(build_lambda(h, lambda));
  RR_TRY(phase(6));
  RR_TRY(m.alloc(&h->dpart, rr::dense_part_rows(N, F) * F));
  RR_TRY(alloc_solve_workspace(h));
  for (void *p : {(void *)C, (void *)rowabs, (void *)cs_part, (void *)scratch64, (void *)remap, (void *)w.key,
                  (void *)w.iota, (void *)w.cl_ptr, (void *)w.members, (void *)w.counts,
                  (void *)w.cursor, (void *)w.tmp, (void *)w.scan_scratch, (void *)w.mm,
                  (void *)w.changes})
    m.release(p);
  RR_TRY(phase(7));
  return RR_OK;
}

// The sliced patterns of X and X^T and, in mixed precision, the split form:
// they depend on X alone, so rr_setup builds them on a second stream from a
// second host thread while the clustering, the coarse Gram and the factor run
// on the first.
rr_status build_patterns(rr_handle *h, cudaStream_t st) {
  const int64_t N = h->N, F = h->F;
  RR_TRY(rr::sliced_build(N, F, h->row_ptr, h->col_idx, h->pcsr, h->err, st));
  RR_TRY(rr::sliced_build(F, N, h->col_ptr, h->row_idx, h->pcsc, h->err, st));
  if (h->opt.precision == RR_PREC_MIXED)
    RR_TRY(rr::split_build(N, F, h->row_ptr, h->col_idx, h->col_ptr, h->row_idx,
                           h->opt.split_head, h->opt.gather, h->split, h->err, st));
  RR_CUDA(cudaStreamSynchronize(st));
  return RR_OK;
}

struct PatternJob {
  cudaStream_t st = nullptr;
  cudaEvent_t ready = nullptr;
  std::thread worker;
  rr_status status = RR_OK;
  std::string err;
  int64_t launches = 0;
  // waits for the worker and adds its launches to this thread's count
  rr_status finish() {
    if (worker.joinable()) {
      worker.join();
      rr_launch_counter += launches;
      launches = 0;
    }
    if (status != RR_OK) rr_set_error("%s", err.c_str());
    return status;
  }
  ~PatternJob() {
    if (worker.joinable()) worker.join();
    if (ready) cudaEventDestroy(ready);
    if (st) cudaStreamDestroy(st);
  }
  rr_status start(rr_handle *h, cudaStream_t main) {
    int least = 0, greatest = 0;
    RR_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    RR_CUDA(cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, least));
    RR_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    RR_CUDA(cudaEventRecord(ready, main));
    RR_CUDA(cudaStreamWaitEvent(st, ready, 0));
    worker = std::thread([this, h] {
      const int64_t l0 = rr_launch_counter;
      status = build_patterns(h, st);
      if (status != RR_OK) err = rr_last_error();
      launches = rr_launch_counter - l0;
    });
    return RR_OK;
  }
};

rr_status setup_impl(rr_handle *h, const rr_matrix *X, double lambda, int32_t k) {
  cudaStream_t st = h->st;
  DevArena &m = h->mem;
  auto t_last = std::chrono::steady_clock::now();
  // wall time of a finished phase (the stream is drained so device work counts)
  static const char *const kPhaseNames[8] = {
      "rr_setup: copy and validate", "rr_setup: CSC build", "rr_setup: clustering (seeding)",
      "rr_setup: clustering (Lloyd)", "rr_setup: clusters", "rr_setup: coarse Gram",
      "rr_setup: coarse factor", "rr_setup: patterns and workspace"};
  NvtxPhases ranges;
  ranges.next(kPhaseNames[0]);
  auto phase = [&](int i) -> rr_status {
    RR_CUDA(cudaStreamSynchronize(st));
    const auto now = std::chrono::steady_clock::now();
    h->phase_ms[i] += std::chrono::duration<double, std::milli>(now - t_last).count();
    t_last = now;
    if (i + 1 < 8) ranges.next(kPhaseNames[i + 1]);
    return RR_OK;
  };
  const int64_t N = X->n_rows, F = X->n_cols, nnz = X->nnz;
  h->N = N;
  h->F = F;
  h->nnz = nnz;
  h->k_req = k;
  RR_TRY(m.alloc(&h->err, 1));
  RR_CUDA(cudaMallocHost(&h->err_host, sizeof(int32_t)));
  RR_CUDA(cudaMemsetAsync(h->err, 0, sizeof(int32_t), st));

  // ---- X on the device
  RR_TRY(m.alloc(&h->row_ptr, N + 1));
  RR_TRY(m.alloc(&h->col_idx, nnz));
  if (X->on_device) {
    int64_t ends[2];
    RR_CUDA(cudaMemcpyAsync(&ends[0], X->row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaMemcpyAsync(&ends[1], X->row_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    if (ends[0] != 0 || ends[1] != nnz) {
      rr_set_error("row_ptr[0] must be 0 and row_ptr[N] must equal nnz");
      return RR_INVALID_ARG;
    }
    RR_CUDA(cudaMemcpyAsync(h->row_ptr, X->row_ptr, sizeof(int64_t) * (N + 1), cudaMemcpyDeviceToDevice, st));
    RR_CUDA(cudaMemcpyAsync(h->col_idx, X->col_idx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, st));
    RR_TRY(rr::validate_csr(N, F, nnz, h->row_ptr, h->col_idx, h->err, st));
    RR_TRY(check_dev_error(h, "rr_setup"));
  } else {
    // the ends on the host; the rest on the device after the copy (a pass over
    // nnz indices on one host core would cost more than the copy itself)
    if (X->row_ptr[0] != 0 || X->row_ptr[N] != nnz) {
      rr_set_error("row_ptr[0] must be 0 and row_ptr[N] must equal nnz");
      return RR_INVALID_ARG;
    }
    RR_CUDA(cudaMemcpyAsync(h->row_ptr, X->row_ptr, sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, st));
    RR_CUDA(cudaMemcpyAsync(h->col_idx, X->col_idx, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st));
    RR_TRY(rr::validate_csr(N, F, nnz, h->row_ptr, h->col_idx, h->err, st));
    RR_TRY(check_dev_error(h, "rr_setup"));
  }

  RR_TRY(phase(0));
  // ---- transposed copy (CSC), rows ascending within columns
  const int64_t big = std::max(N, F) + 1;
  int64_t *scratch64 = nullptr;
  const int64_t scan_len = rr::scan_scratch_len(big) + 8;
  RR_TRY(m.alloc(&scratch64, 2 * big + scan_len + 256));
  int32_t *tmp32 = nullptr;
  RR_TRY(m.alloc(&tmp32, std::max(nnz, F)));
  RR_TRY(m.alloc(&h->col_ptr, F + 1));
  RR_TRY(m.alloc(&h->row_idx, nnz));
  RR_TRY(rr::transpose_pattern(N, F, nnz, h->row_ptr, h->col_idx, h->col_ptr, h->row_idx,
                               scratch64, scratch64 + big, tmp32, scratch64 + 2 * big, st));

  RR_TRY(phase(1));
  PatternJob patterns;
  RR_TRY(patterns.start(h, st));
  rr::KmeansBuffers kb{};
  if (h->opt.clustering == RR_CLUSTER_LEADER) {
    // ---- leader-follower clustering (Section 3.4, Algorithm 1)
    rr::LfBuffers lb{};
    RR_TRY(m.alloc(&lb.rl, std::max<int64_t>(nnz, 1)));
    RR_TRY(m.alloc(&lb.rl_cnt, N));
    RR_TRY(m.alloc(&lb.rowmask, N));
    RR_TRY(m.alloc(&lb.nlead, k));
    RR_TRY(m.alloc(&lb.best, 64));
    RR_TRY(m.alloc(&lb.S, 1));
    RR_TRY(m.alloc(&h->centers, k));
    RR_TRY(m.alloc(&h->labels, F));
    RR_TRY(m.alloc(&h->n_S, 2 * (int64_t)k));
    RR_CUDA(cudaMemsetAsync(h->centers, 0xff, sizeof(int32_t) * k, st));
    int32_t n_lead = 0;
    RR_TRY(rr::leader_follower(N, F, h->row_ptr, h->col_ptr, h->row_idx, h->opt.lf_tol2, k, lb,
                               h->labels, h->centers, &n_lead, h->err, st));
    RR_TRY(check_dev_error(h, "rr_setup (leader-follower)"));
    h->kmeans_iters = 0;
    RR_TRY(m.alloc(&h->gsum, F));
    RR_TRY(rr::feature_work(F, h->row_ptr, h->col_ptr, h->row_idx, h->gsum, st));
    m.release(lb.rl);
    m.release(lb.rl_cnt);
    m.release(lb.rowmask);
    m.release(lb.nlead);
    m.release(lb.best);
    m.release(lb.S);
    RR_TRY(phase(2));
    RR_TRY(phase(3));
  } else {
  // ---- k-means++ seeding and Lloyd steps (Section 3.4)
  const int64_t ntiles = rr::kmeans_seed_tiles(F);
  RR_TRY(m.alloc(&kb.d2, F));
  RR_TRY(m.alloc(&kb.ov, F));
  RR_TRY(m.alloc(&kb.part_i, ntiles + 1));
  RR_TRY(m.alloc(&h->centers, k));
  kb.centers = h->centers;
  RR_TRY(m.alloc(&h->labels, F));
  kb.labels = h->labels;
  RR_TRY(m.alloc(&kb.next, F));
  RR_TRY(m.alloc(&kb.prev, F));
  RR_TRY(m.alloc(&kb.mcount, N));
  RR_TRY(m.alloc(&kb.mptr, N + 1));
  RR_TRY(m.alloc(&kb.dlist, std::max<int64_t>(2 * nnz, F) + 1));
  RR_TRY(m.alloc(&kb.dcount, N));
  RR_TRY(m.alloc(&kb.work, 1));
  RR_TRY(m.alloc(&kb.scan_scratch, rr::scan_scratch_len(N) + 8));
  RR_TRY(m.alloc(&h->n_S, 2 * (int64_t)k));
  kb.n_S = h->n_S;
  RR_TRY(m.alloc(&kb.Q, k));
  RR_TRY(m.alloc(&kb.qr, k));
  RR_TRY(m.alloc(&kb.D, F * (int64_t)k));
  RR_TRY(m.alloc(&kb.changes, 1));
  RR_TRY(m.alloc(&kb.work_ctr, 1));
  RR_TRY(m.alloc(&kb.order, F));
  RR_TRY(m.alloc(&kb.hot, F));
  RR_TRY(m.alloc(&kb.hot_col, 2048));
  RR_TRY(m.alloc(&kb.hot_n, 1));
  RR_TRY(m.alloc(&kb.task_ptr, F + 1));
  RR_TRY(m.alloc(&kb.task_it, rr::kmeans_pull_tasks_max(F, nnz)));
  RR_TRY(m.alloc(&kb.moved, F));
  RR_TRY(m.alloc(&kb.touched, N));
  RR_TRY(m.alloc(&kb.sparse_n, 4));
  if (h->opt.init_centers) {
    std::vector<char> seen(F, 0);
    for (int32_t s = 0; s < k; ++s) {
      const int32_t c = h->opt.init_centers[s];
      if (c < 0 || c >= F || seen[c]) {
        rr_set_error("init_centers[%d] = %d is out of range or repeated", s, c);
        return RR_INVALID_ARG;
      }
      seen[c] = 1;
    }
    RR_CUDA(cudaMemcpyAsync(h->centers, h->opt.init_centers, sizeof(int32_t) * k,
                            cudaMemcpyHostToDevice, st));
  } else {
    RR_TRY(rr::kmeanspp_seed(N, F, nnz, h->row_ptr, h->col_idx, h->col_ptr, h->row_idx, k,
                             h->opt.seed, h->opt.seed_pull_work, kb, st));
  }
  RR_TRY(phase(2));
  // seeded here: the seeding's nearest centres are the first Lloyd step's labels
  const bool seeded = !h->opt.init_centers && h->opt.kmeans_max_iter >= 1;
  if (!seeded) RR_TRY(rr::kmeans_init_labels(F, k, kb, st));
  RR_TRY(m.alloc(&h->gsum, F));
  RR_TRY(rr::kmeans_work_order(N, F, k, h->row_ptr, h->col_ptr, h->row_idx, kb, h->gsum, scratch64, st));
  int64_t *changes_host = nullptr;
  RR_CUDA(cudaMallocHost(&changes_host, sizeof(int64_t)));
  int32_t it = 0;
  rr_status ks = RR_OK;
  bool done = false;
  if (seeded) {
    ks = rr::kmeans_seeded_labels(F, k, kb, changes_host, st);
    it = 1;
    done = ks != RR_OK || *changes_host == 0;
  }
  while (!done && it < h->opt.kmeans_max_iter) {
    // the first step's moved features are the centres (labels of -1 before)
    const int64_t moved = it == 0 ? -1 : *changes_host;
    ++it;
    ks = rr::kmeans_lloyd_step(N, F, nnz, h->row_ptr, h->col_idx, h->col_ptr, h->row_idx, k, kb,
                               changes_host, h->opt.lloyd_pull_work, moved, st);
    if (ks != RR_OK || *changes_host == 0) break;
  }
  cudaFreeHost(changes_host);
  RR_TRY(ks);
  h->kmeans_iters = it;
  m.release(kb.D);
  m.release(kb.prev);
  m.release(kb.mcount);
  m.release(kb.mptr);
  m.release(kb.dlist);
  m.release(kb.dcount);
  m.release(kb.work);
  m.release(kb.scan_scratch);
  m.release(kb.d2);
  m.release(kb.ov);
  m.release(kb.Q);
  m.release(kb.qr);
  m.release(kb.hot);
  m.release(kb.hot_col);
  m.release(kb.hot_n);
  m.release(kb.task_ptr);
  m.release(kb.task_it);
  m.release(kb.moved);
  m.release(kb.touched);
  m.release(kb.sparse_n);

  RR_TRY(phase(3));
  }
  // ---- compaction, member lists, prolongation scale
  int32_t *remap = nullptr;
  RR_TRY(m.alloc(&remap, k + 1));
  int32_t k_eff = 0;
  RR_TRY(rr::compact_clusters(F, k, h->labels, h->n_S, remap, &k_eff, st));
  h->k_eff = k_eff;
  RR_TRY(m.alloc(&h->cl_ptr, k_eff + 1));
  RR_TRY(m.alloc(&h->members, F));
  int64_t *iota = nullptr;
  RR_TRY(m.alloc(&iota, F + 1));
  RR_TRY(rr::iota_i64(iota, F + 1, st));
  RR_TRY(rr::transpose_pattern(F, k_eff, F, iota, h->labels, h->cl_ptr, h->members, scratch64,
                               scratch64 + big, tmp32, scratch64 + 2 * big, st));
  RR_TRY(m.alloc(&h->s, k_eff));
  RR_TRY(rr::prolong_scale(k_eff, h->n_S, h->s, st));
  RR_TRY(rr::restrict_plan(k_eff, h->cl_ptr, h->rplan, scratch64, st));
  RR_TRY(rr::restrict_plan(k_eff, h->cl_ptr, h->bplan, scratch64, st, rr::kRestrictItemBatch));

  RR_TRY(phase(4));
  // ---- exact coarse Gram G = C^T C (C = X * onehot(labels), integer counts)
  const int64_t n_pad = round_up(std::max<int64_t>(N, 1), 64);
  const int32_t k_pad = (int32_t)round_up(k_eff, 128);
  const size_t ncount = (size_t)k_pad * n_pad;
  int32_t *C32 = nullptr;
  void *C16 = nullptr;
  int32_t *maxc_dev = nullptr;
  RR_TRY(m.alloc(&maxc_dev, 1));
  RR_TRY(m.alloc(&h->G, (int64_t)k_eff * k_eff));
  rr_status gs = m.alloc(&C32, ncount);
  int32_t max_count = 0;
  if (gs == RR_OK)
    gs = rr::coarse_counts(N, n_pad, k_pad, h->row_ptr, h->col_idx, h->labels, C32, maxc_dev, st);
  if (gs == RR_OK &&
      (cudaMemcpyAsync(&max_count, maxc_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess)) {
    rr_set_error("coarse counts failed");
    gs = RR_CUDA_ERROR;
  }
  if (gs == RR_OK && max_count >= 8192) {
    rr_set_error("rr_setup: a row holds %d features of one cluster (limit 8191)", max_count);
    gs = RR_UNSUPPORTED;
  }
  h->gram_on_tensor_cores = h->opt.gram == RR_GRAM_AUTO && max_count <= 2048 &&
                            rr::gram_tc_chunk(max_count) >= 64;
  if (gs == RR_OK && h->gram_on_tensor_cores) {
    gs = m.alloc(reinterpret_cast<uint16_t **>(&C16), ncount);
    if (gs == RR_OK) gs = rr::counts_to_half((int64_t)ncount, C32, C16, st);
    if (gs == RR_OK) m.release(C32), C32 = nullptr;
    if (gs == RR_OK)
      gs = rr::gram_tensor_cores(k_eff, k_pad, n_pad, C16, max_count, h->G, h->err, st,
                                 h->opt.wait_limit);
  } else if (gs == RR_OK) {
    gs = rr::gram_exact_cuda_cores(k_eff, k_pad, n_pad, C32, h->G, st);
  }
  if (gs == RR_OK) gs = check_dev_error(h, "coarse Gram");
  if (C32) m.release(C32);
  if (C16) m.release(C16);
  RR_TRY(gs);

  RR_TRY(phase(5));
  // ---- per-lambda coarse factor and smoother
  const int64_t kk = (int64_t)k_eff * k_eff;
  RR_TRY(m.alloc(&h->Ac, kk));
  RR_TRY(m.alloc(&h->Lw, kk));
  RR_TRY(m.alloc(&h->Linv, kk));
  RR_TRY(m.alloc(&h->Ainv, kk));
  RR_TRY(m.alloc(&h->d, F));
  RR_TRY(m.alloc(&h->omega_dev, 1));
  RR_TRY(m.alloc(&h->max_bits, 1));
  RR_TRY(coarse_eigen_setup(h));
  if (h->opt.precision == RR_PREC_MIXED && !h->mu)
    RR_TRY(m.alloc(&h->Ainv32, (int64_t)k_eff * ((k_eff + 3) & ~3)));
  // the smoother now; the coarse factor is started when rr_setup returns
  RR_TRY(build_smoother(h, lambda));

  RR_TRY(phase(6));
  // ---- the patterns (built alongside) and the solve workspace
  RR_TRY(patterns.finish());
  RR_TRY(check_dev_error(h, "rr_setup (patterns)"));
  // the gather kernels are timed here, with nothing else running
  if (h->opt.precision == RR_PREC_MIXED || h->opt.gather != RR_GATHER_AUTO) {
    const bool split = h->opt.gather == RR_GATHER_LANES_STAGED;
    RR_TRY(rr::sliced_choose_gather(h->pcsr, split ? RR_GATHER_LANES : h->opt.gather, st));
    RR_TRY(rr::sliced_choose_gather(h->pcsc, split ? RR_GATHER_STAGED : h->opt.gather, st));
  }
  if (h->opt.precision == RR_PREC_MIXED) RR_TRY(rr::split_set_wd(h->split, h->omega, h->d, st));
  RR_TRY(alloc_solve_workspace(h));
  m.release(tmp32);
  m.release(scratch64);
  m.release(iota);
  m.release(remap);
  m.release(kb.part_i);
  m.release(kb.next);
  m.release(kb.changes);
  m.release(kb.work_ctr);
  m.release(kb.order);
  RR_TRY(phase(7));
  return RR_OK;
}

// ---- the operator: t = X^T (X v) + lambda v, finished by the epilogue ep.
// x32_ready: the FP32 copy of v is already in the X pass's vector (written by
// the kernel that made v; sparse X, fp32 only).
rr_status op_apply(rr_handle *h, const double *v, const rr::CscEpilogue &ep, const int32_t *stop,
                   cudaStream_t st, bool fp32 = false, bool x32_ready = false) {
  if (h->dense) return rr::dense_operator(h->N, h->F, h->Xd, v, h->u, h->dpart, ep, fp32, st);
  if (fp32 && h->split.active) return rr::split_apply(h->split, v, ep, stop, st, x32_ready);
  RR_TRY(rr::sliced_gather(h->pcsr, v, nullptr, stop, st, fp32, x32_ready));
  RR_TRY(rr::sliced_gather(h->pcsc, nullptr, &h->pcsr, stop, st, fp32));
  RR_TRY(rr::sliced_epilogue(h->pcsc, ep, st));
  return RR_OK;
}

// b = X^T y (FP64).
rr_status rhs_apply(rr_handle *h, const double *y, double *b, cudaStream_t st) {
  rr::CscEpilogue rhs{rr::CSC_RHS, 0.0, 0.0, nullptr, nullptr, nullptr, b, nullptr, nullptr};
  if (h->dense) return rr::dense_transposed(h->N, h->F, h->Xd, y, h->dpart, rhs, false, st);
  RR_TRY(rr::sliced_gather(h->pcsc, y, nullptr, nullptr, st));
  RR_TRY(rr::sliced_epilogue(h->pcsc, rhs, st));
  return RR_OK;
}

// ---- the preconditioner: z = M^{-1} r, with <r, z> partials in part_rz.
// The X pass's FP32 vector when the PCG loop's producers can write the
// applied vectors' FP32 copies there (mixed precision, sparse X), else nullptr.
float *pcg_x32(rr_handle *h) {
  if (h->opt.precision != RR_PREC_MIXED || h->dense) return nullptr;
  return static_cast<float *>(h->split.active ? h->split.xt.xq : h->pcsr.xq);
}

// x32: where the producers of the applied vectors also write their FP32
// copies (the X pass's vector), or nullptr; with z1_ready, z1's copy is there.
rr_status apply_precond(rr_handle *h, const double *r, double *z, const int32_t *stop, int *n_rz,
                        bool z1_ready, cudaStream_t st, bool fp32 = false, float *x32 = nullptr) {
  const int64_t F = h->F;
  *n_rz = rr::kVecGrid;
  switch (h->opt.solver) {
    case RR_SOLVER_CG:
      return rr::jacobi(F, 1.0, r, nullptr, z, h->part_rz, stop, st);
    case RR_SOLVER_DCG:
      return rr::jacobi(F, 1.0, r, h->d, z, h->part_rz, stop, st);
    default: {
      // symmetric two-level cycle: z1 = w D^-1 r; r1 = r - A z1; e_c = A_c^-1 P^T r1;
      // z2 = z1 + P e_c; r2 = r - A z2; z = z2 + w D^-1 r2
      if (!z1_ready) RR_TRY(rr::jacobi(F, h->omega, r, h->d, h->z1, nullptr, stop, st));
      rr::CscEpilogue pre{rr::CSC_PRE, h->lambda, h->omega, h->z1, r, h->d, h->r1, nullptr, stop};
      RR_TRY(op_apply(h, h->z1, pre, stop, st, fp32, x32 != nullptr && z1_ready));
      RR_TRY(rr::restrict_clusters(h->rplan, h->members, h->r1, h->s, stop, st));
      RR_TRY(coarse_step(h, stop, st, fp32));
      RR_TRY(rr::prolong_add(F, h->labels, h->s, h->ec, h->z1, h->z2, stop, st, x32));
      rr::CscEpilogue post{rr::CSC_POST, h->lambda, h->omega, h->z2, r, h->d, z, h->part_rz, stop};
      return op_apply(h, h->z2, post, stop, st, fp32, x32 != nullptr);
    }
  }
}

// ---- one PCG iteration on the handle's vectors (w_int, r, z, p, q); every
// kernel returns at once when S->converged is set.
rr_status pcg_iteration(rr_handle *h, cudaStream_t st) {
  const int64_t F = h->F;
  const bool twolevel = h->opt.solver == RR_SOLVER_TWOLEVEL;
  const int32_t *stop = &h->S->converged;
  const bool fp32 = h->opt.precision == RR_PREC_MIXED;
  float *x32 = pcg_x32(h);
  int n_rz = 0;
  RR_TRY(apply_precond(h, h->r, h->z, stop, &n_rz, twolevel, st, fp32, x32));
  RR_TRY(rr::pcg_direction(F, h->part_rz, n_rz, h->z, h->p, h->S, st, x32));
  rr::CscEpilogue ap{rr::CSC_PCG, h->lambda, h->omega, h->p, nullptr, nullptr, h->q, h->part_pq, stop};
  RR_TRY(op_apply(h, h->p, ap, stop, st, fp32, x32 != nullptr));
  RR_TRY(rr::pcg_update(F, h->part_rz, n_rz, h->part_pq, rr::kVecGrid, h->p, h->q, h->w_int,
                        h->r, h->omega, h->d, twolevel ? h->z1 : nullptr, h->part_rr, h->S, st,
                        twolevel ? x32 : nullptr,
                        (fp32 && h->split.active) ? h->split.wd : nullptr, h->history,
                        h->hist_cap));
  return RR_OK;
}

void drop_fcg_cache(rr_handle *h);

void destroy_graph(rr_handle *h) {
  drop_fcg_cache(h);
  if (h->loop_exec) cudaGraphExecDestroy(h->loop_exec);
  if (h->loop_graph) cudaGraphDestroy(h->loop_graph);
  h->loop_exec = nullptr;
  h->loop_graph = nullptr;
}

// The whole iteration loop as one graph: a conditional while node whose body
// is one PCG iteration followed by a kernel that keeps the loop going while
// the device-side state says "not converged and below the iteration limit".
rr_status build_loop_graph(rr_handle *h) {
  destroy_graph(h);
  cudaGraph_t g = nullptr;
  RR_CUDA(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle hc;
  RR_CUDA(cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hc;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  RR_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaStream_t cs = h->cap_stream;
  RR_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  const int64_t l0 = rr_launch_counter;
  rr_status s = pcg_iteration(h, cs);
  if (s == RR_OK) s = rr::loop_condition(hc, h->S, cs);
  h->body_kernels = rr_launch_counter - l0;   // recorded, not launched
  rr_launch_counter = l0;
  cudaGraph_t captured = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(cs, &captured);
  if (s != RR_OK || ec != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    if (s != RR_OK) return s;
    rr_set_error("graph capture failed: %s", cudaGetErrorString(ec));
    return RR_CUDA_ERROR;
  }
  h->loop_graph = g;
  RR_CUDA(cudaGraphInstantiate(&h->loop_exec, g, 0));
  return RR_OK;
}

rr_status true_residual(rr_handle *h, const double *w, double *rr_out) {
  cudaStream_t st = h->st;
  rr::CscEpilogue ep{rr::CSC_RESID, h->lambda, h->omega, w, h->b, h->d, h->rt, h->part_bb, nullptr};
  RR_TRY(op_apply(h, w, ep, nullptr, st));
  RR_TRY(rr::sum_parts(h->part_bb, rr::kVecGrid, h->scal, st));
  RR_CUDA(cudaMemcpyAsync(h->scal_host, h->scal, sizeof(double), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  *rr_out = h->scal_host[0];
  return RR_OK;
}

// Runs PCG iterations until convergence or the limit: one graph launch, or
// (use_graphs = 0) batches of check_every iterations with a read-back each.
rr_status run_iterations(rr_handle *h, int32_t limit) {
  cudaStream_t st = h->st;
  *h->limit_host = limit;
  RR_CUDA(cudaMemcpyAsync(&h->S->limit, h->limit_host, sizeof(int32_t), cudaMemcpyHostToDevice, st));
  if (h->opt.use_graphs) {
    if (!h->loop_exec) RR_TRY(build_loop_graph(h));
    const int32_t it0 = h->S_host->iter;
    RR_CUDA(cudaGraphLaunch(h->loop_exec, st));
    RR_CUDA(cudaMemcpyAsync(h->S_host, h->S, sizeof(rr::PcgScalars), cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    // every run of the loop body launches all of its kernels
    rr_launch_counter += h->body_kernels * std::max<int64_t>(1, h->S_host->iter - it0);
  } else {
    const int32_t every = std::max(1, h->opt.check_every);
    for (;;) {
      for (int32_t c = 0; c < every; ++c) RR_TRY(pcg_iteration(h, st));
      RR_CUDA(cudaMemcpyAsync(h->S_host, h->S, sizeof(rr::PcgScalars), cudaMemcpyDeviceToHost, st));
      RR_CUDA(cudaStreamSynchronize(st));
      if (h->S_host->converged || h->S_host->iter >= limit) break;
    }
  }
  RR_CUDA(cudaMemcpyAsync(h->S_host, h->S, sizeof(rr::PcgScalars), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  return RR_OK;
}

// b = X^T y (y == NULL: b is already set); w = 0; r = b; ||b||;
// z1 = omega D^-1 r (no synchronisation).
rr_status solve_start(rr_handle *h, const double *y, double tol, cudaStream_t st) {
  const int64_t F = h->F;
  if (y) RR_TRY(rhs_apply(h, y, h->b, st));
  RR_CUDA(cudaMemsetAsync(h->w_int, 0, sizeof(double) * F, st));
  RR_TRY(rr::copy_f64(h->r, h->b, F, st));
  RR_TRY(rr::dot_parts(F, h->b, h->b, h->part_bb, st));
  RR_CUDA(cudaMemsetAsync(h->S, 0, sizeof(rr::PcgScalars), st));
  RR_TRY(rr::pcg_start(h->part_bb, rr::kVecGrid, h->part_bb, rr::kVecGrid, tol, 1, h->S, st));
  if (h->opt.solver == RR_SOLVER_TWOLEVEL)
    RR_TRY(rr::jacobi(F, h->omega, h->r, h->d, h->z1, nullptr, nullptr, st, pcg_x32(h)));
  return RR_OK;
}

// Refinement: continue from w with the true residual rt and a fresh direction.
rr_status solve_restart(rr_handle *h, double tol, cudaStream_t st) {
  const int64_t F = h->F;
  RR_TRY(rr::copy_f64(h->r, h->rt, F, st));
  RR_TRY(rr::dot_parts(F, h->r, h->r, h->part_rr, st));
  RR_TRY(rr::pcg_start(h->part_bb, 1, h->part_rr, rr::kVecGrid, tol, 0, h->S, st));
  if (h->opt.solver == RR_SOLVER_TWOLEVEL)
    RR_TRY(rr::jacobi(F, h->omega, h->r, h->d, h->z1, nullptr, nullptr, st, pcg_x32(h)));
  return RR_OK;
}

rr_status solve_impl(rr_handle *h, const double *y, double *w, double tol, rr_info *info) {
  cudaStream_t st = h->st;
  const int64_t F = h->F;
  RR_TRY(solve_start(h, y, tol, st));
  RR_CUDA(cudaMemcpyAsync(h->S_host, h->S, sizeof(rr::PcgScalars), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));

  const int32_t max_iter = h->opt.max_iter;
  int32_t restarts = 0;
  double true_rr = 0.0;
  rr_status result = RR_OK;
  for (;;) {
    RR_TRY(run_iterations(h, max_iter));
    const rr::PcgScalars Sh = *h->S_host;
    if (Sh.nonfinite) {
      rr_set_error("rr_solve: non-finite residual or dot product");
      result = RR_NONFINITE;
      break;
    }
    RR_TRY(true_residual(h, h->w_int, &true_rr));
    if (!isfinite(true_rr)) {
      rr_set_error("rr_solve: non-finite true residual");
      result = RR_NONFINITE;
      break;
    }
    if (sqrt(true_rr) <= Sh.target) break;
    if (Sh.iter >= max_iter || restarts >= h->opt.max_restarts) {
      rr_set_error("rr_solve: not converged after %d iterations (%d restarts)", Sh.iter, restarts);
      result = RR_NOT_CONVERGED;
      break;
    }
    // refinement: continue from w with the true residual and a fresh direction
    ++restarts;
    RR_TRY(solve_restart(h, tol, st));
  }
  if (w) RR_TRY(rr::copy_f64(w, h->w_int, F, st));
  RR_CUDA(cudaMemcpyAsync(h->S_host, h->S, sizeof(rr::PcgScalars), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  if (info) {
    const rr::PcgScalars Sh = *h->S_host;
    info->iters = Sh.iter;
    info->restarts = restarts;
    info->rel_res = Sh.bnorm > 0 ? sqrt(Sh.rr) / Sh.bnorm : 0.0;
    info->true_rel_res = Sh.bnorm > 0 ? sqrt(true_rr) / Sh.bnorm : 0.0;
  }
  return result;
}

// ---- flexible CG (Algorithm 3, m = 1) with the two-level cycle; the coarse
// solve is the network's (net != NULL, with the Cholesky fallback pass) or
// the Cholesky solve.
rr_status fcg_reserve(rr_handle *h) {
  if (h->Sf) return RR_OK;
  RR_TRY(h->mem.alloc(&h->p_prev, h->F));
  RR_TRY(h->mem.alloc(&h->q_prev, h->F));
  RR_TRY(h->mem.alloc(&h->part_zq, rr::kVecGrid));
  RR_TRY(h->mem.alloc(&h->part3, 3 * rr::kVecGrid));
  RR_TRY(h->mem.alloc(&h->Sf, 1));
  RR_CUDA(cudaMallocHost(&h->Sf_host, sizeof(rr::FcgScalars)));
  return RR_OK;
}

// The cycle's second half from e_c: z2 = z1 + P e_c; z = z2 + omega D^-1 (r - A z2);
// then the FCG direction p and q = A p with its dots. All kernels skip when *stop.
rr_status fcg_tail(rr_handle *h, const int32_t *stop, bool fp32, cudaStream_t st) {
  const int64_t F = h->F;
  RR_TRY(rr::prolong_add(F, h->labels, h->s, h->ec, h->z1, h->z2, stop, st));
  rr::CscEpilogue post{rr::CSC_POST, h->lambda, h->omega, h->z2, h->r, h->d, h->z, h->part_rz, stop};
  RR_TRY(op_apply(h, h->z2, post, stop, st, fp32));
  RR_TRY(rr::fcg_dot(F, h->z, h->q_prev, h->part_zq, stop, st));
  RR_TRY(rr::fcg_direction(F, h->part_zq, h->Sf, h->z, h->p_prev, h->p, stop, st));
  rr::CscEpilogue ap{rr::CSC_PCG, h->lambda, h->omega, h->p, nullptr, nullptr, h->q, h->part_pq, stop};
  RR_TRY(op_apply(h, h->p, ap, stop, st, fp32));
  RR_TRY(rr::fcg_dots(F, h->p, h->r, h->q, h->part3, stop, st));
  return RR_OK;
}

rr_status tlfcg_reserve(rr_handle *h) {
  if (h->St) return RR_OK;
  for (double **v : {&h->tz, &h->tr, &h->tp, &h->tq, &h->tzz}) RR_TRY(h->mem.alloc(v, h->F));
  for (double **v : {&h->t_rz, &h->t_pq, &h->t_rr}) RR_TRY(h->mem.alloc(v, rr::kVecGrid));
  RR_TRY(h->mem.alloc(&h->St, 1));
  RR_CUDA(cudaMemsetAsync(h->St, 0, sizeof(rr::PcgScalars), h->st));
  return RR_OK;
}

// One TLFCG iteration: z = z1 + P A_c^-1 P^T r1 with (z1, r1) after two plain
// CG steps on A z1 = r from z1 = 0 (the rougher), then the FCG(1) step. The
// rougher's kernels stop when the outer loop has converged.
rr_status tlfcg_iteration(rr_handle *h, cudaStream_t st) {
  const bool fp32 = h->opt.precision == RR_PREC_MIXED;
  const int64_t F = h->F;
  const int32_t *stop = &h->Sf->converged;
  const int32_t *istop = &h->St->converged;
  RR_TRY(rr::inner_start(h->St, stop, st));
  RR_TRY(rr::copy_f64(h->tr, h->r, F, st));
  RR_CUDA(cudaMemsetAsync(h->tz, 0, sizeof(double) * F, st));
  for (int j = 0; j < 2; ++j) {
    RR_TRY(rr::jacobi(F, 1.0, h->tr, nullptr, h->tzz, h->t_rz, istop, st));
    RR_TRY(rr::pcg_direction(F, h->t_rz, rr::kVecGrid, h->tzz, h->tp, h->St, st));
    rr::CscEpilogue ap{rr::CSC_PCG, h->lambda, h->omega, h->tp, nullptr, nullptr, h->tq, h->t_pq, istop};
    RR_TRY(op_apply(h, h->tp, ap, istop, st, fp32));
    RR_TRY(rr::pcg_update(F, h->t_rz, rr::kVecGrid, h->t_pq, rr::kVecGrid, h->tp, h->tq, h->tz,
                          h->tr, 1.0, nullptr, nullptr, h->t_rr, h->St, st));
  }
  RR_TRY(rr::restrict_clusters(h->rplan, h->members, h->tr, h->s, stop, st));
  RR_TRY(coarse_step(h, stop, st, fp32));
  RR_TRY(rr::prolong_add(F, h->labels, h->s, h->ec, h->tz, h->z, stop, st));
  RR_TRY(rr::fcg_dot(F, h->z, h->q_prev, h->part_zq, stop, st));
  RR_TRY(rr::fcg_direction(F, h->part_zq, h->Sf, h->z, h->p_prev, h->p, stop, st));
  rr::CscEpilogue ap{rr::CSC_PCG, h->lambda, h->omega, h->p, nullptr, nullptr, h->q, h->part_pq, stop};
  RR_TRY(op_apply(h, h->p, ap, stop, st, fp32));
  RR_TRY(rr::fcg_dots(F, h->p, h->r, h->q, h->part3, stop, st));
  RR_TRY(rr::fcg_update(h->F, h->part_pq, h->part3, h->p, h->q, h->w_int, h->r, h->omega, h->d,
                        h->z1, h->p_prev, h->q_prev, h->part_rr, h->Sf, st));
  RR_TRY(rr::fcg_finish(h->part_rr, h->part_pq, h->Sf, h->history, h->hist_cap, st));
  return RR_OK;
}

rr_status fcg_iteration(rr_handle *h, const rr_mlp *net, cudaStream_t st) {
  if (h->opt.solver == RR_SOLVER_TLFCG) return tlfcg_iteration(h, st);
  const bool fp32 = h->opt.precision == RR_PREC_MIXED;
  const int32_t *stop = &h->Sf->converged;
  // pre-smoothing (z1 from the previous update), restriction
  rr::CscEpilogue pre{rr::CSC_PRE, h->lambda, h->omega, h->z1, h->r, h->d, h->r1, nullptr, stop};
  RR_TRY(op_apply(h, h->z1, pre, stop, st, fp32));
  RR_TRY(rr::restrict_clusters(h->rplan, h->members, h->r1, h->s, stop, st));
  if (net) {
    RR_TRY(rr::mlp_coarse(net, h->rplan, h->s, h->ec, stop, st));
  } else {
    RR_TRY(coarse_step(h, stop, st, fp32));
  }
  RR_TRY(fcg_tail(h, stop, fp32, st));
  if (net) {
    // the step is checked before it is taken; a rejected learned step is
    // redone with the Cholesky coarse solve (same restriction)
    RR_TRY(rr::fcg_decide(h->part_rz, h->part_pq, h->part3, h->Sf, st));
    const int32_t *fb = &h->Sf->skip_fb;
    RR_TRY(coarse_step(h, fb, st, fp32));
    RR_TRY(fcg_tail(h, fb, fp32, st));
  }
  RR_TRY(rr::fcg_update(h->F, h->part_pq, h->part3, h->p, h->q, h->w_int, h->r, h->omega, h->d,
                        h->z1, h->p_prev, h->q_prev, h->part_rr, h->Sf, st));
  RR_TRY(rr::fcg_finish(h->part_rr, h->part_pq, h->Sf, h->history, h->hist_cap, st));
  return RR_OK;
}

struct GraphExec {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t body = 0;
  ~GraphExec() {
    if (exec) cudaGraphExecDestroy(exec);
    if (g) cudaGraphDestroy(g);
  }
};

void drop_fcg_cache(rr_handle *h) {
  delete static_cast<GraphExec *>(h->fcg_cache);
  h->fcg_cache = nullptr;
}

rr_status build_fcg_graph(rr_handle *h, const rr_mlp *net, GraphExec &G) {
  RR_CUDA(cudaGraphCreate(&G.g, 0));
  cudaGraphConditionalHandle hc;
  RR_CUDA(cudaGraphConditionalHandleCreate(&hc, G.g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hc;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  RR_CUDA(cudaGraphAddNode(&node, G.g, nullptr, nullptr, 0, &cp));
  cudaStream_t cs = h->cap_stream;
  RR_CUDA(cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal));
  const int64_t l0 = rr_launch_counter;
  rr_status s = fcg_iteration(h, net, cs);
  if (s == RR_OK) s = rr::fcg_condition(hc, h->Sf, cs);
  G.body = rr_launch_counter - l0;   // recorded, not launched
  rr_launch_counter = l0;
  cudaGraph_t captured = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(cs, &captured);
  if (s != RR_OK || ec != cudaSuccess) {
    cudaGraphDestroy(G.g);
    G.g = nullptr;
    cudaGetLastError();
    if (s != RR_OK) return s;
    rr_set_error("FCG graph capture failed: %s", cudaGetErrorString(ec));
    return RR_CUDA_ERROR;
  }
  RR_CUDA(cudaGraphInstantiate(&G.exec, G.g, 0));
  return RR_OK;
}

rr_status fcg_run(rr_handle *h, const rr_mlp *net, GraphExec *G, int32_t limit) {
  cudaStream_t st = h->st;
  h->Sf_host->limit = limit;
  RR_CUDA(cudaMemcpyAsync(&h->Sf->limit, &h->Sf_host->limit, sizeof(int32_t), cudaMemcpyHostToDevice, st));
  RR_CUDA(cudaMemcpyAsync(h->Sf_host, h->Sf, sizeof(rr::FcgScalars), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  const int32_t it0 = h->Sf_host->iter;
  if (G) {
    RR_CUDA(cudaGraphLaunch(G->exec, st));
    RR_CUDA(cudaMemcpyAsync(h->Sf_host, h->Sf, sizeof(rr::FcgScalars), cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    rr_launch_counter += G->body * std::max<int64_t>(1, h->Sf_host->iter - it0);
    return RR_OK;
  }
  const int32_t every = std::max(1, h->opt.check_every);
  for (;;) {
    for (int32_t c = 0; c < every; ++c) RR_TRY(fcg_iteration(h, net, st));
    RR_CUDA(cudaMemcpyAsync(h->Sf_host, h->Sf, sizeof(rr::FcgScalars), cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    if (h->Sf_host->converged || h->Sf_host->iter >= limit) return RR_OK;
  }
}

rr_status solve_fcg_impl(rr_handle *h, const rr_mlp *net, const double *y, double *w, double tol,
                         rr_info *info) {
  cudaStream_t st = h->st;
  const int64_t F = h->F;
  RR_TRY(fcg_reserve(h));
  if (h->opt.solver == RR_SOLVER_TLFCG) RR_TRY(tlfcg_reserve(h));
  if (y) RR_TRY(rhs_apply(h, y, h->b, st));
  RR_CUDA(cudaMemsetAsync(h->w_int, 0, sizeof(double) * F, st));
  RR_CUDA(cudaMemsetAsync(h->p_prev, 0, sizeof(double) * F, st));
  RR_CUDA(cudaMemsetAsync(h->q_prev, 0, sizeof(double) * F, st));
  RR_TRY(rr::copy_f64(h->r, h->b, F, st));
  RR_TRY(rr::dot_parts(F, h->b, h->b, h->part_bb, st));
  RR_CUDA(cudaMemsetAsync(h->Sf, 0, sizeof(rr::FcgScalars), st));
  RR_TRY(rr::fcg_start(h->part_bb, rr::kVecGrid, h->part_bb, tol, 1, net ? 1 : 0, h->Sf, st));
  RR_TRY(rr::jacobi(F, h->omega, h->r, h->d, h->z1, nullptr, nullptr, st));

  // the graph is kept in the handle when no network is involved (a network's
  // buffers may be freed between calls); set_lambda drops it
  GraphExec graph;
  GraphExec *G = nullptr;
  if (h->opt.use_graphs) {
    if (net) {
      RR_TRY(build_fcg_graph(h, net, graph));
      G = &graph;
    } else {
      if (!h->fcg_cache) {
        GraphExec *c = new GraphExec();
        const rr_status bs = build_fcg_graph(h, nullptr, *c);
        if (bs != RR_OK) {
          delete c;
          return bs;
        }
        h->fcg_cache = c;
      }
      G = static_cast<GraphExec *>(h->fcg_cache);
    }
  }
  const int32_t max_iter = h->opt.max_iter;
  int32_t restarts = 0;
  double true_rr = 0.0;
  rr_status result = RR_OK;
  for (;;) {
    RR_TRY(fcg_run(h, net, G, max_iter));
    const rr::FcgScalars Sh = *h->Sf_host;
    if (Sh.nonfinite) {
      rr_set_error("rr_solve_fcg: non-finite residual or dot product");
      result = RR_NONFINITE;
      break;
    }
    RR_TRY(true_residual(h, h->w_int, &true_rr));
    if (!isfinite(true_rr)) {
      rr_set_error("rr_solve_fcg: non-finite true residual");
      result = RR_NONFINITE;
      break;
    }
    if (sqrt(true_rr) <= Sh.target) break;
    if (Sh.iter >= max_iter || restarts >= h->opt.max_restarts) {
      rr_set_error("rr_solve_fcg: not converged after %d iterations (%d restarts)", Sh.iter, restarts);
      result = RR_NOT_CONVERGED;
      break;
    }
    ++restarts;
    RR_TRY(rr::copy_f64(h->r, h->rt, F, st));
    RR_TRY(rr::dot_parts(F, h->r, h->r, h->part_rr, st));
    RR_TRY(rr::fcg_start(h->part_bb, 1, h->part_rr, tol, 0, net ? 1 : 0, h->Sf, st));
    RR_TRY(rr::jacobi(F, h->omega, h->r, h->d, h->z1, nullptr, nullptr, st));
  }
  if (w) RR_TRY(rr::copy_f64(w, h->w_int, F, st));
  RR_CUDA(cudaMemcpyAsync(h->Sf_host, h->Sf, sizeof(rr::FcgScalars), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  if (info) {
    const rr::FcgScalars Sh = *h->Sf_host;
    info->iters = Sh.iter;
    info->restarts = restarts;
    info->fallbacks = Sh.fallbacks;
    info->rel_res = Sh.bnorm > 0 ? sqrt(Sh.rr) / Sh.bnorm : 0.0;
    info->true_rel_res = Sh.bnorm > 0 ? sqrt(true_rr) / Sh.bnorm : 0.0;
  }
  return result;
}

// ---- several independent problems in one graph: the PCG loop of every
// problem is a conditional while node of one parent graph, all of them
// parallel branches, so the problems' kernels can run concurrently.
struct ManyGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~ManyGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (g) cudaGraphDestroy(g);
  }
};

rr_status build_many_graph(int32_t n, rr_handle *const *hs, ManyGraph &G, std::vector<int64_t> &body) {
  RR_CUDA(cudaGraphCreate(&G.g, 0));
  body.assign(n, 0);
  for (int32_t i = 0; i < n; ++i) {
    rr_handle *h = hs[i];
    cudaGraphConditionalHandle hc;
    RR_CUDA(cudaGraphConditionalHandleCreate(&hc, G.g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wait = nullptr, node;
    if (h->ready) RR_CUDA(cudaGraphAddEventWaitNode(&wait, G.g, nullptr, 0, h->ready));
    RR_CUDA(cudaGraphAddNode(&node, G.g, wait ? &wait : nullptr, nullptr, wait ? 1 : 0, &cp));
    cudaStream_t cs = h->cap_stream;
    RR_CUDA(cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
    const int64_t l0 = rr_launch_counter;
    rr_status s = pcg_iteration(h, cs);
    if (s == RR_OK) s = rr::loop_condition(hc, h->S, cs);
    body[i] = rr_launch_counter - l0;   // recorded, not launched
    rr_launch_counter = l0;
    cudaGraph_t captured = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cs, &captured);
    if (s != RR_OK || ec != cudaSuccess) {
      cudaGraphDestroy(G.g);
      G.g = nullptr;
      cudaGetLastError();
      if (s != RR_OK) return s;
      rr_set_error("rr_solve_many: graph capture failed: %s", cudaGetErrorString(ec));
      return RR_CUDA_ERROR;
    }
  }
  RR_CUDA(cudaGraphInstantiate(&G.exec, G.g, 0));
  return RR_OK;
}

rr_status solve_many_impl(int32_t n, rr_handle *const *hs, const double *const *ys,
                          double *const *ws, double tol, cudaStream_t st, rr_info *infos) {
  std::vector<int32_t> restarts(n, 0), done(n, 0);
  std::vector<double> true_rr(n, 0.0);
  std::vector<rr_status> result(n, RR_OK);
  for (int32_t i = 0; i < n; ++i) {
    RR_TRY(solve_start(hs[i], ys[i], tol, st));
    hs[i]->S_host->limit = hs[i]->opt.max_iter;
  }
  ManyGraph G;
  std::vector<int64_t> body;
  RR_TRY(build_many_graph(n, hs, G, body));
  static const int32_t kStopped = 1;
  for (;;) {
    std::vector<int32_t> it0(n);
    for (int32_t i = 0; i < n; ++i) {
      rr_handle *h = hs[i];
      // a while node runs its body once per launch before testing the
      // condition: a finished problem that stopped on its iteration cap is
      // marked converged so that a relaunch for the others leaves it as it is
      if (done[i] && !h->S_host->converged)
        RR_CUDA(cudaMemcpyAsync(&h->S->converged, &kStopped, sizeof(int32_t),
                                cudaMemcpyHostToDevice, st));
      *h->limit_host = h->opt.max_iter;
      RR_CUDA(cudaMemcpyAsync(&h->S->limit, h->limit_host, sizeof(int32_t), cudaMemcpyHostToDevice, st));
      RR_CUDA(cudaMemcpyAsync(h->S_host, h->S, sizeof(rr::PcgScalars), cudaMemcpyDeviceToHost, st));
    }
    RR_CUDA(cudaStreamSynchronize(st));
    for (int32_t i = 0; i < n; ++i) it0[i] = hs[i]->S_host->iter;
    RR_CUDA(cudaGraphLaunch(G.exec, st));
    for (int32_t i = 0; i < n; ++i)
      RR_CUDA(cudaMemcpyAsync(hs[i]->S_host, hs[i]->S, sizeof(rr::PcgScalars), cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    bool any = false;
    for (int32_t i = 0; i < n; ++i) {
      rr_handle *h = hs[i];
      rr_launch_counter += body[i] * std::max<int64_t>(1, h->S_host->iter - it0[i]);
      if (done[i]) continue;
      const rr::PcgScalars Sh = *h->S_host;
      if (Sh.nonfinite) {
        result[i] = RR_NONFINITE;
        done[i] = 1;
        continue;
      }
      RR_TRY(true_residual(h, h->w_int, &true_rr[i]));
      if (!isfinite(true_rr[i])) {
        result[i] = RR_NONFINITE;
        done[i] = 1;
      } else if (sqrt(true_rr[i]) <= Sh.target) {
        done[i] = 1;
      } else if (Sh.iter >= h->opt.max_iter || restarts[i] >= h->opt.max_restarts) {
        result[i] = RR_NOT_CONVERGED;
        done[i] = 1;
      } else {
        ++restarts[i];
        RR_TRY(solve_restart(h, tol, st));
        any = true;
      }
    }
    if (!any) break;
  }
  rr_status worst = RR_OK;
  for (int32_t i = 0; i < n; ++i) {
    rr_handle *h = hs[i];
    RR_TRY(rr::copy_f64(ws[i], h->w_int, h->F, st));
    RR_CUDA(cudaMemcpyAsync(h->S_host, h->S, sizeof(rr::PcgScalars), cudaMemcpyDeviceToHost, st));
    if (result[i] != RR_OK && worst != RR_NONFINITE) worst = result[i];
  }
  RR_CUDA(cudaStreamSynchronize(st));
  for (int32_t i = 0; i < n; ++i) {
    const rr_status e = check_dev_error(hs[i], "rr_solve_many");
    if (e != RR_OK) return e;
    if (!infos) continue;
    rr_handle *h = hs[i];
    const rr::PcgScalars Sh = *h->S_host;
    rr_info &I = infos[i];
    I.iters = Sh.iter;
    I.restarts = restarts[i];
    I.rel_res = Sh.bnorm > 0 ? sqrt(Sh.rr) / Sh.bnorm : 0.0;
    I.true_rel_res = Sh.bnorm > 0 ? sqrt(true_rr[i]) / Sh.bnorm : 0.0;
    I.k_eff = h->k_eff;
    I.kmeans_iters = h->kmeans_iters;
    I.omega = h->omega;
    I.setup_ms = h->setup_ms;
    I.gram_tensor_cores = h->gram_on_tensor_cores ? 1 : 0;
    I.gather_staged = (h->pcsr.staged ? 1 : 0) | (h->pcsc.staged ? 2 : 0);
    I.fallbacks = 0;
    for (int j = 0; j < 8; ++j) I.setup_phase_ms[j] = h->phase_ms[j];
  }
  if (worst == RR_NOT_CONVERGED) rr_set_error("rr_solve_many: some problems did not reach tol");
  if (worst == RR_NONFINITE) rr_set_error("rr_solve_many: non-finite values in some problems");
  return worst;
}


// ---- Bayesian regression by Gibbs sampling with noise injection (Section 2,
// Eq. (ni_xtx)); the draws are k_bayes.cu's.
constexpr uint64_t kStreamGamma = 1ULL << 20;

// u = X v in FP64 (the residual y - X w that tau is drawn from).
rr_status matvec_f64(rr_handle *h, const double *v, double *u, cudaStream_t st) {
  if (h->dense) return rr::dense_matvec(h->N, h->F, h->Xd, v, u, nullptr, false, st);
  RR_TRY(rr::sliced_gather(h->pcsr, v, nullptr, nullptr, st, false));
  RR_TRY(rr::sliced_slot_sum(h->pcsr, u, st));
  return RR_OK;
}

rr_status bayes_impl(rr_handle *h, const double *y, const rr_bayes_params &p, int32_t n_samples,
                     int32_t burnin, double *w_mean, double *lam_trace, double *tau_trace,
                     int32_t *iters) {
  cudaStream_t st = h->st;
  const int64_t N = h->N, F = h->F;
  if (!h->bayes_y) RR_TRY(h->mem.alloc(&h->bayes_y, std::max<int64_t>(N, 1)));
  if (w_mean) RR_CUDA(cudaMemsetAsync(w_mean, 0, sizeof(double) * F, st));
  const bool draw_tau = p.a_tau > 0.0;
  double lam = p.lambda0, tau = p.tau0;
  rr_status result = RR_OK;
  for (int32_t t = 0; t < n_samples; ++t) {
    // b = X^T (y + e1) + e2 / tau
    RR_TRY(rr::bayes_noise_y(N, y, p.seed, t, tau, h->bayes_y, st));
    RR_TRY(rhs_apply(h, h->bayes_y, h->b, st));
    RR_TRY(rr::bayes_add_e2(F, h->b, p.seed, t, lam, tau, st));
    // the system at lambda / tau, solved from that b
    destroy_graph(h);
    RR_TRY(build_lambda(h, lam / tau));
    rr_info info{};
    result = h->opt.solver == RR_SOLVER_TLFCG ? solve_fcg_impl(h, nullptr, nullptr, nullptr, p.tol, &info)
                                             : solve_impl(h, nullptr, nullptr, p.tol, &info);
    if (result != RR_OK) break;
    if (iters) iters[t] = info.iters;
    if (w_mean && t >= burnin) RR_TRY(rr::bayes_accum(F, h->w_int, w_mean, st));
    // lambda | w, then tau | w
    RR_TRY(rr::dot_parts(F, h->w_int, h->w_int, h->part_rr, st));
    RR_TRY(rr::bayes_gamma(p.alpha + 0.5 * (double)F, p.beta, h->part_rr, rr::kVecGrid, p.seed,
                           kStreamGamma + 2 * (uint64_t)t, h->scal, st));
    if (draw_tau) {
      RR_TRY(matvec_f64(h, h->w_int, h->u, st));
      RR_TRY(rr::bayes_resid(N, y, h->u, h->bayes_y, st));
      RR_TRY(rr::dot_parts(N, h->bayes_y, h->bayes_y, h->part_rr, st));
      RR_TRY(rr::bayes_gamma(p.a_tau + 0.5 * (double)N, p.b_tau, h->part_rr, rr::kVecGrid, p.seed,
                             kStreamGamma + 2 * (uint64_t)t + 1, h->scal + 2, st));
    }
    RR_CUDA(cudaMemcpyAsync(h->scal_host, h->scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    if (h->scal_host[1] != 1.0 || (draw_tau && h->scal_host[3] != 1.0)) {
      rr_set_error("rr_bayes: no gamma draw accepted in 1000 attempts at sample %d", t);
      result = RR_NONFINITE;
      break;
    }
    lam = h->scal_host[0];
    if (draw_tau) tau = h->scal_host[2];
    if (!(lam > 0.0) || !isfinite(lam) || !(tau > 0.0) || !isfinite(tau)) {
      rr_set_error("rr_bayes: lambda or tau not positive and finite at sample %d", t);
      result = RR_NONFINITE;
      break;
    }
    if (lam_trace) lam_trace[t] = lam;
    if (tau_trace) tau_trace[t] = tau;
  }
  if (w_mean && n_samples > burnin)
    RR_TRY(rr::bayes_scale(F, 1.0 / (double)(n_samples - burnin), w_mean, st));
  return result;
}
}  // namespace

extern "C" {

void rr_default_options(rr_options *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->kmeans_max_iter = 50;
  o->max_iter = 20000;
  o->seed = 0;
  o->init_centers = nullptr;
  o->solver = RR_SOLVER_TWOLEVEL;
  o->precision = RR_PREC_FP64;
  o->check_every = 8;
  o->max_restarts = 5;
  o->use_graphs = 1;
  o->gram = RR_GRAM_AUTO;
  o->gather = RR_GATHER_AUTO;
  o->clustering = RR_CLUSTER_KMEANS;
  o->lf_tol2 = 1.0;
  o->stream = nullptr;
}

const char *rr_last_error(void) { return g_err; }

int64_t rr_launch_count(void) { return rr_launch_counter; }

rr_status rr_setup(const rr_matrix *X, double lambda, int32_t k, const rr_options *o,
                   rr_handle **out) {
  NvtxRange nvtx_range("rr_setup");
  g_err[0] = 0;
  if (!X || !out) {
    rr_set_error("rr_setup: X and out must not be NULL");
    return RR_INVALID_ARG;
  }
  *out = nullptr;
  if (X->layout != RR_CSR_BINARY && X->layout != RR_DENSE_F32_ROWMAJOR) {
    rr_set_error("rr_setup: unknown layout %d", X->layout);
    return RR_INVALID_ARG;
  }
  if (X->layout == RR_CSR_BINARY &&
      (X->n_rows < 1 || X->n_cols < 1 || X->nnz < 0 || !X->row_ptr || (X->nnz > 0 && !X->col_idx) ||
       X->values)) {
    rr_set_error("rr_setup: bad matrix description");
    return RR_INVALID_ARG;
  }
  if (X->layout == RR_DENSE_F32_ROWMAJOR &&
      (X->n_rows < 1 || X->n_cols < 1 || !X->values || X->row_ptr || X->col_idx)) {
    rr_set_error("rr_setup: a dense X needs values and no row_ptr / col_idx");
    return RR_INVALID_ARG;
  }
  if (!(lambda > 0.0) || !isfinite(lambda)) {
    rr_set_error("rr_setup: lambda must be positive and finite");
    return RR_INVALID_ARG;
  }
  if (k < 1 || k > X->n_cols) {
    rr_set_error("rr_setup: k must be in [1, F]");
    return RR_INVALID_ARG;
  }
  if ((X->layout == RR_CSR_BINARY && X->nnz >= (1LL << 31)) || X->n_rows >= (1LL << 31) ||
      X->n_cols >= (1LL << 31)) {
    rr_set_error("rr_setup: nnz (CSR), N and F must be below 2^31");
    return RR_UNSUPPORTED;
  }
  if (k > 16384) {
    rr_set_error("rr_setup: k above 16384 is not supported");
    return RR_UNSUPPORTED;
  }
  rr_options opt;
  if (o) opt = *o; else rr_default_options(&opt);
  if (opt.precision != RR_PREC_FP64 && opt.precision != RR_PREC_MIXED) {
    rr_set_error("rr_setup: unknown precision %d", opt.precision);
    return RR_INVALID_ARG;
  }
  if (opt.kmeans_max_iter < 1 || opt.max_iter < 1) {
    rr_set_error("rr_setup: kmeans_max_iter and max_iter must be positive");
    return RR_INVALID_ARG;
  }
  if (opt.gather < RR_GATHER_AUTO || opt.gather > RR_GATHER_LANES_STAGED) {
    rr_set_error("rr_setup: unknown gather %d", opt.gather);
    return RR_INVALID_ARG;
  }
  if (opt.coarse != RR_COARSE_CHOLESKY && opt.coarse != RR_COARSE_EIGEN) {
    rr_set_error("rr_setup: unknown coarse %d", opt.coarse);
    return RR_INVALID_ARG;
  }
  if (opt.solver < RR_SOLVER_TWOLEVEL || opt.solver > RR_SOLVER_TLFCG) {
    rr_set_error("rr_setup: unknown solver %d", opt.solver);
    return RR_INVALID_ARG;
  }
  if (opt.clustering != RR_CLUSTER_KMEANS && opt.clustering != RR_CLUSTER_LEADER) {
    rr_set_error("rr_setup: unknown clustering %d", opt.clustering);
    return RR_INVALID_ARG;
  }
  if (opt.clustering == RR_CLUSTER_LEADER &&
      (X->layout != RR_CSR_BINARY || opt.init_centers || !isfinite(opt.lf_tol2))) {
    rr_set_error("rr_setup: leader-follower clustering needs binary X, no init_centers and a "
                 "finite lf_tol2");
    return RR_INVALID_ARG;
  }
  rr_handle *h = new rr_handle();
  h->opt = opt;
  h->opt.init_centers = nullptr;
  h->st = static_cast<cudaStream_t>(opt.stream);
  const auto t0 = std::chrono::steady_clock::now();
  h->opt.init_centers = opt.init_centers;
  // the setup runs on a stream of the highest priority (after the caller's
  // stream's earlier work), so that its latency-bound k-means++ rounds go
  // first while the pattern build runs beside them at the lowest priority;
  // it is synchronised before rr_setup returns
  cudaStream_t user = h->st, hp = nullptr;
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
      cudaStreamCreateWithPriority(&hp, cudaStreamNonBlocking, greatest) == cudaSuccess) {
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ev, user) != cudaSuccess || cudaStreamWaitEvent(hp, ev, 0) != cudaSuccess) {
      cudaStreamDestroy(hp);
      hp = nullptr;
    } else {
      h->st = hp;
    }
    if (ev) cudaEventDestroy(ev);
  }
  cudaGetLastError();
  rr_status s = X->layout == RR_DENSE_F32_ROWMAJOR ? setup_impl_dense(h, X, lambda, k)
                                                   : setup_impl(h, X, lambda, k);
  h->opt.init_centers = nullptr;
  if (hp) {
    if (cudaStreamSynchronize(hp) != cudaSuccess && s == RR_OK) {
      rr_set_error("rr_setup: %s", cudaGetErrorString(cudaGetLastError()));
      s = RR_CUDA_ERROR;
    }
    h->st = user;
    cudaStreamDestroy(hp);
  }
  if (s == RR_OK && X->layout != RR_DENSE_F32_ROWMAJOR) s = start_coarse_factor(h, lambda);
  if (s != RR_OK) {
    rr_free(h);
    return s;
  }
  h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = h;
  return RR_OK;
}

rr_status rr_set_lambda(rr_handle *h, double lambda) {
  if (h) RR_TRY(wait_coarse_host(h));
  NvtxRange nvtx_range("rr_set_lambda");
  if (!h) {
    rr_set_error("rr_set_lambda: NULL handle");
    return RR_INVALID_ARG;
  }
  if (!(lambda > 0.0) || !isfinite(lambda)) {
    rr_set_error("rr_set_lambda: lambda must be positive and finite");
    return RR_INVALID_ARG;
  }
  destroy_graph(h);   // the captured kernels hold lambda and omega by value
  bool found = false;
  if (!h->mu) RR_TRY(install_prepared(h, lambda, &found));
  if (!found) RR_TRY(build_lambda(h, lambda));
  RR_CUDA(cudaStreamSynchronize(h->st));
  return RR_OK;
}

// A handle for another lambda that shares base's X-dependent setup (X and
// its transpose, the clustering, the coarse Gram, the operator's patterns) and
// owns what depends on lambda or is written while it solves: the coarse
// inverse, the smoother, the solve vectors and scalars, the operator's
// intermediate vectors, its error word and its own stream. d and omega are
// built first (omega is read back: the captured kernels take it by value);
// the coarse factor then runs on the fork's stream and is marked by an event,
// so that rr_solve_many starts the other problems at once.
rr_status fork_impl(rr_handle *base, double lambda, rr_handle *f) {
  DevArena &m = f->mem;
  cudaStream_t st = f->st;
  const int64_t F = f->F, k = f->k_eff;
  RR_TRY(m.alloc(&f->err, 1));
  RR_CUDA(cudaMemsetAsync(f->err, 0, sizeof(int32_t), st));
  RR_CUDA(cudaMallocHost(&f->err_host, sizeof(int32_t)));
  RR_TRY(alloc_solve_workspace(f));
  RR_TRY(m.alloc(&f->d, F));
  RR_TRY(m.alloc(&f->omega_dev, 1));
  RR_TRY(m.alloc(&f->max_bits, 1));
  RR_TRY(m.alloc(&f->Ac, k * k));
  if (f->mu) {
    RR_TRY(m.alloc(&f->dvec, k));
    RR_TRY(m.alloc(&f->ec_tmp, k));
  } else {
    RR_TRY(m.alloc(&f->Lw, k * k));
    RR_TRY(m.alloc(&f->Linv, k * k));
    RR_TRY(m.alloc(&f->Ainv, k * k));
    if (base->Ainv32) RR_TRY(m.alloc(&f->Ainv32, k * ((k + 3) & ~(int64_t)3)));
  }
  // the operator's intermediate vectors
  auto own_pattern = [&](rr::SlicedPattern &P) -> rr_status {
    if (!P.idx) return RR_OK;
    double *xq = nullptr, *psum = nullptr;
    RR_TRY(m.alloc(&xq, std::max<int64_t>(1, P.n_inner)));
    RR_TRY(m.alloc(&psum, std::max<int64_t>(1, P.npieces)));
    P.xq = xq;
    P.psum = psum;
    P.err = f->err;
    return RR_OK;
  };
  RR_TRY(own_pattern(f->pcsr));
  RR_TRY(own_pattern(f->pcsc));
  if (f->split.active) {
    float *zp = nullptr, *up = nullptr;
    RR_TRY(m.alloc(&zp, (int64_t)f->split.nblk * f->split.H));
    RR_TRY(m.alloc(&up, std::max<int32_t>(1, f->split.nblk)));
    f->split.zpart = zp;
    f->split.upart = up;
    RR_TRY(m.alloc(&f->split.wd, F));
    RR_TRY(own_pattern(f->split.xt));
    RR_TRY(own_pattern(f->split.xtt));
  }
  if (f->rplan.k > 0) {
    RR_TRY(m.alloc(&f->rplan.item_sum, std::max<int32_t>(1, f->rplan.n_items)));
    RR_TRY(m.alloc(&f->rplan.rc, std::max<int32_t>(1, f->rplan.k)));
  }
  // the smoother at lambda, omega read back
  RR_CUDA(cudaMemsetAsync(f->max_bits, 0, sizeof(unsigned long long), st));
  RR_LAUNCH(k_jacobi_setup, rr::grid_for(F, kThreads), kThreads, 0, st, F, lambda, f->col_ptr,
            f->gsum, f->d, f->max_bits);
  RR_LAUNCH(k_omega, 1, 32, 0, st, f->max_bits, f->omega_dev);
  double om = 0.0;
  RR_CUDA(cudaMemcpyAsync(&om, f->omega_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  f->omega = om;
  f->lambda = lambda;
  RR_TRY(rr::split_set_wd(f->split, f->omega, f->d, st));
  // the coarse level, left running
  RR_TRY(rr::coarse_operator((int32_t)k, f->G, f->s, lambda, f->Ac, st));
  if (f->mu) {
    RR_TRY(rr::eig_dvec((int32_t)k, f->mu, lambda, f->dvec, st));
  } else {
    RR_CUDA(cudaMemcpyAsync(f->Lw, f->Ac, sizeof(double) * (size_t)k * k, cudaMemcpyDeviceToDevice, st));
    RR_TRY(rr::cholesky((int32_t)k, f->Lw, f->Linv, f->err, st));
    RR_TRY(rr::chol_inverse((int32_t)k, f->Lw, f->Linv, f->Ainv, st));
    if (f->Ainv32) RR_TRY(rr::coarse_to_f32((int32_t)k, f->Ainv, f->Ainv32, st));
  }
  RR_CUDA(cudaEventCreateWithFlags(&f->ready, cudaEventDisableTiming));
  RR_CUDA(cudaEventRecord(f->ready, st));
  return RR_OK;
}

rr_status rr_fork_lambda(rr_handle *base, double lambda, rr_handle **out) {
  NvtxRange nvtx_range("rr_fork_lambda");
  if (!base || !out) {
    rr_set_error("rr_fork_lambda: NULL argument");
    return RR_INVALID_ARG;
  }
  *out = nullptr;
  if (!(lambda > 0.0) || !isfinite(lambda)) {
    rr_set_error("rr_fork_lambda: lambda must be positive and finite");
    return RR_INVALID_ARG;
  }
  if (base->dense || base->fork_of) {
    rr_set_error("rr_fork_lambda: forks of dense-X handles or of forks are not supported");
    return RR_UNSUPPORTED;
  }
  RR_CUDA(cudaStreamSynchronize(base->st));
  rr_handle *f = new rr_handle(*base);
  // nothing of base's is owned by the fork: every owned field starts empty
  f->mem.ptrs.clear();
  f->fork_of = base;
  f->ready = nullptr;
  f->fst = nullptr;
  f->st = nullptr;
  f->cap_stream = nullptr;
  f->loop_graph = nullptr;
  f->loop_exec = nullptr;
  f->limit_host = nullptr;
  f->body_kernels = 0;
  f->S = f->S_host = nullptr;
  f->scal_host = nullptr;
  f->err = f->err_host = nullptr;
  f->batch = nullptr;
  f->bayes_y = nullptr;
  for (auto &P : f->prep) P = rr_handle::Prepared{};
  f->prep_st = nullptr;
  f->prep_Ac = f->prep_Lw = f->prep_Linv = nullptr;
  f->bplan = rr::RestrictPlan{};
  f->p_prev = f->q_prev = f->part_zq = f->part3 = nullptr;
  f->Sf = f->Sf_host = nullptr;
  f->tz = f->tr = f->tp = f->tq = f->tzz = nullptr;
  f->t_rz = f->t_pq = f->t_rr = nullptr;
  f->St = nullptr;
  f->fcg_cache = nullptr;
  f->Lw = f->Linv = f->Ainv = nullptr;
  f->Ainv32 = nullptr;
  f->dvec = f->ec_tmp = nullptr;
  if (cudaStreamCreateWithFlags(&f->st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    f->st = nullptr;
    rr_free(f);
    rr_set_error("rr_fork_lambda: cudaStreamCreate failed");
    return RR_CUDA_ERROR;
  }
  const rr_status s = fork_impl(base, lambda, f);
  if (s != RR_OK) {
    rr_free(f);
    return s;
  }
  *out = f;
  return RR_OK;
}

rr_status rr_prepare_lambdas(rr_handle *h, const double *lambdas, int32_t n) {
  if (h) RR_TRY(wait_coarse_host(h));
  NvtxRange nvtx_range("rr_prepare_lambdas");
  if (!h || (n > 0 && !lambdas) || n < 0 || n > rr_handle::kPrepared) {
    rr_set_error("rr_prepare_lambdas: need a handle and 0 <= n <= %d lambdas",
                 rr_handle::kPrepared);
    return RR_INVALID_ARG;
  }
  for (int32_t i = 0; i < n; ++i)
    if (!(lambdas[i] > 0.0) || !isfinite(lambdas[i])) {
      rr_set_error("rr_prepare_lambdas: every lambda must be positive and finite");
      return RR_INVALID_ARG;
    }
  if (h->fork_of) {
    rr_set_error("rr_prepare_lambdas: not supported on a handle from rr_fork_lambda");
    return RR_UNSUPPORTED;
  }
  if (h->mu || n == 0) return RR_OK;   // the eigen form's lambda change is one vector rescale
  const int64_t kk = (int64_t)h->k_eff * h->k_eff;
  if (!h->prep_st) {
    RR_CUDA(cudaStreamCreateWithFlags(&h->prep_st, cudaStreamNonBlocking));
    RR_TRY(h->mem.alloc(&h->prep_Ac, kk));
    RR_TRY(h->mem.alloc(&h->prep_Lw, kk));
    RR_TRY(h->mem.alloc(&h->prep_Linv, kk));
  }
  // the previous preparations' buffers are reused: let them finish first
  RR_CUDA(cudaStreamSynchronize(h->prep_st));
  for (auto &P : h->prep) P.valid = false;
  for (int32_t i = 0; i < n; ++i) RR_TRY(prepare_one(h, h->prep[i], lambdas[i]));
  return RR_OK;
}

rr_status rr_solve(rr_handle *h, const double *y, double *w, double tol, rr_info *info) {
  NvtxRange nvtx_range("rr_solve");
  if (!h || !y || !w) {
    rr_set_error("rr_solve: handle, y and w must not be NULL");
    return RR_INVALID_ARG;
  }
  if (!(tol > 0.0 && tol < 1.0)) {
    rr_set_error("rr_solve: tol must be in (0, 1)");
    return RR_INVALID_ARG;
  }
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t l0 = rr_launch_counter;
  RR_TRY(wait_coarse(h, h->st));
  rr_status s = h->opt.solver == RR_SOLVER_TLFCG ? solve_fcg_impl(h, nullptr, y, w, tol, info)
                                                 : solve_impl(h, y, w, tol, info);
  if (s == RR_OK || s == RR_NOT_CONVERGED) {
    const rr_status e = check_dev_error(h, "rr_solve");
    if (e != RR_OK) s = e;
  }
  if (info) {
    info->fallbacks = 0;
    info->k_eff = h->k_eff;
    info->kmeans_iters = h->kmeans_iters;
    info->omega = h->omega;
    info->setup_ms = h->setup_ms;
    info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    info->launches = rr_launch_counter - l0;
    info->gram_tensor_cores = h->gram_on_tensor_cores ? 1 : 0;
    info->gather_staged = (h->pcsr.staged ? 1 : 0) | (h->pcsc.staged ? 2 : 0);
    for (int i = 0; i < 8; ++i) info->setup_phase_ms[i] = h->phase_ms[i];
  }
  return s;
}

rr_status rr_solve_fcg(rr_handle *h, const rr_mlp *net, const double *y, double *w, double tol,
                       rr_info *info) {
  if (h) RR_TRY(wait_coarse(h, h->st));
  NvtxRange nvtx_range("rr_solve_fcg");
  if (!h || !y || !w) {
    rr_set_error("rr_solve_fcg: handle, y and w must not be NULL");
    return RR_INVALID_ARG;
  }
  if (!(tol > 0.0 && tol < 1.0)) {
    rr_set_error("rr_solve_fcg: tol must be in (0, 1)");
    return RR_INVALID_ARG;
  }
  if (h->opt.solver != RR_SOLVER_TWOLEVEL) {
    rr_set_error("rr_solve_fcg: the handle's solver must be RR_SOLVER_TWOLEVEL");
    return RR_UNSUPPORTED;
  }
  if (net && rr::mlp_k(net) != h->k_eff) {
    rr_set_error("rr_solve_fcg: the network's k (%d) differs from k_eff (%d)", rr::mlp_k(net),
                 h->k_eff);
    return RR_INVALID_ARG;
  }
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t l0 = rr_launch_counter;
  if (info) memset(info, 0, sizeof(*info));
  rr_status s = solve_fcg_impl(h, net, y, w, tol, info);
  if (s == RR_OK || s == RR_NOT_CONVERGED) {
    const rr_status e = check_dev_error(h, "rr_solve_fcg");
    if (e != RR_OK) s = e;
  }
  if (info) {
    info->k_eff = h->k_eff;
    info->kmeans_iters = h->kmeans_iters;
    info->omega = h->omega;
    info->setup_ms = h->setup_ms;
    info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    info->launches = rr_launch_counter - l0;
    info->gram_tensor_cores = h->gram_on_tensor_cores ? 1 : 0;
    info->gather_staged = (h->pcsr.staged ? 1 : 0) | (h->pcsc.staged ? 2 : 0);
    for (int i = 0; i < 8; ++i) info->setup_phase_ms[i] = h->phase_ms[i];
  }
  return s;
}

rr_status rr_solve_many(int32_t nprob, rr_handle *const *hs, const double *const *ys,
                        double *const *ws, double tol, void *stream, rr_info *infos) {
  NvtxRange nvtx_range("rr_solve_many");
  if (nprob < 1 || !hs || !ys || !ws || !(tol > 0.0 && tol < 1.0)) {
    rr_set_error("rr_solve_many: nprob < 1, NULL arrays or tol not in (0, 1)");
    return RR_INVALID_ARG;
  }
  for (int32_t i = 0; i < nprob; ++i) {
    if (!hs[i] || !ys[i] || !ws[i]) {
      rr_set_error("rr_solve_many: NULL handle, target or solution of problem %d", i);
      return RR_INVALID_ARG;
    }
    for (int32_t j = 0; j < i; ++j)
      if (hs[j] == hs[i]) {
        rr_set_error("rr_solve_many: problems %d and %d share a handle", j, i);
        return RR_INVALID_ARG;
      }
    if (hs[i]->opt.solver == RR_SOLVER_TLFCG) {
      rr_set_error("rr_solve_many: problem %d uses RR_SOLVER_TLFCG (PCG solvers only)", i);
      return RR_UNSUPPORTED;
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t l0 = rr_launch_counter;
  // every problem's work is issued on `stream` for the duration of the call
  // (every handle's own stream is drained before any handle is switched, so
  // that an error return leaves all handles on their own streams)
  // (a fork's coarse factor may still run on its stream: the fork's branch of
  // the graph waits on its event instead, so the other problems start at once)
  for (int32_t i = 0; i < nprob; ++i)
    if (!hs[i]->fork_of || !hs[i]->ready) RR_CUDA(cudaStreamSynchronize(hs[i]->st));
  std::vector<cudaStream_t> saved(nprob);
  for (int32_t i = 0; i < nprob; ++i) {
    saved[i] = hs[i]->st;
    hs[i]->st = st;
  }
  if (infos) memset(infos, 0, sizeof(rr_info) * nprob);
  const rr_status s = solve_many_impl(nprob, hs, ys, ws, tol, st, infos);
  cudaStreamSynchronize(st);
  for (int32_t i = 0; i < nprob; ++i) hs[i]->st = saved[i];
  if (infos) {
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (int32_t i = 0; i < nprob; ++i) {
      infos[i].solve_ms = ms;
      infos[i].launches = rr_launch_counter - l0;
    }
  }
  return s;
}

rr_status rr_apply(rr_handle *h, const double *v, double *out) {
  if (!h || !v || !out || v == out) {
    rr_set_error("rr_apply: NULL argument, or v and out alias");
    return RR_INVALID_ARG;
  }
  rr::CscEpilogue ep{rr::CSC_APPLY, h->lambda, h->omega, v, nullptr, nullptr, out, nullptr, nullptr};
  RR_TRY(op_apply(h, v, ep, nullptr, h->st, h->opt.precision == RR_PREC_MIXED));
  return RR_OK;
}

rr_status rr_precondition(rr_handle *h, const double *r, double *z) {
  if (!h || !r || !z || r == z) {
    rr_set_error("rr_precondition: NULL argument, or r and z alias");
    return RR_INVALID_ARG;
  }
  int n = 0;
  RR_TRY(wait_coarse(h, h->st));
  RR_TRY(apply_precond(h, r, z, nullptr, &n, false, h->st));
  return RR_OK;
}

rr_status rr_rhs(rr_handle *h, const double *y, double *b) {
  if (!h || !y || !b) {
    rr_set_error("rr_rhs: NULL argument");
    return RR_INVALID_ARG;
  }
  rr::CscEpilogue ep{rr::CSC_RHS, 0.0, 0.0, nullptr, nullptr, nullptr, b, nullptr, nullptr};
  if (h->dense)
    return rr::dense_transposed(h->N, h->F, h->Xd, y, h->dpart, ep,
                                h->opt.precision == RR_PREC_MIXED, h->st);
  RR_TRY(rr::sliced_gather(h->pcsc, y, nullptr, nullptr, h->st, h->opt.precision == RR_PREC_MIXED));
  RR_TRY(rr::sliced_epilogue(h->pcsc, ep, h->st));
  return RR_OK;
}

rr_status rr_matvec(rr_handle *h, const double *v, double *u) {
  if (!h || !v || !u) {
    rr_set_error("rr_matvec: NULL argument");
    return RR_INVALID_ARG;
  }
  if (h->dense)
    return rr::dense_matvec(h->N, h->F, h->Xd, v, u, nullptr, h->opt.precision == RR_PREC_MIXED,
                            h->st);
  RR_TRY(rr::sliced_gather(h->pcsr, v, nullptr, nullptr, h->st, h->opt.precision == RR_PREC_MIXED));
  RR_TRY(rr::sliced_slot_sum(h->pcsr, u, h->st));
  return RR_OK;
}

rr_status rr_get_labels(const rr_handle *h, int32_t *labels_host) {
  if (!h || !labels_host) {
    rr_set_error("rr_get_labels: NULL argument");
    return RR_INVALID_ARG;
  }
  RR_CUDA(cudaMemcpyAsync(labels_host, h->labels, sizeof(int32_t) * h->F, cudaMemcpyDeviceToHost, h->st));
  RR_CUDA(cudaStreamSynchronize(h->st));
  return RR_OK;
}

rr_status rr_get_centers(const rr_handle *h, int32_t *centers_host) {
  if (!h || !centers_host) {
    rr_set_error("rr_get_centers: NULL argument");
    return RR_INVALID_ARG;
  }
  RR_CUDA(cudaMemcpyAsync(centers_host, h->centers, sizeof(int32_t) * h->k_req, cudaMemcpyDeviceToHost, h->st));
  RR_CUDA(cudaStreamSynchronize(h->st));
  return RR_OK;
}

rr_status rr_get_coarse(const rr_handle *h, double *Ac_host, int64_t *G_host) {
  if (!h) {
    rr_set_error("rr_get_coarse: NULL handle");
    return RR_INVALID_ARG;
  }
  RR_TRY(wait_coarse_host(h));
  if (h->dense && G_host) {
    rr_set_error("rr_get_coarse: the integer Gram exists for binary X only");
    return RR_UNSUPPORTED;
  }
  const size_t kk = (size_t)h->k_eff * h->k_eff;
  if (Ac_host)
    RR_CUDA(cudaMemcpyAsync(Ac_host, h->Ac, sizeof(double) * kk, cudaMemcpyDeviceToHost, h->st));
  std::vector<double> g;
  if (G_host) {
    g.resize(kk);
    RR_CUDA(cudaMemcpyAsync(g.data(), h->G, sizeof(double) * kk, cudaMemcpyDeviceToHost, h->st));
  }
  RR_CUDA(cudaStreamSynchronize(h->st));
  if (G_host)
    for (size_t i = 0; i < kk; ++i) G_host[i] = (int64_t)g[i];
  return RR_OK;
}

rr_status rr_bayes(rr_handle *h, const double *y, const rr_bayes_params *p, int32_t n_samples,
                   int32_t burnin, double *w_mean, double *lam_trace, double *tau_trace,
                   int32_t *iters) {
  if (h && h->fork_of) {
    rr_set_error("rr_bayes: not supported on a handle from rr_fork_lambda");
    return RR_UNSUPPORTED;
  }
  if (h) RR_TRY(wait_coarse_host(h));
  NvtxRange nvtx_range("rr_bayes");
  if (!h || !y || !p) {
    rr_set_error("rr_bayes: handle, y and params must not be NULL");
    return RR_INVALID_ARG;
  }
  if (n_samples < 1 || burnin < 0 || burnin >= n_samples) {
    rr_set_error("rr_bayes: need n_samples >= 1 and 0 <= burnin < n_samples");
    return RR_INVALID_ARG;
  }
  const bool ok = p->alpha > 0.0 && isfinite(p->alpha) && p->beta >= 0.0 && isfinite(p->beta) &&
                  p->alpha + 0.5 * (double)h->F >= 1.0 && p->lambda0 > 0.0 &&
                  isfinite(p->lambda0) && p->tau0 > 0.0 && isfinite(p->tau0) && p->tol > 0.0 &&
                  p->tol < 1.0 && isfinite(p->a_tau) &&
                  (p->a_tau <= 0.0 || (p->b_tau >= 0.0 && isfinite(p->b_tau) &&
                                       p->a_tau + 0.5 * (double)h->N >= 1.0));
  if (!ok) {
    rr_set_error("rr_bayes: parameters out of range (alpha > 0, beta >= 0, lambda0, tau0 > 0, "
                 "tol in (0, 1), b_tau >= 0 when a_tau > 0)");
    return RR_INVALID_ARG;
  }
  const double lam_keep = h->lambda;
  rr_status s = bayes_impl(h, y, *p, n_samples, burnin, w_mean, lam_trace, tau_trace, iters);
  // the handle's own lambda back
  destroy_graph(h);
  const rr_status s2 = build_lambda(h, lam_keep);
  if (s == RR_OK) s = s2;
  const cudaError_t ce = cudaStreamSynchronize(h->st);
  if (ce != cudaSuccess && s == RR_OK) {
    rr_set_error("rr_bayes: %s", cudaGetErrorString(ce));
    s = RR_CUDA_ERROR;
  }
  if (s == RR_OK || s == RR_NOT_CONVERGED || s == RR_NONFINITE) {
    const rr_status e = check_dev_error(h, "rr_bayes");
    if (e != RR_OK) s = e;
  }
  return s;
}

rr_status rr_get_eigen(const rr_handle *h, double *mu_host, double *Q_host, int32_t *sweeps) {
  if (!h || !h->mu) {
    rr_set_error("rr_get_eigen: NULL handle or a handle without the eigen coarse solve");
    return RR_INVALID_ARG;
  }
  const int32_t k = h->k_eff;
  if (mu_host)
    RR_CUDA(cudaMemcpyAsync(mu_host, h->mu, sizeof(double) * k, cudaMemcpyDeviceToHost, h->st));
  if (Q_host) {   // Q[i][e] = component i of eigenvector e (the rows of Qv transposed)
    std::vector<double> v((size_t)k * k);
    RR_CUDA(cudaMemcpyAsync(v.data(), h->Qv, sizeof(double) * v.size(), cudaMemcpyDeviceToHost, h->st));
    RR_CUDA(cudaStreamSynchronize(h->st));
    for (int64_t e = 0; e < k; ++e)
      for (int64_t i = 0; i < k; ++i) Q_host[i * k + e] = v[e * k + i];
  }
  RR_CUDA(cudaStreamSynchronize(h->st));
  if (sweeps) *sweeps = h->eig_sweeps;
  return RR_OK;
}

rr_status rr_query(const rr_handle *h, int64_t *n_rows, int64_t *n_cols, int32_t *k_eff,
                   double *omega, double *lambda) {
  if (!h) {
    rr_set_error("rr_query: NULL handle");
    return RR_INVALID_ARG;
  }
  if (n_rows) *n_rows = h->N;
  if (n_cols) *n_cols = h->F;
  if (k_eff) *k_eff = h->k_eff;
  if (omega) *omega = h->omega;
  if (lambda) *lambda = h->lambda;
  return RR_OK;
}

void rr_free(rr_handle *h) {
  if (!h) return;
  if (h->fork_of) {   // its own allocations, streams, events and pinned words only
    if (h->st) cudaStreamSynchronize(h->st);
    destroy_graph(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->limit_host) cudaFreeHost(h->limit_host);
    if (h->ready) cudaEventDestroy(h->ready);
    h->mem.free_all();
    if (h->err_host) cudaFreeHost(h->err_host);
    if (h->S_host) cudaFreeHost(h->S_host);
    if (h->scal_host) cudaFreeHost(h->scal_host);
    if (h->Sf_host) cudaFreeHost(h->Sf_host);
    if (h->st) cudaStreamDestroy(h->st);
    delete h;
    return;
  }
  cudaStreamSynchronize(h->st);
  if (h->fst) {
    cudaStreamSynchronize(h->fst);
    cudaStreamDestroy(h->fst);
  }
  if (h->ready) cudaEventDestroy(h->ready);
  destroy_graph(h);
  rr::batch_free(h->batch);
  h->batch = nullptr;
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->limit_host) cudaFreeHost(h->limit_host);
  if (h->prep_st) {
    cudaStreamSynchronize(h->prep_st);
    cudaStreamDestroy(h->prep_st);
  }
  for (auto &P : h->prep)
    if (P.done) cudaEventDestroy(P.done);
  rr::restrict_free(h->rplan);
  rr::restrict_free(h->bplan);
  rr::sliced_free(h->pcsr);
  rr::sliced_free(h->pcsc);
  rr::split_free(h->split);
  h->mem.free_all();
  if (h->err_host) cudaFreeHost(h->err_host);
  if (h->S_host) cudaFreeHost(h->S_host);
  if (h->scal_host) cudaFreeHost(h->scal_host);
  if (h->Sf_host) cudaFreeHost(h->Sf_host);
  delete h;
}

}  // extern "C"
