// Flexible CG, Algorithm 3 with m = 1 (Notay's FCG(1)): the new direction is
// the preconditioned residual A-orthogonalised against the previous direction,
//   p_i = z_i - (<z_i, A p_{i-1}> / <p_{i-1}, A p_{i-1}>) p_{i-1}   (p_0 = z_0),
//   alpha_i = <p_i, r_i> / <p_i, A p_i>,  w += alpha p,  r -= alpha A p,
// which stays a valid Krylov method when the preconditioner changes between
// steps (here: the learned coarse correction). The learned variant checks each
// step before it is taken and redoes it with the Cholesky coarse solve when
// <r, z> <= 0, when z or alpha is not finite, or when the step would not
// reduce ||r||_2, the predicted ||r - alpha q||^2 = ||r||^2 - 2 alpha <r, q> +
// alpha^2 ||q||^2 being computed in FP64 from the same partial sums.
// Scalars are fixed-order sums of per-block partials (repeatable bits).
#include "common.cuh"
#include "kernels.h"

namespace rr {

namespace {

__device__ __forceinline__ bool stopped(const int32_t *stop) { return stop && *stop; }

// partial <a, b> per block (kVecGrid blocks)
__global__ void k_fcg_dot(int64_t F, const double *__restrict__ a, const double *__restrict__ b,
                          double *__restrict__ part, const int32_t *__restrict__ stop) {
  pdl_wait();
  if (stopped(stop)) return;
  __shared__ double sm[kWarps + 1];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += a[i] * b[i];
  const double t = block_sum(acc, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// p = z - beta p_prev, beta = <z, q_prev> / <p_prev, q_prev> (p = z on a (re)start).
__global__ void k_fcg_direction(int64_t F, const double *__restrict__ part_zq, int n,
                                const FcgScalars *__restrict__ S, const double *__restrict__ z,
                                const double *__restrict__ p_prev, double *__restrict__ p,
                                const int32_t *__restrict__ stop) {
  pdl_wait();
  if (stopped(stop)) return;
  __shared__ double sm[kWarps + 1];
  const bool first = S->first;
  const double beta = first ? 0.0 : sum_partials(part_zq, n, sm) / S->pq_prev;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = first ? z[i] : z[i] - beta * p_prev[i];
}

// partials of <p, r>, <r, q>, <q, q> into part3[0..n), [n..2n), [2n..3n).
__global__ void k_fcg_dots(int64_t F, const double *__restrict__ p, const double *__restrict__ r,
                           const double *__restrict__ q, double *__restrict__ part3, int n,
                           const int32_t *__restrict__ stop) {
  pdl_wait();
  if (stopped(stop)) return;
  __shared__ double sm[kWarps + 1];
  double pr = 0.0, rq = 0.0, qq = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double qi = q[i], ri = r[i];
    pr += p[i] * ri;
    rq += ri * qi;
    qq += qi * qi;
  }
  pr = block_sum(pr, sm);
  rq = block_sum(rq, sm);
  qq = block_sum(qq, sm);
  if (threadIdx.x == 0) {
    part3[blockIdx.x] = pr;
    part3[n + blockIdx.x] = rq;
    part3[2 * n + blockIdx.x] = qq;
  }
}

// One block: decides whether the learned step is redone with the Cholesky
// coarse solve (skip_fb = 0) or kept (skip_fb = 1).
__global__ void k_fcg_decide(const double *__restrict__ part_rz, const double *__restrict__ part_pq,
                             const double *__restrict__ part3, int n, FcgScalars *S) {
  pdl_wait();
  __shared__ double sm[kWarps + 1];
  if (S->converged) {
    if (threadIdx.x == 0) S->skip_fb = 1;
    return;
  }
  const double rz = sum_partials(part_rz, n, sm);
  const double pq = sum_partials(part_pq, n, sm);
  const double pr = sum_partials(part3, n, sm);
  const double rq = sum_partials(part3 + n, n, sm);
  const double qq = sum_partials(part3 + 2 * n, n, sm);
  if (threadIdx.x == 0) {
    const double alpha = pr / pq;
    const double pred = S->rr - 2.0 * alpha * rq + alpha * alpha * qq;
    const bool fb = S->learned && (!(rz > 0.0) || !isfinite(rz) || !isfinite(alpha) ||
                                   !(pred < S->rr));
    S->skip_fb = fb ? 0 : 1;
    if (fb) S->fallbacks += 1;
  }
}

// w += alpha p; r -= alpha q; z1 = omega D^-1 r (next pre-smoothing);
// p_prev = p; q_prev = q; partial ||r||^2.
__global__ void k_fcg_update(int64_t F, const double *__restrict__ part_pq,
                             const double *__restrict__ part3, int n, const double *__restrict__ p,
                             const double *__restrict__ q, double *__restrict__ w,
                             double *__restrict__ r, double omega, const double *__restrict__ d,
                             double *__restrict__ z1, double *__restrict__ p_prev,
                             double *__restrict__ q_prev, double *__restrict__ part_rr,
                             const FcgScalars *__restrict__ S) {
  pdl_wait();
  if (S->converged) return;
  __shared__ double sm[kWarps + 1];
  const double pq = sum_partials(part_pq, n, sm);
  const double pr = sum_partials(part3, n, sm);
  const double alpha = pr / pq;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double pi = p[i], qi = q[i];
    w[i] += alpha * pi;
    const double ri = r[i] - alpha * qi;
    r[i] = ri;
    acc += ri * ri;
    z1[i] = omega * ri / d[i];
    p_prev[i] = pi;
    q_prev[i] = qi;
  }
  const double t = block_sum(acc, sm);
  if (threadIdx.x == 0) part_rr[blockIdx.x] = t;
}

__global__ void k_fcg_finish(const double *__restrict__ part_rr, const double *__restrict__ part_pq,
                             int n, FcgScalars *S, double *__restrict__ history, int32_t hist_cap) {
  pdl_wait();
  if (S->converged) return;
  __shared__ double sm[kWarps + 1];
  const double rr = sum_partials(part_rr, n, sm);
  const double pq = sum_partials(part_pq, n, sm);
  if (threadIdx.x == 0) {
    S->rr = rr;
    S->pq_prev = pq;
    S->first = 0;
    S->skip_fb = 1;
    const int32_t it = S->iter + 1;
    S->iter = it;
    const double rn = sqrt(rr);
    if (history && it <= hist_cap) history[it - 1] = rn / S->bnorm;
    if (!isfinite(rr) || !isfinite(pq)) {
      S->nonfinite = 1;
      S->converged = 1;
    } else if (rn <= S->target) {
      S->converged = 1;
    }
  }
}

__global__ void k_fcg_start(const double *__restrict__ bb_part, const double *__restrict__ rr_part,
                            int n, double tol, int32_t set_bnorm, int32_t learned, FcgScalars *S) {
  pdl_wait();
  __shared__ double sm[kWarps + 1];
  const double bb = sum_partials(bb_part, n, sm);
  const double rr = sum_partials(rr_part, n, sm);
  if (threadIdx.x == 0) {
    if (set_bnorm) {
      S->bnorm = sqrt(bb);
      S->target = tol * S->bnorm;
      S->iter = 0;
      S->fallbacks = 0;
      S->nonfinite = isfinite(bb) ? 0 : 1;
    }
    S->learned = learned;
    S->rr = rr;
    S->pq_prev = 0.0;
    S->first = 1;
    S->skip_fb = 1;
    S->converged = (S->nonfinite || sqrt(rr) <= S->target) ? 1 : 0;
  }
}

__global__ void k_fcg_condition(cudaGraphConditionalHandle hc, const FcgScalars *__restrict__ S) {
  pdl_wait();
  if (threadIdx.x == 0)
    cudaGraphSetConditional(hc, (!S->converged && S->iter < S->limit) ? 1u : 0u);
}

}  // namespace

rr_status fcg_dot(int64_t F, const double *a, const double *b, double *part, const int32_t *stop,
                  cudaStream_t st) {
  RR_LAUNCH_PDL(k_fcg_dot, kVecGrid, kThreads, 0, st, F, a, b, part, stop);
  return RR_OK;
}

rr_status fcg_direction(int64_t F, const double *part_zq, const FcgScalars *S, const double *z,
                        const double *p_prev, double *p, const int32_t *stop, cudaStream_t st) {
  RR_LAUNCH_PDL(k_fcg_direction, kVecGrid, kThreads, 0, st, F, part_zq, kVecGrid, S, z, p_prev, p, stop);
  return RR_OK;
}

rr_status fcg_dots(int64_t F, const double *p, const double *r, const double *q, double *part3,
                   const int32_t *stop, cudaStream_t st) {
  RR_LAUNCH_PDL(k_fcg_dots, kVecGrid, kThreads, 0, st, F, p, r, q, part3, kVecGrid, stop);
  return RR_OK;
}

rr_status fcg_decide(const double *part_rz, const double *part_pq, const double *part3,
                     FcgScalars *S, cudaStream_t st) {
  RR_LAUNCH_PDL(k_fcg_decide, 1, kThreads, 0, st, part_rz, part_pq, part3, kVecGrid, S);
  return RR_OK;
}

rr_status fcg_update(int64_t F, const double *part_pq, const double *part3, const double *p,
                     const double *q, double *w, double *r, double omega, const double *d,
                     double *z1, double *p_prev, double *q_prev, double *part_rr,
                     const FcgScalars *S, cudaStream_t st) {
  RR_LAUNCH_PDL(k_fcg_update, kVecGrid, kThreads, 0, st, F, part_pq, part3, kVecGrid, p, q, w, r, omega,
            d, z1, p_prev, q_prev, part_rr, S);
  return RR_OK;
}

rr_status fcg_finish(const double *part_rr, const double *part_pq, FcgScalars *S, double *history,
                     int32_t hist_cap, cudaStream_t st) {
  RR_LAUNCH_PDL(k_fcg_finish, 1, kThreads, 0, st, part_rr, part_pq, kVecGrid, S, history, hist_cap);
  return RR_OK;
}

rr_status fcg_start(const double *bb_part, int n_bb, const double *rr_part, double tol,
                    int32_t set_bnorm, int32_t learned, FcgScalars *S, cudaStream_t st) {
  (void)n_bb;
  RR_LAUNCH_PDL(k_fcg_start, 1, kThreads, 0, st, bb_part, rr_part, kVecGrid, tol, set_bnorm, learned, S);
  return RR_OK;
}

rr_status fcg_condition(cudaGraphConditionalHandle hc, const FcgScalars *S, cudaStream_t st) {
  RR_LAUNCH_PDL(k_fcg_condition, 1, 32, 0, st, hc, S);
  return RR_OK;
}

}  // namespace rr
