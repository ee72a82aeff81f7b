// Bayesian ridge regression by Gibbs sampling with noise injection (Section
// 2, Eq. (ni_xtx)): the device side of rr_bayes. Each step solves
//
//   (X^T X + (lambda / tau) I) w = X^T (y + e1) + e2 / tau,
//   e1 ~ N(0, tau^-1 I_N),  e2 ~ N(0, lambda I_F),
//
// then draws lambda | w ~ Gamma(alpha + F/2, beta + ||w||^2 / 2) and
// tau | w ~ Gamma(a_tau + N/2, b_tau + ||y - X w||^2 / 2).
//
// The random draws come from a counter-based generator, SplitMix64 (Steele,
// Lea & Flood, OOPSLA 2014) evaluated on (seed, stream, index): uniform
// U = (x >> 11) 2^-53 of output index + 1 of the stream whose base is
// mix(mix(seed) xor stream * 0xD1B54A32D192ED03); normal i of a stream by
// Box-Muller from the uniforms i and 2^40 + i. Step t takes e1 from stream
// 2 t and e2 from stream 2 t + 1; Gamma(a, rate) by Marsaglia & Tsang (2000)
// on stream 2^20 + 2 t (lambda) or 2^20 + 2 t + 1 (tau), attempt j drawing
// x from the uniforms 2 j and 2 j + 1 and u = U(2^32 + j).
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace rr {

namespace {

__device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t sm_base(uint64_t seed, uint64_t stream) {
  return sm_mix(sm_mix(seed) ^ (stream * 0xD1B54A32D192ED03ULL));
}

__device__ __forceinline__ double sm_uniform(uint64_t base, uint64_t i) {
  return (double)(sm_mix(base + (i + 1) * 0x9E3779B97F4A7C15ULL) >> 11) * 0x1.0p-53;
}

__device__ __forceinline__ double sm_normal(uint64_t base, uint64_t i) {
  const double u1 = 1.0 - sm_uniform(base, i);
  const double u2 = sm_uniform(base, (1ULL << 40) + i);
  return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

// yt = y + e1, e1 = tau^-1/2 Z(seed, 2 t, i)
__global__ void k_bayes_noise_y(int64_t N, const double *__restrict__ y, uint64_t seed,
                                int64_t step, double tau, double *__restrict__ yt) {
  const uint64_t base = sm_base(seed, (uint64_t)(2 * step));
  const double s = 1.0 / sqrt(tau);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    yt[i] = y[i] + sm_normal(base, (uint64_t)i) * s;
}

// b += e2 / tau, e2 = lambda^1/2 Z(seed, 2 t + 1, j)
__global__ void k_bayes_add_e2(int64_t F, double *__restrict__ b, uint64_t seed, int64_t step,
                               double lam, double tau) {
  const uint64_t base = sm_base(seed, (uint64_t)(2 * step + 1));
  const double s = sqrt(lam);
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < F;
       j += (int64_t)gridDim.x * blockDim.x)
    b[j] += sm_normal(base, (uint64_t)j) * s / tau;
}

// r = y - u
__global__ void k_bayes_resid(int64_t N, const double *__restrict__ y, const double *__restrict__ u,
                              double *__restrict__ r) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    r[i] = y[i] - u[i];
}

// out[0] = Gamma(a, rate0 + ss / 2) with ss the fixed-order sum of the
// partials; out[1] = 1 if an attempt was accepted (one thread)
__global__ void k_bayes_gamma(double a, double rate0, const double *__restrict__ part, int n_part,
                              uint64_t seed, uint64_t stream, double *__restrict__ out) {
  __shared__ double sm[kWarps + 1];
  const double ss = sum_partials(part, n_part, sm);
  if (threadIdx.x != 0) return;
  const double rate = rate0 + 0.5 * ss;
  const uint64_t base = sm_base(seed, stream);
  const double d = a - 1.0 / 3.0;
  const double c = 1.0 / sqrt(9.0 * d);
  out[1] = 0.0;
  for (uint64_t j = 0; j < 1000; ++j) {
    const double u1 = sm_uniform(base, 2 * j), u2 = sm_uniform(base, 2 * j + 1);
    const double x = sqrt(-2.0 * log(1.0 - u1)) * cos(2.0 * M_PI * u2);
    // separately rounded products and sums (no fused multiply-add), in the
    // order the definition writes them
    const double t = __dadd_rn(1.0, __dmul_rn(c, x));
    const double v = __dmul_rn(__dmul_rn(t, t), t);
    if (v <= 0.0) continue;
    const double u = sm_uniform(base, (1ULL << 32) + j);
    const double rhs = __dadd_rn(__dsub_rn(__dadd_rn(__dmul_rn(__dmul_rn(0.5, x), x), d),
                                           __dmul_rn(d, v)),
                                 __dmul_rn(d, log(v)));
    if (log(u) < rhs) {
      out[0] = __dmul_rn(d, v) / rate;
      out[1] = 1.0;
      return;
    }
  }
}

__global__ void k_bayes_accum(int64_t F, const double *__restrict__ w, double *__restrict__ acc) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < F;
       j += (int64_t)gridDim.x * blockDim.x)
    acc[j] += w[j];
}

__global__ void k_bayes_scale(int64_t F, double s, double *__restrict__ v) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < F;
       j += (int64_t)gridDim.x * blockDim.x)
    v[j] *= s;
}

}  // namespace

rr_status bayes_noise_y(int64_t N, const double *y, uint64_t seed, int64_t step, double tau,
                        double *yt, cudaStream_t st) {
  RR_LAUNCH(k_bayes_noise_y, grid_for(N, kThreads), kThreads, 0, st, N, y, seed, step, tau, yt);
  return RR_OK;
}

rr_status bayes_add_e2(int64_t F, double *b, uint64_t seed, int64_t step, double lam, double tau,
                       cudaStream_t st) {
  RR_LAUNCH(k_bayes_add_e2, grid_for(F, kThreads), kThreads, 0, st, F, b, seed, step, lam, tau);
  return RR_OK;
}

rr_status bayes_resid(int64_t N, const double *y, const double *u, double *r, cudaStream_t st) {
  RR_LAUNCH(k_bayes_resid, grid_for(N, kThreads), kThreads, 0, st, N, y, u, r);
  return RR_OK;
}

rr_status bayes_gamma(double a, double rate0, const double *part, int n_part, uint64_t seed,
                      uint64_t stream, double *out, cudaStream_t st) {
  RR_LAUNCH(k_bayes_gamma, 1, kThreads, 0, st, a, rate0, part, n_part, seed, stream, out);
  return RR_OK;
}

rr_status bayes_accum(int64_t F, const double *w, double *acc, cudaStream_t st) {
  RR_LAUNCH(k_bayes_accum, grid_for(F, kThreads), kThreads, 0, st, F, w, acc);
  return RR_OK;
}

rr_status bayes_scale(int64_t F, double s, double *v, cudaStream_t st) {
  RR_LAUNCH(k_bayes_scale, grid_for(F, kThreads), kThreads, 0, st, F, s, v);
  return RR_OK;
}

}  // namespace rr
