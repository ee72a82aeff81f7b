"""Oracle: Bayesian ridge regression by Gibbs sampling with noise injection.

Test infrastructure only.

Section 2 (Bayesian regression): with the likelihood y ~ N(X w, tau^-1 I_N)
and the prior w ~ N(0, lambda^-1 I_F), lambda ~ Gamma(alpha, beta) (shape,
rate), a sample of w given lambda and tau is the solution of

    (X^T X + (lambda / tau) I) w = X^T (y + e1) + e2 / tau,
    e1 ~ N(0, tau^-1 I_N),  e2 ~ N(0, lambda I_F)              (Eq. ni_xtx)

(its mean is (X^T X + (lambda/tau) I)^-1 X^T y and its covariance
(tau X^T X + lambda I)^-1, the conditional posterior of w). The Gibbs sampler
alternates it with the conjugate updates

    lambda | w ~ Gamma(alpha + F / 2, beta + ||w||^2 / 2),
    tau | w    ~ Gamma(a_tau + N / 2, b_tau + ||y - X w||^2 / 2)

(tau fixed when a_tau <= 0), so lambda / tau, the regularisation of the
system, changes at every step: the paper's case for a coarse solve that is
reused across lambda (Section 4; eigen.py). Each system is solved by the
two-level PCG of twolevel.py / krylov.py.

Random draws (the same definition on the GPU, implemented there on its own):
  uniforms U(seed, stream, i) and normals Z(seed, stream, i) are those of
  gen.synth (SplitMix64 on (seed, stream, index); Box-Muller with the
  uniforms i and 2^40 + i). Step t draws e1 from stream 2 t (N normals,
  times tau^-1/2) and e2 from stream 2 t + 1 (F normals, times lambda^1/2).
  Gamma(a, rate) by Marsaglia & Tsang (2000, "A simple method for generating
  gamma variables", a >= 1): d = a - 1/3, c = 1 / sqrt(9 d); attempt j draws
  x from the uniforms 2 j, 2 j + 1 of the stream (x = sqrt(-2 ln(1 - U))
  cos(2 pi U')) and u = U(2^32 + j); it accepts when v = (1 + c x)^3 > 0 and
  ln u < x^2 / 2 + d - d v + d ln v, returning d v / rate. lambda of step t
  uses stream 2^20 + 2 t, tau stream 2^20 + 2 t + 1.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from gen import synth

from . import krylov
from . import sparse as osp

STREAM_GAMMA = 1 << 20


@dataclasses.dataclass
class Params:
    alpha: float = 1.0      # lambda ~ Gamma(alpha, beta)
    beta: float = 1.0
    a_tau: float = 1.0      # tau ~ Gamma(a_tau, b_tau); a_tau <= 0: tau fixed at tau0
    b_tau: float = 1.0
    lambda0: float = 1.0
    tau0: float = 1.0
    seed: int = 0
    tol: float = 1e-8


def gamma_draw(a, rate, seed, stream):
    """Gamma(shape a >= 1, rate) by Marsaglia & Tsang on the counter-based draws."""
    d = a - 1.0 / 3.0
    c = 1.0 / math.sqrt(9.0 * d)
    for j in range(1000):
        u1, u2 = synth.uniform(seed, stream, 2, 2 * j)
        x = math.sqrt(-2.0 * math.log(1.0 - u1)) * math.cos(2.0 * math.pi * u2)
        t = 1.0 + c * x
        v = t * t * t
        if v <= 0.0:
            continue
        u = synth.uniform(seed, stream, 1, (1 << 32) + j)[0]
        if math.log(u) < 0.5 * x * x + d - d * v + d * math.log(v):
            return d * v / rate
    raise RuntimeError("gamma_draw: no acceptance in 1000 attempts")


def noise_sample(two, y, lam, tau, seed, step, tol, max_iter=100000):
    """One w given lambda and tau: the noise-injected system of Eq. (ni_xtx),
    solved by the oracle's two-level PCG at lambda / tau."""
    M = two.M
    N, F = M.shape
    e1 = synth.normal(seed, 2 * step, N) / math.sqrt(tau)
    e2 = synth.normal(seed, 2 * step + 1, F) * math.sqrt(lam)
    b = osp.rhs(M, y + e1) + e2 / tau
    t = two.with_lambda(lam / tau)
    return krylov.pcg(t.A, t.apply, b, tol=tol, max_iter=max_iter, max_restarts=20)


def gibbs(two, y, p: Params, n_samples, burnin=0):
    """The chain: (lambda trace, tau trace, mean of w over the samples after
    burnin, iterations of each solve). two: a two-level setup (its clustering
    is reused at every lambda / tau)."""
    M = two.M
    N, F = M.shape
    lam, tau = p.lambda0, p.tau0
    lams, taus, iters = [], [], []
    wsum = np.zeros(F)
    for t in range(n_samples):
        res = noise_sample(two, y, lam, tau, p.seed, t, p.tol)
        w = res.w
        iters.append(res.iters)
        if t >= burnin:
            wsum += w
        lam = gamma_draw(p.alpha + 0.5 * F, p.beta + 0.5 * float(w @ w), p.seed,
                         STREAM_GAMMA + 2 * t)
        if p.a_tau > 0.0:
            r = y - osp.X_mv(M, w)
            tau = gamma_draw(p.a_tau + 0.5 * N, p.b_tau + 0.5 * float(r @ r), p.seed,
                             STREAM_GAMMA + 2 * t + 1)
        lams.append(lam)
        taus.append(tau)
    return np.array(lams), np.array(taus), wsum / max(1, n_samples - burnin), iters
