"""Oracle: training pairs of the learned coarse correction, in FP64.

Test infrastructure only. The paper has no learned component; this is the
plain definition the CUDA path's rr_harvest follows. Two-level PCG (the
symmetric cycle of Section 3.1 as preconditioner, x_0 = 0, r_0 = b as in
Algorithm 3's initialisation) runs on (X^T X + lambda I) w = b; at every
iteration i, inside the preconditioner application to r_i,
    z1 = omega D^-1 r_i                    (pre-smoothing)
    r1 = r_i - A z1
    x_i = P^T r1                           (the restricted residual: the network's input)
    t_i = P^T (e_i - z1),  e_i = w_ref - w_i  (the remaining error, restricted: the target)
so that A (e_i - z1) = r1: t_i is what an exact coarse correction of the
remaining error would carry on the coarse space (P t_i = P P^T (e_i - z1),
its orthogonal projection, since P^T P = I).
"""
from __future__ import annotations

import numpy as np

from oracle import twolevel


def harvest_pairs(tl: twolevel.TwoLevel, b, w_ref, n_iter):
    """(X, T, history): the pairs of the first n_iter PCG iterations (fewer if
    the iteration reaches r = 0)."""
    b = np.asarray(b, np.float64)
    w = np.zeros_like(b)
    r = b.copy()
    xs, ts = [], []
    p = None
    rho_old = None
    for _ in range(n_iter):
        # the preconditioner application, step by step
        z1 = tl.omega * r / tl.d
        r1 = r - tl.A(z1)
        xs.append(twolevel.restrict(tl.labels, tl.s, r1))
        ts.append(twolevel.restrict(tl.labels, tl.s, (w_ref - w) - z1))
        e_c = twolevel.chol_solve(tl.L, xs[-1])
        z2 = z1 + twolevel.prolong(tl.labels, tl.s, e_c)
        r2 = r - tl.A(z2)
        z = z2 + tl.omega * r2 / tl.d
        # CG recurrences
        rho = r @ z
        p = z.copy() if p is None else z + (rho / rho_old) * p
        q = tl.A(p)
        alpha = rho / (p @ q)
        w = w + alpha * p
        r = r - alpha * q
        rho_old = rho
        if not np.any(r):
            break
    return np.array(xs), np.array(ts)
