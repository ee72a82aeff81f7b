"""Oracle: Krylov solvers for (X^T X + lambda I) w = X^T y.

Test infrastructure only.

  CG / DCG    Section 4, Table 2: CG, and CG with the diagonal (Jacobi)
              preconditioner.
  PCG         preconditioned CG with a fixed SPD preconditioner (the
              two-level cycle), x_0 = 0, r_0 = b (Algorithm 3's initialisation).
  FCG(m)      Algorithm 3 (flexible CG): p_i = z_i - sum over the last m_i
              directions of <z_i, A p_k>/<p_k, A p_k> p_k, truncation
              m_0 = 0, m_i = max(1, i mod (m+1)).
  stopping    ||r_i||_2 <= tol ||b||_2 on the recurrence residual (the
              residual plotted in Section 4's figures), followed by a check
              of the true residual b - A w; while that is above tol the
              correction equation is solved again from zero (refinement).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Result:
    w: np.ndarray
    iters: int
    rel_res: float          # recurrence residual / ||b||
    true_rel_res: float     # ||b - A w|| / ||b||
    history: list           # recurrence ||r_i|| / ||b|| after every iteration
    restarts: int = 0
    snapshots: dict = dataclasses.field(default_factory=dict)   # tol -> first iterate below it


def _snap(snaps, pending, w, rel):
    """Copies w for every pending tolerance the recurrence residual has reached."""
    for t in [t for t in pending if rel <= t]:
        snaps[t] = w.copy()
        pending.remove(t)


def _pcg_core(A, Minv, b, target, max_iter, history, bnorm, snap=None):
    """snap: optional (snapshots, pending tolerances, offset w0): the iterate
    w0 + x is recorded at the first iteration whose recurrence residual is
    below each pending tolerance times ||b||."""
    x = np.zeros_like(b)
    r = b.copy()
    if np.linalg.norm(r) <= target:
        return x, r, 0
    z = Minv(r)
    p = z.copy()
    rho = r @ z
    for it in range(1, max_iter + 1):
        q = A(p)
        alpha = rho / (p @ q)
        x += alpha * p
        r -= alpha * q
        rn = np.linalg.norm(r)
        history.append(rn / bnorm)
        if snap is not None and snap[1]:
            _snap(snap[0], snap[1], snap[2] + x, rn / bnorm)
        if rn <= target:
            return x, r, it
        z = Minv(r)
        rho_new = r @ z
        p = z + (rho_new / rho) * p
        rho = rho_new
    return x, r, max_iter


def pcg(A, Minv, b, tol=1e-8, max_iter=10000, max_restarts=5, snap_tols=()):
    """PCG with the stopping rule and true-residual refinement above.
    snap_tols: looser tolerances at which the iterate is also recorded
    (Result.snapshots), at the first iteration whose recurrence residual
    reaches each: the iterate a solve to that tolerance stops at, when that
    solve needs no refinement restart."""
    b = np.asarray(b, np.float64)
    bnorm = float(np.linalg.norm(b))
    hist = []
    if bnorm == 0.0:
        return Result(np.zeros_like(b), 0, 0.0, 0.0, hist)
    target = tol * bnorm
    snaps, pending = {}, [t for t in snap_tols if t > tol]
    w, r, its = _pcg_core(A, Minv, b, target, max_iter, hist, bnorm,
                          (snaps, pending, np.zeros_like(b)))
    rel = float(np.linalg.norm(r)) / bnorm
    true_r = b - A(w)
    restarts = 0
    while np.linalg.norm(true_r) > target and restarts < max_restarts and its < max_iter:
        restarts += 1
        dw, r, more = _pcg_core(A, Minv, true_r, target, max_iter - its, hist, bnorm,
                                (snaps, pending, w))
        its += more
        w = w + dw
        rel = float(np.linalg.norm(r)) / bnorm
        true_r = b - A(w)
    return Result(w, its, rel, float(np.linalg.norm(true_r)) / bnorm, hist, restarts, snaps)


def cg(A, b, **kw):
    """Unpreconditioned CG (Table 2's CG)."""
    return pcg(A, lambda r: r.copy(), b, **kw)


def dcg(A, d, b, **kw):
    """Diagonally preconditioned CG (Table 2's DCG), d = diag(A)."""
    return pcg(A, lambda r: r / d, b, **kw)


def fcg(A, Minv, b, m=1, tol=1e-8, max_iter=10000, on_step=None):
    """Flexible CG, Algorithm 3. Minv(r, i) may change with i (or be non-linear).
    on_step(i, r, z) may return a replacement z (used for the learned-correction
    fallback). Returns Result (no refinement restarts)."""
    b = np.asarray(b, np.float64)
    bnorm = float(np.linalg.norm(b))
    x = np.zeros_like(b)
    r = b.copy()
    hist = []
    if bnorm == 0.0:
        return Result(x, 0, 0.0, 0.0, hist)
    P, AP, PAP = [], [], []
    it = 0
    while it < max_iter and np.linalg.norm(r) > tol * bnorm:
        z = Minv(r, it)
        if on_step is not None:
            z2 = on_step(it, r, z)
            if z2 is not None:
                z = z2
        m_i = 0 if it == 0 else max(1, it % (m + 1))
        p = z.copy()
        for k in range(max(0, len(P) - m_i), len(P)):
            p -= (z @ AP[k]) / PAP[k] * P[k]
        q = A(p)
        pq = p @ q
        alpha = (p @ r) / pq
        x += alpha * p
        r -= alpha * q
        P.append(p); AP.append(q); PAP.append(pq)
        if len(P) > m + 1:
            P.pop(0); AP.pop(0); PAP.pop(0)
        it += 1
        hist.append(float(np.linalg.norm(r)) / bnorm)
    true_r = b - A(x)
    return Result(x, it, float(np.linalg.norm(r)) / bnorm,
                  float(np.linalg.norm(true_r)) / bnorm, hist)
