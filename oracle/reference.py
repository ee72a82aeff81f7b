"""Oracle: exact solutions of Eq. (1) for large binary workloads, several at once.

Test infrastructure only (the solution-parity checks of the tests at full
size and the error figures that the benchmark reports beside its timings).

The solution w = (X^T X + lambda I)^-1 X^T y is unique, so it is computed by
the oracle's own two-level PCG (twolevel.py, krylov.py) run to relative
residual 1e-12, far below the 1e-8 being checked; the iterate at which that
run first reaches each looser tolerance is recorded too (the oracle's own
answer at that tolerance). Independent systems run in separate processes
(started with "spawn", so that a parent holding a GPU context is safe); each
process rebuilds X from the seeded generator and the preconditioner from the
oracle's cluster labels, which it is given.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

TOL_REF = 1e-12


def _solve_one(job):
    from gen import synth
    from . import kmeans as km
    from . import krylov, twolevel
    from . import sparse as osp
    km.set_threads(1)
    spec, lam, y, raw_labels, snap_tols = job
    X = synth.zipf_binary(*spec)
    ref = twolevel.from_labels(X.n_rows, X.n_cols, X.row_ptr, X.col_idx, lam, raw_labels)
    b = osp.rhs(ref.M, y)
    res = krylov.pcg(ref.A, ref.apply, b, tol=TOL_REF, max_iter=100000, max_restarts=20,
                     snap_tols=snap_tols)
    return res.w, res.snapshots, res.iters, res.true_rel_res


def oracle_labels(spec, k, seed, kmeans_max_iter=50, threads=0):
    """The oracle's k-means++ centres, Lloyd labels (raw, before compaction)
    and Lloyd step count for the Zipf workload spec = (N, F, density, s, seed
    of X)."""
    from gen import synth
    from . import kmeans as km
    from . import sparse as osp
    X = synth.zipf_binary(*spec)
    cp, ri = osp.csc_pattern(X.n_rows, X.n_cols, X.row_ptr, X.col_idx)
    centers = km.kmeanspp_binary(X.n_rows, X.n_cols, X.row_ptr, X.col_idx, cp, ri, k, seed)
    km.set_threads(threads)
    labels, iters = km.lloyd_binary(X.n_rows, X.n_cols, X.row_ptr, X.col_idx, cp, ri, centers,
                                    kmeans_max_iter)
    return centers, labels, iters


def exact_solutions(spec, raw_labels, jobs, snap_tols=(1e-8,), processes=None):
    """For each (lambda, y) in jobs: (w_ref, {tol: oracle iterate}, iterations,
    true relative residual), computed in parallel processes."""
    n = processes or max(1, min(len(jobs), (os.cpu_count() or 2) - 1))
    work = [(tuple(spec), float(lam), np.ascontiguousarray(y, np.float64), raw_labels,
             tuple(snap_tols)) for lam, y in jobs]
    if n == 1:
        return [_solve_one(j) for j in work]
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(_solve_one, work)


def start(spec, raw_labels, jobs, snap_tols=(1e-8,), processes=None):
    """exact_solutions started in the background: returns (pool, AsyncResult);
    call .get() on the result, then pool.close()."""
    n = processes or max(1, min(len(jobs), (os.cpu_count() or 2) - 1))
    work = [(tuple(spec), float(lam), np.ascontiguousarray(y, np.float64), raw_labels,
             tuple(snap_tols)) for lam, y in jobs]
    pool = mp.get_context("spawn").Pool(n)
    return pool, pool.map_async(_solve_one, work)
