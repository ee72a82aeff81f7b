"""Pins of the FP64 oracle to facts the paper and the mathematics fix.

CPU only. Each test names the passage it checks. None of them re-types the
oracle's formula: they compare against closed forms, library routines
(numpy.linalg), brute force with exact rationals, or invariants.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from gen import synth
from oracle import kmeans as km
from oracle import krylov, mlp
from oracle import sparse as osp
from oracle import twolevel as tl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def csr_of(dense):
    dense = np.asarray(dense)
    rows, cols = np.nonzero(dense)
    row_ptr = np.zeros(dense.shape[0] + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=dense.shape[0]), out=row_ptr[1:])
    return dense.shape[0], dense.shape[1], row_ptr, cols.astype(np.int32)


def random_binary(n, f, p, seed):
    rng = np.random.default_rng(seed)
    return (rng.random((n, f)) < p).astype(np.int64)


# ---------------------------------------------------------------- generator / RNG

def test_splitmix64_published_output():
    g = json.load(open(os.path.join(GOLDEN, "splitmix64.json")))
    for t, hx in enumerate(g["outputs_hex"]):
        assert km.splitmix64(g["seed"], t) == int(hx, 16)


def test_generator_zipf_shape():
    X = synth.zipf_binary(2000, 1000, 0.01, 1.1, seed=0)
    assert X.row_ptr[0] == 0 and np.all(np.diff(X.row_ptr) >= 0)
    assert X.col_idx.min() >= 0 and X.col_idx.max() < 1000
    # expected nnz = density * N * F, within a few standard deviations
    assert abs(X.nnz - 20000) < 1500
    counts = np.sort(np.bincount(X.col_idx, minlength=1000))[::-1]
    q = synth.zipf_column_probs(1000, 0.01, 1.1)
    # the heaviest columns follow the power law of their rank
    assert abs(counts[0] - q[0] * 2000) < 5 * math.sqrt(2000) + 1
    assert counts[:10].sum() > counts[500:].sum() / 10


# ---------------------------------------------------------------- operator / CSC

def test_csc_is_stable_transpose():
    D = random_binary(30, 17, 0.3, 1)
    n, f, rp, ci = csr_of(D)
    cp, ri = osp.csc_pattern(n, f, rp, ci)
    for j in range(f):
        rows = ri[cp[j]:cp[j + 1]]
        assert np.array_equal(rows, np.nonzero(D[:, j])[0])


def test_apply_A_matches_dense():
    D = random_binary(40, 25, 0.2, 2)
    M = osp.from_csr(*csr_of(D))
    v = np.random.default_rng(0).standard_normal(25)
    ref = (D.T @ D + 0.3 * np.eye(25)) @ v
    assert np.allclose(osp.apply_A(M, 0.3, v), ref, rtol=1e-14, atol=1e-12)


# ---------------------------------------------------------------- closed forms (Eq. 1, Eq. rr)

def test_single_feature_closed_form():
    """One feature: w = x^T y / (x^T x + lambda) (Eq. rr with F = 1)."""
    x = np.array([1, 0, 1, 1, 0, 1])[:, None]
    y = np.array([0.5, -1.0, 2.0, 0.25, 3.0, -0.75])
    lam = 0.37
    M = osp.from_csr(*csr_of(x))
    b = osp.rhs(M, y)
    w_exact = (x[:, 0] @ y) / (x[:, 0] @ x[:, 0] + lam)
    A = lambda v: osp.apply_A(M, lam, v)
    assert abs(krylov.cg(A, b, tol=1e-14).w[0] - w_exact) < 1e-14
    two = tl.setup_binary(*csr_of(x), lam, 1)
    assert abs(krylov.pcg(two.A, two.apply, b, tol=1e-14).w[0] - w_exact) < 1e-14


def test_disjoint_supports_diagonal_system():
    """Disjoint column supports make X^T X diagonal: DCG finishes in one step
    and w_i = x_i^T y / (n_i + lambda)."""
    D = np.zeros((9, 3), np.int64)
    D[0:2, 0] = 1
    D[2:7, 1] = 1
    D[7:9, 2] = 1
    y = np.arange(1.0, 10.0)
    lam = 0.5
    M = osp.from_csr(*csr_of(D))
    A = lambda v: osp.apply_A(M, lam, v)
    b = osp.rhs(M, y)
    d = osp.col_sq_norms(M) + lam
    res = krylov.dcg(A, d, b, tol=1e-14)
    assert res.iters == 1
    expect = np.array([y[0:2].sum() / 2.5, y[2:7].sum() / 5.5, y[7:9].sum() / 2.5])
    assert np.allclose(res.w, expect, rtol=1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_solvers_agree_with_dense_solve(seed):
    """CG, DCG and two-level PCG reach the solution of Eq. (1) given by a dense solve."""
    D = random_binary(60, 40, 0.15, seed)
    D[:, 5] = D[:, 3]                      # a duplicated feature
    lam = 0.05
    n, f, rp, ci = csr_of(D)
    y = np.random.default_rng(seed).standard_normal(n)
    two = tl.setup_binary(n, f, rp, ci, lam, 8, seed=seed)
    b = osp.rhs(two.M, y)
    w_ref = np.linalg.solve(D.T @ D + lam * np.eye(f), D.T @ y)
    for res in (krylov.cg(two.A, b, tol=1e-13), krylov.dcg(two.A, two.d, b, tol=1e-13),
                krylov.pcg(two.A, two.apply, b, tol=1e-13)):
        assert np.linalg.norm(res.w - w_ref) / np.linalg.norm(w_ref) < 1e-10
        assert res.true_rel_res <= 1e-13


# ---------------------------------------------------------------- Cholesky (Section 4, LAPACK's role)

def test_cholesky_against_library():
    rng = np.random.default_rng(3)
    B = rng.standard_normal((30, 30))
    A = B @ B.T + 0.1 * np.eye(30)
    L = tl.cholesky(A)
    assert np.allclose(L, np.linalg.cholesky(A), rtol=1e-12, atol=1e-12)
    assert np.allclose(np.triu(L, 1), 0.0)
    b = rng.standard_normal(30)
    assert np.allclose(tl.chol_solve(L, b), np.linalg.solve(A, b), rtol=1e-10)
    with pytest.raises(tl.NotSPD):
        tl.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))


# ---------------------------------------------------------------- P and the coarse operator (Section 3.2)

def test_prolongation_orthonormal_and_averaging():
    labels = np.array([0, 1, 0, 2, 1, 0, 2, 2, 2], np.int32)
    n_S = np.bincount(labels).astype(np.int64)
    P = tl.prolongation_dense(labels, tl.prolong_scale(n_S))
    assert np.allclose(P.T @ P, np.eye(3), atol=1e-15)
    Pa = tl.averaging_dense(labels, n_S)
    # the averaging operator gives diag(1/n_S), not a projection
    assert np.allclose(Pa.T @ Pa, np.diag(1.0 / n_S), atol=1e-15)
    r = np.arange(9.0)
    assert np.allclose(tl.restrict(labels, tl.prolong_scale(n_S), r), P.T @ r)
    e = np.array([1.0, -2.0, 0.5])
    assert np.allclose(tl.prolong(labels, tl.prolong_scale(n_S), e), P @ e)


@pytest.mark.parametrize("seed", [0, 4])
def test_galerkin_coarse_operator(seed):
    """A_c built from the exact integer Gram equals P^T A P formed densely."""
    D = random_binary(50, 30, 0.2, seed)
    lam = 0.01
    n, f, rp, ci = csr_of(D)
    two = tl.setup_binary(n, f, rp, ci, lam, 6, seed=seed)
    P = tl.prolongation_dense(two.labels, two.s)
    ref = P.T @ (D.T @ D + lam * np.eye(f)) @ P
    assert np.allclose(two.Ac, ref, rtol=1e-13, atol=1e-13)
    # the coarse regularisation equals the fine one because P^T P = I
    X = D.astype(float)
    assert np.allclose(tl.coarse_operator_dense(X, two.labels, two.s, lam), ref, rtol=1e-13)


def test_theorem1_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "theorem1_example.json")))
    base = np.array(g["x"], np.int64)
    X, groups = synth.duplicated_features(base, g["counts"])
    lam = 1e-3
    n, f, rp, ci = csr_of(X)
    two = tl.setup_binary(n, f, rp, ci, lam, 2, centers=[0, 2])
    assert np.array_equal(two.labels, groups)
    ev = np.linalg.eigvalsh(two.Ac) - lam
    assert np.allclose(ev, g["eigenvalues"], rtol=1e-14)


@pytest.mark.parametrize("seed", [0, 1])
def test_theorem1_random_duplicates(seed):
    """Theorem 1: on duplicated features the non-zero spectrum of X^T X equals
    that of P^T X^T X P, and its eigenvectors are constant within clusters,
    so P P^T leaves them unchanged."""
    rng = np.random.default_rng(seed)
    base = (rng.random((40, 6)) < 0.4).astype(np.int64)
    base[0] = 1                              # no all-zero columns
    counts = [3, 1, 4, 2, 5, 2]
    X, groups = synth.duplicated_features(base, counts)
    perm = rng.permutation(X.shape[1])
    X, groups = X[:, perm], groups[perm]
    centers = [int(np.nonzero(groups == g)[0][0]) for g in range(6)]
    n, f, rp, ci = csr_of(X)
    two = tl.setup_binary(n, f, rp, ci, 1e-6, 6, centers=centers)
    ev_c = np.sort(np.linalg.eigvalsh(two.Ac) - 1e-6)
    ev, V = np.linalg.eigh((X.T @ X).astype(float))
    nz = ev > 1e-9 * ev.max()
    assert nz.sum() == np.linalg.matrix_rank(base)
    assert np.allclose(np.sort(ev[nz]), ev_c[ev_c > 1e-9 * ev.max()], rtol=1e-10)
    P = tl.prolongation_dense(two.labels, two.s)
    assert np.allclose(P @ (P.T @ V[:, nz]), V[:, nz], atol=1e-10)


# ---------------------------------------------------------------- the cycle (Section 3.1)

def _tiny_two_level(seed=0, lam=0.02, k=7):
    D = random_binary(45, 28, 0.18, seed)
    n, f, rp, ci = csr_of(D)
    two = tl.setup_binary(n, f, rp, ci, lam, k, seed=seed)
    A = D.T @ D + lam * np.eye(f)
    return two, A


def _dense_of(fn, f):
    return np.stack([fn(e) for e in np.eye(f)], axis=1)


def test_coarse_correction_exact_on_coarse_space():
    """The coarse-grid correction reproduces any error in range(P) exactly."""
    two, A = _tiny_two_level()
    P = tl.prolongation_dense(two.labels, two.s)
    e_c = np.random.default_rng(1).standard_normal(two.k_eff)
    e = P @ e_c
    back = P @ two.coarse_correction(A @ e)
    assert np.linalg.norm(back - e) <= 1e-12 * np.linalg.norm(e)


def test_cycle_error_propagation_is_T():
    """I - M^{-1} A equals T = (I - S A)(I - P A_c^{-1} P^T A)(I - S A)."""
    two, A = _tiny_two_level(seed=2)
    f = A.shape[0]
    P = tl.prolongation_dense(two.labels, two.s)
    S = two.omega * np.diag(1.0 / two.d)
    I = np.eye(f)
    T = (I - S @ A) @ (I - P @ np.linalg.solve(P.T @ A @ P, P.T @ A)) @ (I - S @ A)
    Minv = _dense_of(two.apply, f)
    assert np.allclose(I - Minv @ A, T, atol=1e-10)


@pytest.mark.parametrize("seed", [0, 3, 5])
def test_preconditioner_spd(seed):
    two, A = _tiny_two_level(seed=seed)
    f = A.shape[0]
    Minv = _dense_of(two.apply, f)
    assert np.linalg.norm(Minv - Minv.T) <= 1e-12 * np.linalg.norm(Minv)
    assert np.linalg.eigvalsh(0.5 * (Minv + Minv.T)).min() > 0.0
    np.linalg.cholesky(0.5 * (Minv + Minv.T))


def test_omega_below_spectral_bound():
    """w lambda_max(D^{-1} A) <= 1, so 2 D/w - A is SPD (smoother convergent in the A-norm)."""
    two, A = _tiny_two_level(seed=6)
    Dm = np.diag(1.0 / np.sqrt(two.d))
    lmax = np.linalg.eigvalsh(Dm @ A @ Dm).max()
    assert two.omega * lmax <= 1.0 + 1e-12
    assert np.linalg.eigvalsh(2.0 / two.omega * np.diag(two.d) - A).min() > 0.0


def test_two_level_fewer_iterations_than_cg_and_dcg():
    """Section 4: the two-level method needs fewer iterations than CG and DCG."""
    X, y, _, p = synth.workload("zipf_2000x1000")
    two = tl.setup_binary(X.n_rows, X.n_cols, X.row_ptr, X.col_idx, 1e-2, 50, seed=0)
    b = osp.rhs(two.M, y)
    it_two = krylov.pcg(two.A, two.apply, b, tol=1e-8).iters
    assert it_two < krylov.dcg(two.A, two.d, b, tol=1e-8).iters
    assert it_two < krylov.cg(two.A, b, tol=1e-8).iters


# ---------------------------------------------------------------- FCG (Algorithm 3)

def test_fcg_matches_pcg_for_fixed_spd_preconditioner():
    """With a fixed SPD preconditioner, FCG(1) and PCG generate the same iterates."""
    two, A = _tiny_two_level(seed=7, lam=0.1)
    b = A @ np.random.default_rng(7).standard_normal(A.shape[0])
    Aop = lambda v: A @ v
    r1 = krylov.pcg(Aop, two.apply, b, tol=1e-10)
    r2 = krylov.fcg(Aop, lambda r, i: two.apply(r), b, m=1, tol=1e-10)
    n = min(len(r1.history), len(r2.history))
    assert abs(r1.iters - r2.iters) <= 1
    h1, h2 = np.array(r1.history[:n]), np.array(r2.history[:n])
    early = h1 > 1e-3          # before rounding differences are amplified
    assert early.sum() >= 4
    assert np.allclose(h1[early], h2[early], rtol=1e-6)
    w = np.linalg.solve(A, b)
    assert np.linalg.norm(r2.w - w) < 1e-8 * np.linalg.norm(w)


def test_rougher_is_two_step_krylov_minimiser():
    """Two CG steps from zero give the element of span{r, A r} that minimises
    the A-norm of the error: z* = V (V^T A V)^-1 V^T r, V = [r, A r]; the
    TLFCG cycle then adds the coarse correction of r - A z*."""
    two, A = _tiny_two_level(seed=8)
    r = np.random.default_rng(3).standard_normal(A.shape[0])
    V = np.stack([r, A @ r], axis=1)
    zstar = V @ np.linalg.solve(V.T @ A @ V, V.T @ r)
    P = tl.prolongation_dense(two.labels, two.s)
    want = zstar + P @ np.linalg.solve(P.T @ A @ P, P.T @ (r - A @ zstar))
    got = two.apply_tlfcg(r)
    assert np.allclose(got, want, rtol=1e-9, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("seed", [0, 1])
def test_tlfcg_reaches_dense_solution(seed):
    """FCG(1) with the rougher cycle solves Eq. (1): the same w as a dense
    solve, in fewer iterations than plain CG (Table 2's claim for TLFCG)."""
    rng = np.random.default_rng(20 + seed)
    D = (rng.random((300, 120)) < 0.05).astype(np.int64)
    n, f, rp, ci = csr_of(D)
    two = tl.setup_binary(n, f, rp, ci, 1e-2, 12, seed=seed)
    y = rng.standard_normal(n)
    b = osp.rhs(two.M, y)
    res = krylov.fcg(two.A, lambda r, i: two.apply_tlfcg(r), b, m=1, tol=1e-10)
    w = np.linalg.solve(osp.dense_A(two.M, 1e-2), b)
    assert np.linalg.norm(res.w - w) <= 1e-7 * np.linalg.norm(w)
    cg = krylov.cg(two.A, b, tol=1e-10, max_iter=5000)
    assert res.iters < cg.iters


def test_fcg_truncation_rule():
    """m_0 = 0 and m_i = max(1, i mod (m+1)): with m = 3, FCG on an SPD system
    with the identity preconditioner is CG and converges in <= f steps."""
    rng = np.random.default_rng(8)
    B = rng.standard_normal((12, 12))
    A = B @ B.T + np.eye(12)
    b = rng.standard_normal(12)
    res = krylov.fcg(lambda v: A @ v, lambda r, i: r.copy(), b, m=3, tol=1e-12)
    assert res.iters <= 14
    assert np.allclose(res.w, np.linalg.solve(A, b), rtol=1e-9)


# ---------------------------------------------------------------- k-means (Section 3.4)

def _brute_force_lloyd(X, centers, max_iter):
    """Lloyd with exact rational centroids and distances computed directly."""
    X = np.asarray(X, np.int64)
    N, F = X.shape
    cols = [[Fraction(int(v)) for v in X[:, i]] for i in range(F)]
    cent = [cols[c][:] for c in centers]
    size = [1] * len(centers)
    labels = None
    it = 0
    while it < max_iter:
        it += 1
        new = []
        for i in range(F):
            best, bd = None, None
            for S in range(len(cent)):
                if size[S] == 0:
                    continue
                dist = sum((cols[i][r] - cent[S][r]) ** 2 for r in range(N))
                if bd is None or dist < bd:
                    best, bd = S, dist
            new.append(best)
        if new == labels:
            break
        labels = new
        k = len(cent)
        size = [labels.count(S) for S in range(k)]
        cent = [[sum((cols[i][r] for i in range(F) if labels[i] == S), Fraction(0)) / size[S]
                 if size[S] else Fraction(0) for r in range(N)] for S in range(k)]
    return np.array(labels, np.int32), it


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_lloyd_matches_brute_force(seed):
    D = random_binary(12, 18, 0.35, 10 + seed)
    n, f, rp, ci = csr_of(D)
    cp, ri = osp.csc_pattern(n, f, rp, ci)
    centers = np.random.default_rng(seed).choice(f, size=4, replace=False)
    lab, it = km.lloyd_binary(n, f, rp, ci, cp, ri, centers, 50)
    ref, it_ref = _brute_force_lloyd(D, centers, 50)
    assert np.array_equal(lab, ref)
    assert it == it_ref


def test_lloyd_fixed_point_at_exit():
    """At convergence every label is the exact argmin for the exact means."""
    D = random_binary(15, 25, 0.3, 42)
    n, f, rp, ci = csr_of(D)
    cp, ri = osp.csc_pattern(n, f, rp, ci)
    lab, it = km.lloyd_binary(n, f, rp, ci, cp, ri, [0, 5, 9, 17, 21], 100)
    assert it < 100
    X = D.astype(object)
    for i in range(f):
        best = None
        for S in sorted(set(lab.tolist())):
            members = np.nonzero(lab == S)[0]
            mu = [Fraction(int(X[r, members].sum()), len(members)) for r in range(n)]
            dist = sum((Fraction(int(X[r, i])) - mu[r]) ** 2 for r in range(n))
            if best is None or dist < best[1]:
                best = (S, dist)
        assert lab[i] == best[0]


def test_lloyd_recovers_duplicate_groups():
    """Definition 1's ideal data with one centre per group: one assignment
    step gives the groups and the second changes nothing."""
    rng = np.random.default_rng(5)
    base = (rng.random((30, 5)) < 0.5).astype(np.int64)
    base[0] = 1
    X, groups = synth.duplicated_features(base, [2, 3, 1, 4, 2])
    perm = rng.permutation(X.shape[1])
    X, groups = X[:, perm], groups[perm]
    centers = [int(np.nonzero(groups == g)[0][-1]) for g in range(5)]
    n, f, rp, ci = csr_of(X)
    cp, ri = osp.csc_pattern(n, f, rp, ci)
    lab, it = km.lloyd_binary(n, f, rp, ci, cp, ri, centers, 10)
    assert np.array_equal(lab, groups)
    assert it == 2


def test_kmeanspp_picks_other_group():
    """Seeding: a second centre is never drawn where the squared distance to
    the first is zero (duplicates of the first centre)."""
    base = np.array([[1, 0], [1, 1], [0, 1], [1, 0]], np.int64)
    X, groups = synth.duplicated_features(base, [5, 4])
    n, f, rp, ci = csr_of(X)
    cp, ri = osp.csc_pattern(n, f, rp, ci)
    for seed in range(20):
        c = km.kmeanspp_binary(n, f, rp, ci, cp, ri, 2, seed)
        assert groups[c[0]] != groups[c[1]]
    # more centres than distinct features: the rest are the lowest unchosen ids
    c = km.kmeanspp_binary(n, f, rp, ci, cp, ri, 4, 0)
    assert len(set(c.tolist())) == 4


def test_kmeanspp_draw_follows_d2_weights():
    """The second centre is drawn with probability proportional to D^2."""
    X = np.zeros((8, 4), np.int64)
    X[0:1, 0] = 1          # feature 0: 1 row
    X[0:2, 1] = 1          # feature 1: overlaps 0 in one row
    X[2:6, 2] = 1          # feature 2: 4 disjoint rows
    X[6:8, 3] = 1          # feature 3: 2 disjoint rows
    n, f, rp, ci = csr_of(X)
    cp, ri = osp.csc_pattern(n, f, rp, ci)
    counts = np.zeros(4)
    firsts = 0
    for seed in range(4000):
        c = km.kmeanspp_binary(n, f, rp, ci, cp, ri, 2, seed)
        if c[0] == 0:
            firsts += 1
            counts[c[1]] += 1
    # D^2 from feature 0: [0, 1, 5, 3] -> probabilities [0, 1/9, 5/9, 3/9]
    p = counts / counts.sum()
    assert counts[0] == 0
    assert np.allclose(p[1:], [1 / 9, 5 / 9, 3 / 9], atol=0.06)
    assert abs(firsts / 4000 - 0.25) < 0.04


def _brute_force_lloyd_real(X, centers, max_iter):
    """Lloyd on real features with exact rational arithmetic (every float32
    value is a rational), the same rules: singleton starts, means over members,
    squared Euclidean distance, ties to the smallest cluster, empty clusters
    skipped, stop at the first step that changes no label."""
    X = np.asarray(X, np.float32)
    N, F = X.shape
    cols = [[Fraction(float(v)) for v in X[:, i]] for i in range(F)]
    cent = [cols[c][:] for c in centers]
    size = [1] * len(centers)
    labels = None
    it = 0
    while it < max_iter:
        it += 1
        new = []
        for i in range(F):
            best, bd = None, None
            for S in range(len(cent)):
                if size[S] == 0:
                    continue
                dist = sum((cols[i][r] - cent[S][r]) ** 2 for r in range(N))
                if bd is None or dist < bd:
                    best, bd = S, dist
            new.append(best)
        if new == labels:
            break
        labels = new
        size = [labels.count(S) for S in range(len(cent))]
        cent = [[sum((cols[i][r] for i in range(F) if labels[i] == S), Fraction(0)) / size[S]
                 if size[S] else Fraction(0) for r in range(N)] for S in range(len(cent))]
    return np.array(labels, np.int32), it


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_lloyd_dense_matches_exact_arithmetic(seed):
    """Section 3.4 on dense X: the FP64 Lloyd (blocked row sums) gives the
    labels and step count of exact rational Lloyd on random data (no near
    ties), here 70 rows (two blocks of 64 and a ragged one) and 16 features."""
    rng = np.random.default_rng(30 + seed)
    X = rng.standard_normal((70, 16)).astype(np.float32)
    X[:, 8:] += 1.5 * rng.standard_normal((1, 8)).astype(np.float32)   # two loose groups
    centers = rng.choice(16, size=4, replace=False)
    lab, it = km.lloyd_dense(X, centers, 30)
    ref, it_ref = _brute_force_lloyd_real(X, centers, 30)
    assert np.array_equal(lab, ref)
    assert it == it_ref


def test_kmeanspp_dense_draw_follows_d2_weights():
    """Dense k-means++: the second centre is drawn with probability
    proportional to the squared Euclidean distance to the first."""
    X = np.array([[1, 1, 0, 3],
                  [0, 1, 0, 0],
                  [0, 0, 2, 0]], np.float32)   # D^2 from feature 0: [0, 1, 5, 4]
    counts = np.zeros(4)
    firsts = 0
    for seed in range(4000):
        c = km.kmeanspp_dense(X, 2, seed)
        if c[0] == 0:
            firsts += 1
            counts[c[1]] += 1
    p = counts / counts.sum()
    assert counts[0] == 0
    assert np.allclose(p[1:], [0.1, 0.5, 0.4], atol=0.06)
    assert abs(firsts / 4000 - 0.25) < 0.04


def test_dense_omega_below_spectral_bound():
    """The Gershgorin omega on dense correlated X: w lambda_max(D^{-1} A) <= 1."""
    X = synth.dense_ar1(120, 30, 0.9, 4)
    two = tl.setup_dense(X, 0.1, 3, seed=0)
    A = osp.dense_A(two.M, 0.1)
    Dm = np.diag(1.0 / np.sqrt(two.d))
    lmax = np.linalg.eigvalsh(Dm @ A @ Dm).max()
    assert two.omega * lmax <= 1.0 + 1e-12
    assert np.allclose(two.d, np.diag(A))


def test_dense_kmeans_recovers_groups():
    rng = np.random.default_rng(9)
    base = rng.standard_normal((20, 3)).astype(np.float32)
    X, groups = synth.duplicated_features(base, [3, 2, 4])
    centers = [int(np.nonzero(groups == g)[0][0]) for g in range(3)]
    lab, it = km.lloyd_dense(X, centers, 10)
    assert np.array_equal(lab, groups) and it == 2


# ---------------------------------------------------------------- MLP (learned coarse correction)

def test_mlp_gradients_finite_differences():
    rng = np.random.default_rng(11)
    p = mlp.init_params(6, 5, lambda n: rng.random(n))
    for name in ("b1", "b2", "b3"):
        p[name] = 0.1 * rng.standard_normal(p[name].shape)
    X = rng.standard_normal((4, 6))
    T = rng.standard_normal((4, 6))
    g = mlp.backward(p, X, T)
    h = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(p, X, T)
            flat[idx] = old - h
            lm = mlp.loss(p, X, T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd))


def _metric_case():
    rng = np.random.default_rng(12)
    p = mlp.init_params(6, 5, lambda n: rng.random(n))
    for name in ("b1", "b2", "b3"):
        p[name] = 0.1 * rng.standard_normal(p[name].shape)
    X = rng.standard_normal((4, 6))
    T = rng.standard_normal((4, 6))
    C = rng.standard_normal((6, 6))
    return p, X, T, C


def test_mlp_metric_loss_is_plain_loss_of_transformed_output():
    """With W = C^T C the weighted loss 0.5/B sum (o - t)^T W (o - t) is the
    plain loss of the network whose output layer is multiplied by C, against
    the targets C t (an invariant: ||C d||^2 = d^T C^T C d)."""
    p, X, T, C = _metric_case()
    q = dict(p, W3=C @ p["W3"], b3=C @ p["b3"])
    assert np.isclose(mlp.loss(p, X, T, C.T @ C), mlp.loss(q, X, T @ C.T), rtol=1e-12)
    assert mlp.loss(p, X, T, np.eye(6)) == pytest.approx(mlp.loss(p, X, T), rel=1e-14)


def test_mlp_metric_gradients_finite_differences():
    """The weighted loss's gradients against central finite differences."""
    p, X, T, C = _metric_case()
    W = C.T @ C + np.eye(6)
    g = mlp.backward(p, X, T, W)
    h = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(p, X, T, W)
            flat[idx] = old - h
            lm = mlp.loss(p, X, T, W)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd))


def test_adam_first_step_is_lr_times_sign():
    p = {"W": np.array([1.0, -2.0, 3.0])}
    g = {"W": np.array([0.5, -7.0, 1e-3])}
    mlp.adam_step(p, g, {}, lr=0.01)
    assert np.allclose(p["W"], [0.99, -1.99, 2.99], atol=1e-6)


def test_learned_correction_positively_homogeneous():
    """e_c = ||r_c|| net(r_c / ||r_c||) scales with r_c even though the network
    itself does not (nonzero biases: a bias-free ReLU network would be
    homogeneous on its own and hide a missing rescaling)."""
    rng = np.random.default_rng(12)
    p = mlp.init_params(5, 4, lambda n: rng.random(n))
    for name in ("b1", "b2", "b3"):
        p[name] = 0.3 * rng.standard_normal(p[name].shape)
    rc = rng.standard_normal(5)
    o1, _ = mlp.forward(p, rc[None, :])
    o2, _ = mlp.forward(p, 3.5 * rc[None, :])
    assert not np.allclose(o2, 3.5 * o1)          # the network alone is not homogeneous
    assert np.allclose(mlp.coarse_correction(p, 3.5 * rc), 3.5 * mlp.coarse_correction(p, rc))


def test_harvest_pairs_first_two_iterations_closed_form():
    """The oracle's training pairs against the same quantities written out with
    dense matrices: iteration 0 has w_0 = 0, r_0 = b; iteration 1 has
    w_1 = alpha_0 z_0 with z_0 = M^-1 b and alpha_0 = <b, z_0> / <z_0, A z_0>.
    Then z1 = omega D^-1 r, x = P^T (r - A z1), t = P^T (w* - w - z1) with the
    dense P of Section 3.2 and w* the dense solve."""
    from oracle import learned
    X = synth.zipf_binary(120, 60, 0.08, 1.1, 4)
    lam = 0.05
    T = tl.setup_binary(X.n_rows, X.n_cols, X.row_ptr, X.col_idx, lam, 7, seed=2)
    y, _ = synth.ridge_targets(X, 9)
    b = osp.rhs(T.M, y)
    A = osp.dense_A(T.M, lam)
    P = tl.prolongation_dense(T.labels, T.s)
    w_star = np.linalg.solve(A, b)
    Xs, Ts = learned.harvest_pairs(T, b, w_star, 2)

    def pair(w, r):
        z1 = T.omega * r / np.diag(A)
        return P.T @ (r - A @ z1), P.T @ (w_star - w - z1)

    x0, t0 = pair(np.zeros_like(b), b)
    z0 = T.apply(b)
    a0 = (b @ z0) / (z0 @ A @ z0)
    x1, t1 = pair(a0 * z0, b - a0 * (A @ z0))
    for got, want in ((Xs[0], x0), (Ts[0], t0), (Xs[1], x1), (Ts[1], t1)):
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
    # the restricted remaining error and the restricted residual are the same
    # vector seen through A: x = P^T A u, t = P^T u with u = w* - w - z1
    u0 = w_star - T.omega * b / np.diag(A)
    assert np.allclose(P.T @ (A @ u0), Xs[0], rtol=1e-10, atol=1e-12 * np.linalg.norm(b))


def test_compact_drops_empty_clusters_in_order():
    """Empty clusters are dropped and the others renumbered in their order."""
    labels, n_S = km.compact(np.array([4, 1, 4, 7, 1, 4], np.int32))
    assert labels.tolist() == [1, 0, 1, 2, 0, 1]
    assert n_S.tolist() == [2, 3, 1]


def test_with_lambda_equals_fresh_setup_with_same_clustering():
    """Section 4: at another lambda only the coarse factor and the smoother
    change; a fresh setup from the same initial centres gives the same."""
    two, _ = _tiny_two_level(seed=9)
    D = two.M.X.toarray()
    n, f, rp, ci = csr_of(D)
    other = two.with_lambda(0.5)
    fresh = tl.setup_binary(n, f, rp, ci, 0.5, len(two.centers), centers=two.centers)
    assert np.array_equal(other.labels, fresh.labels)
    assert np.array_equal(other.Ac, fresh.Ac)
    assert np.array_equal(other.d, fresh.d) and other.omega == fresh.omega


def test_coarse_counts_and_integer_gram_by_brute_force():
    """Section 3.2: C = X onehot(labels) counts a row's features per cluster and
    G = C^T C (X_c = X P = C D_s); checked by loops over Python integers, and
    by the invariant sum_{S,T} G[S,T] = sum_r (row length)^2."""
    D = random_binary(23, 17, 0.35, 8)
    n, f, rp, ci = csr_of(D)
    labels = np.array([2, 0, 1, 2, 3, 0, 1, 1, 3, 2, 0, 3, 1, 2, 0, 0, 3], np.int32)
    k = 4
    C = tl.coarse_counts(n, f, rp, ci, labels, k).toarray()
    G = tl.coarse_gram_binary(n, f, rp, ci, labels, k)
    Cb = [[sum(int(D[r, j]) for j in range(f) if labels[j] == S) for S in range(k)]
          for r in range(n)]
    Gb = [[sum(Cb[r][S] * Cb[r][T] for r in range(n)) for T in range(k)] for S in range(k)]
    assert C.tolist() == Cb
    assert G.dtype == np.int64 and G.tolist() == Gb
    assert int(G.sum()) == int((D.sum(axis=1) ** 2).sum())


def test_gershgorin_rowsums_by_brute_force():
    """Section 3.1's damping bound uses the row sums of |X^T X|, here summed
    entry by entry from the dense product, for binary and signed dense X."""
    D = random_binary(15, 9, 0.4, 9)
    M = osp.from_csr(*csr_of(D))
    A = D.T @ D
    assert np.array_equal(osp.gershgorin_rowsums(M), np.abs(A).sum(axis=1).astype(float))
    Xd = np.random.default_rng(2).standard_normal((12, 7))
    Md = osp.from_dense(Xd)
    brute = [sum(abs(sum(Xd[r, i] * Xd[r, j] for r in range(12))) for j in range(7))
             for i in range(7)]
    # |X|^T |X| 1 bounds the row sums of |X^T X| from above (equal for X >= 0)
    assert np.all(osp.gershgorin_rowsums(Md) >= np.array(brute) - 1e-12)


def test_triangular_solves_against_library():
    """Section 4's coarse solve as two triangular solves, checked against
    scipy.linalg.solve_triangular."""
    from scipy.linalg import solve_triangular
    rng = np.random.default_rng(11)
    L = np.tril(rng.standard_normal((12, 12))) + 6 * np.eye(12)
    b = rng.standard_normal(12)
    assert np.allclose(tl.forward_sub(L, b), solve_triangular(L, b, lower=True), rtol=1e-13)
    assert np.allclose(tl.back_sub_t(L, b), solve_triangular(L.T, b, lower=False), rtol=1e-13)


def test_dense_matrix_products_match_numpy():
    """Eq. (1)'s operator for a dense X: X v, X^T u and (X^T X + lambda I) v."""
    rng = np.random.default_rng(12)
    Xd = rng.standard_normal((9, 5))
    M = osp.from_dense(Xd)
    v, u = rng.standard_normal(5), rng.standard_normal(9)
    assert np.allclose(osp.X_mv(M, v), Xd @ v, rtol=1e-14)
    assert np.allclose(osp.Xt_mv(M, u), Xd.T @ u, rtol=1e-14)
    assert np.allclose(osp.apply_A(M, 0.2, v), (Xd.T @ Xd + 0.2 * np.eye(5)) @ v, rtol=1e-13)


def test_lloyd_threads_do_not_change_labels():
    """The Lloyd assignment step may run on several threads; each feature's
    argmin is exact integer arithmetic of its own, so the labels and the step
    count are the same on one thread and on all of them."""
    X = synth.zipf_binary(3001, 1777, 0.006, 1.1, 5)
    cp, ri = osp.csc_pattern(X.n_rows, X.n_cols, X.row_ptr, X.col_idx)
    c = km.kmeanspp_binary(X.n_rows, X.n_cols, X.row_ptr, X.col_idx, cp, ri, 37, 5)
    out = []
    for t in (1, 0):
        km.set_threads(t)
        out.append(km.lloyd_binary(X.n_rows, X.n_cols, X.row_ptr, X.col_idx, cp, ri, c, 50))
    km.set_threads(0)
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]


def test_reference_solutions_are_the_dense_solution():
    """oracle.reference (exact solutions in spawned processes, the
    preconditioner rebuilt from given labels) against a dense Cholesky solve,
    and its 1e-8 snapshot against the oracle's own PCG run to 1e-8."""
    from oracle import reference
    spec = (2000, 1000, 0.01, 1.1, 0)
    X = synth.zipf_binary(*spec)
    Y, _ = synth.ridge_targets_many(X, [0, 1])
    _, raw, _ = reference.oracle_labels(spec, 50, 0)
    lams = (1e-2, 1.0)
    out = reference.exact_solutions(spec, raw, [(lams[0], Y[0]), (lams[1], Y[1])], processes=2)
    M = osp.from_csr(*spec[:2], X.row_ptr, X.col_idx)
    for (w, snaps, iters, rel), lam, y in zip(out, lams, Y):
        b = osp.rhs(M, y)
        ws = np.linalg.solve(osp.dense_A(M, lam), b)
        assert rel <= reference.TOL_REF
        assert np.linalg.norm(w - ws) <= 1e-8 * np.linalg.norm(ws)
        two = tl.from_labels(*spec[:2], X.row_ptr, X.col_idx, lam, raw)
        want = krylov.pcg(two.A, two.apply, b, tol=1e-8)
        assert want.restarts == 0 and np.array_equal(snaps[1e-8], want.w)


# ---------------------------------------------------------------- eigen coarse solve (Section 4)

def test_jacobi_eigh_against_library_eigh():
    """The cyclic Jacobi eigendecomposition against numpy.linalg.eigh: the
    same spectrum, Q orthogonal, Q diag(mu) Q^T = S."""
    from oracle import eigen
    rng = np.random.default_rng(3)
    B = rng.standard_normal((40, 25))
    S = B.T @ B
    mu, Q, sweeps = eigen.jacobi_eigh(S)
    assert 3 <= sweeps <= 15
    assert np.allclose(np.sort(mu), np.linalg.eigvalsh(S), rtol=1e-12, atol=1e-12 * mu.max())
    assert np.allclose(Q.T @ Q, np.eye(25), atol=1e-13)
    assert np.allclose((Q * mu) @ Q.T, S, atol=1e-12 * np.abs(S).max())


def test_eigen_coarse_inverse_equals_cholesky_solve_at_every_lambda():
    """Section 4: one decomposition of X_c^T X_c serves every lambda; the coarse
    solve Q diag(1/(mu+lambda)) Q^T r equals the Cholesky solve of A_c(lambda)."""
    from oracle import eigen
    D = random_binary(60, 30, 0.2, 4)
    n, f, rp, ci = csr_of(D)
    two = tl.setup_binary(n, f, rp, ci, 0.1, 8, seed=2)
    mu, Q, _ = eigen.jacobi_eigh(eigen.coarse_gram_scaled(two.G, two.s))
    rc = np.random.default_rng(5).standard_normal(two.k_eff)
    for lam in (1e-4, 0.1, 3.0, 1e3):
        t = two.with_lambda(lam)
        want = tl.chol_solve(t.L, rc)
        got = eigen.coarse_solve(mu, Q, lam, rc)
        # both solves are backward stable: they agree to about cond(A_c) eps
        tol = max(1e-13, 1e-15 * np.linalg.cond(t.Ac))
        assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want), lam
        assert np.allclose(eigen.coarse_inverse(mu, Q, lam) @ t.Ac, np.eye(two.k_eff),
                           atol=100 * tol)


def test_eigen_theorem1_spectrum():
    """Theorem 1: on duplicated features the eigenvalues of X_c^T X_c (computed
    by the oracle's Jacobi) are the non-zero eigenvalues of X^T X."""
    from oracle import eigen
    rng = np.random.default_rng(1)
    base = (rng.random((30, 5)) < 0.5).astype(np.int64)
    base[0] = 1
    X, groups = synth.duplicated_features(base, [2, 3, 1, 4, 2])
    centers = [int(np.nonzero(groups == g)[0][0]) for g in range(5)]
    n, f, rp, ci = csr_of(X)
    two = tl.setup_binary(n, f, rp, ci, 1e-6, 5, centers=centers)
    mu, _, _ = eigen.jacobi_eigh(eigen.coarse_gram_scaled(two.G, two.s))
    ev = np.linalg.eigvalsh((X.T @ X).astype(float))
    nz = np.sort(ev[ev > 1e-9 * ev.max()])
    assert np.allclose(np.sort(mu[mu > 1e-9 * mu.max()]), nz, rtol=1e-11)


# ---------------------------------------------------------------- Bayesian regression

def test_counter_normals_are_standard_normal():
    """The Box-Muller normals of the counter-based generator: a
    Kolmogorov-Smirnov test against the library normal, and independence of
    neighbouring draws (their correlation)."""
    from scipy import stats
    z = synth.normal(21, 5, 20000)
    assert stats.kstest(z, stats.norm.cdf).pvalue > 1e-3
    assert abs(np.corrcoef(z[:-1], z[1:])[0, 1]) <= 5 / np.sqrt(len(z))


def test_gamma_draw_distribution():
    """Marsaglia & Tsang on the counter-based uniforms draws Gamma(shape a,
    rate): a Kolmogorov-Smirnov test against the library's gamma law and the
    first two moments (a / rate, a / rate^2), at the method's boundary a = 1
    and above."""
    from scipy import stats
    from oracle import bayes
    n = 2000
    for a, rate in ((1.0, 2.0), (3.7, 0.5), (250.5, 40.0)):
        x = np.array([bayes.gamma_draw(a, rate, 11, bayes.STREAM_GAMMA + s) for s in range(n)])
        assert stats.kstest(x, stats.gamma(a, scale=1.0 / rate).cdf).pvalue > 1e-3
        m, v = a / rate, a / rate ** 2
        assert abs(x.mean() - m) <= 5 * np.sqrt(v / n)
        # the sample variance's spread follows from the gamma law's kurtosis 6/a
        assert abs(x.var() / v - 1) <= 5 * np.sqrt((2 + 6 / a) / n)


def _bayes_small():
    X = random_binary(60, 6, 0.3, 8)
    n, f, rp, ci = csr_of(X)
    y = synth.normal(8, 77, n)
    return X, y, tl.setup_binary(n, f, rp, ci, 1.0, 2, seed=0)


def test_noise_injected_sample_has_the_conditional_posterior_moments():
    """Section 2, Eq. (ni_xtx): over the draws of e1 and e2 the solution of the
    noise-injected system has mean (X^T X + (lambda/tau) I)^-1 X^T y and
    covariance (tau X^T X + lambda I)^-1, the conditional posterior of w given
    lambda and tau (Gaussian prior and likelihood; the normal equations in
    closed form with the library solver), checked by sampling."""
    from oracle import bayes
    X, y, two = _bayes_small()
    lam, tau = 20.0, 2.0
    G = (X.T @ X).astype(float)
    f = G.shape[0]
    mean = np.linalg.solve(G + (lam / tau) * np.eye(f), X.T @ y)
    cov = np.linalg.inv(tau * G + lam * np.eye(f))
    n = 3000
    W = np.array([bayes.noise_sample(two, y, lam, tau, 5, t, 1e-12).w for t in range(n)])
    assert np.all(np.abs(W.mean(0) - mean) <= 5 * np.sqrt(np.diag(cov) / n))
    S = np.cov(W.T)
    assert np.linalg.norm(S - cov) / np.linalg.norm(cov) <= 0.15


def test_gibbs_chain_recovers_the_generating_precisions():
    """Section 2's conjugate updates: on data drawn from the model (w with
    precision lambda = 4, noise with precision tau = 100) the chain's draws
    of lambda and tau settle around the generating values (their posteriors
    have relative spread about sqrt(2/F) and sqrt(2/N)), and its mean of w
    is within a few posterior standard deviations of the generating w."""
    from oracle import bayes
    N, F = 4000, 200
    lam_true, tau_true = 4.0, 100.0
    Xs = synth.zipf_binary(N, F, 0.05, 1.1, 5)
    M = osp.from_csr(N, F, Xs.row_ptr, Xs.col_idx)
    w_true = synth.normal(5, 900, F) / np.sqrt(lam_true)
    y = osp.X_mv(M, w_true) + synth.normal(5, 901, N) / np.sqrt(tau_true)
    two = tl.setup_binary(N, F, Xs.row_ptr, Xs.col_idx, 1.0, 20, seed=0)
    p = bayes.Params(alpha=1.0, beta=1.0, a_tau=1.0, b_tau=1.0, lambda0=1.0, tau0=1.0, seed=7,
                     tol=1e-10)
    lams, taus, wmean, _ = bayes.gibbs(two, y, p, n_samples=30, burnin=10)
    assert 0.85 * tau_true <= taus[10:].mean() <= 1.15 * tau_true
    assert 0.6 * lam_true <= lams[10:].mean() <= 1.6 * lam_true
    # the mean of 20 draws is within a few posterior standard deviations,
    # diag((tau X^T X + lambda I)^-1)^1/2, of the generating w
    G = osp.dense_A(M, 0.0)
    sd = np.sqrt(np.diag(np.linalg.inv(tau_true * G + lam_true * np.eye(F))))
    assert np.all(np.abs(wmean - w_true) <= 5 * sd * np.sqrt(1 + 1 / 20))


def test_gibbs_with_fixed_tau():
    """a_tau <= 0 keeps tau at tau0; lambda is still drawn every step."""
    from oracle import bayes
    X, y, two = _bayes_small()
    p = bayes.Params(a_tau=0.0, tau0=3.0, lambda0=2.0, seed=1, tol=1e-10)
    lams, taus, _, _ = bayes.gibbs(two, y, p, n_samples=4)
    assert np.all(taus == 3.0)
    assert len(set(lams.tolist())) == 4


# ---------------------------------------------------------------- leader-follower clustering

def _lf_hand_example():
    # 4 rows, 5 features: f0 = {0, 1}, f1 = {0, 1}, f2 = {2}, f3 = {0, 1, 2}, f4 = {3}
    X = np.zeros((4, 5), dtype=np.int64)
    for j, rows in enumerate(([0, 1], [0, 1], [2], [0, 1, 2], [3])):
        X[rows, j] = 1
    return X


@pytest.mark.parametrize("tol2,leaders,labels", [
    # f0 leads; d2(f1, f0) = 0; d2(f2, f0) = 3; d2(f3, f0) = 1, d2(f3, f2) = 2;
    # d2(f4, f0) = 3, d2(f4, f2) = 2
    (1.5, [0, 2, 4], [0, 0, 1, 0, 2]),
    (2.0, [0, 2, 4], [0, 0, 1, 0, 2]),     # d2 = 2 is not below 2: f4 leads
    (2.5, [0, 2], [0, 0, 1, 0, 1]),
    (3.5, [0], [0, 0, 0, 0, 0]),
    (0.0, [0, 1, 2, 3, 4], [0, 1, 2, 3, 4]),  # nothing is below 0: every feature leads
])
def test_leader_follower_worked_example(tol2, leaders, labels):
    """Algorithm 1 worked by hand on five binary features (squared Euclidean
    distances in the comments), including the strict comparison at d^2 = tol2."""
    from oracle import leader
    n, f, rp, ci = csr_of(_lf_hand_example())
    L, lab = leader.leader_follower_binary(n, f, rp, ci, tol2)
    assert L.tolist() == leaders and lab.tolist() == labels


def test_leader_follower_characterisation():
    """The output of Algorithm 1 is fixed by two properties, checked against a
    brute-force distance matrix (n_i + n_j - 2 X^T X): a leader is at distance
    >= tol from every earlier leader; a follower's nearest earlier leader (the
    earliest on ties) is below tol and is its label."""
    from oracle import leader
    for seed, (n, f, p) in enumerate(((40, 30, 0.2), (60, 80, 0.05), (25, 50, 0.4))):
        X = random_binary(n, f, p, 100 + seed)
        D2 = X.sum(0)[:, None] + X.sum(0)[None, :] - 2 * (X.T @ X)
        nr, nc, rp, ci = csr_of(X)
        for tol2 in (1.0, 3.0, 6.5, 12.0):
            L, lab = leader.leader_follower_binary(nr, nc, rp, ci, tol2)
            Ls = list(L)
            assert Ls == sorted(Ls) and Ls[0] == 0
            for i in range(f):
                earlier = [s for s, c in enumerate(Ls) if c < i]
                if i in Ls:
                    assert lab[i] == Ls.index(i)
                    assert all(D2[i, Ls[s]] >= tol2 for s in earlier)
                else:
                    d = [D2[i, Ls[s]] for s in earlier]
                    best = int(np.argmin(d))
                    assert d[best] < tol2 and lab[i] == earlier[best]


def test_leader_follower_recovers_duplicated_features():
    """Definition 1's duplicated features: with tol2 = 0.5 identical columns
    (d^2 = 0) follow the first of their group and distinct columns (d^2 >= 1)
    never join, so the clusters are the groups, led by their first members."""
    from oracle import leader
    rng = np.random.default_rng(5)
    while True:
        base = (rng.random((30, 6)) < 0.5).astype(np.int64)
        if len({tuple(c) for c in base.T}) == 6 and base.sum(0).min() > 0:
            break
    X, groups = synth.duplicated_features(base, [3, 1, 4, 2, 2, 5])
    n, f, rp, ci = csr_of(X)
    L, lab = leader.leader_follower_binary(n, f, rp, ci, 0.5)
    first = {}
    for j, g in enumerate(groups):
        first.setdefault(int(g), j)
    assert sorted(L.tolist()) == sorted(first.values())
    for j, g in enumerate(groups):
        assert L[lab[j]] == first[int(g)]
