"""The coarse Cholesky's blocked form (CPU restatement of its arithmetic).

The GPU factors A_c in 32-column steps: the diagonal block by right-looking
elimination, which also forms W = L11^{-1} (the same elimination applied to
the identity); the panel as the product L21 = A21 W^T instead of a triangular
solve per row; then the trailing update A22 -= L21 L21^T. This restatement, in
FP64 with a ragged last block, must reproduce LAPACK's factor of SPD matrices
up to condition 1e9 to within that conditioning, and a planted error in the
panel (W instead of W^T) must break it.
"""
import numpy as np

NB = 32


def diag_factor(a):
    nb = a.shape[0]
    a = a.copy()
    for j in range(nb):
        a[j, j] = np.sqrt(a[j, j])
        a[j + 1:, j] /= a[j, j]
        for i in range(j + 1, nb):
            a[i, j + 1:i + 1] -= a[i, j] * a[j + 1:i + 1, j]
    L = np.tril(a)
    w = np.eye(nb)
    for j in range(nb):
        w[j, :j + 1] /= L[j, j]
        for i in range(j + 1, nb):
            w[i, :j + 1] -= L[i, j] * w[j, :j + 1]
    return L, w


def blocked_cholesky(A, transpose_w=True):
    k = A.shape[0]
    L = A.copy()
    for j0 in range(0, k, NB):
        nb = min(NB, k - j0)
        L11, W = diag_factor(L[j0:j0 + nb, j0:j0 + nb])
        L[j0:j0 + nb, j0:j0 + nb] = L11
        rest = slice(j0 + nb, k)
        if j0 + nb < k:
            L[rest, j0:j0 + nb] = L[rest, j0:j0 + nb] @ (W.T if transpose_w else W)
            L21 = L[rest, j0:j0 + nb]
            L[rest, rest] -= np.tril(L21 @ L21.T)
    return np.tril(L)


def spd(k, cond, rng):
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    ev = np.geomspace(1.0, cond, k)
    A = (Q * ev) @ Q.T
    return (A + A.T) / 2


def test_blocked_factor_matches_lapack():
    rng = np.random.default_rng(5)
    for k, cond in [(70, 1e2), (101, 1e6), (160, 1e9), (33, 1e3), (31, 1e4)]:
        A = spd(k, cond, rng)
        L = blocked_cholesky(A)
        ref = np.linalg.cholesky(A)
        # backward error at FP64 level, forward error within the conditioning
        assert np.linalg.norm(L @ L.T - A) <= 1e-13 * np.linalg.norm(A) * k, (k, cond)
        assert np.linalg.norm(L - ref) <= 1e-15 * np.sqrt(cond) * 100 * np.linalg.norm(ref), (k, cond)


def test_planted_panel_error_is_caught():
    rng = np.random.default_rng(6)
    A = spd(101, 1e4, rng)
    with np.errstate(invalid="ignore"):
        L = blocked_cholesky(A, transpose_w=False)
        err = np.linalg.norm(L @ L.T - A)
    # a non-positive pivot (NaN) or a large residual: either way not a factor of A
    assert not (err <= 1e-6 * np.linalg.norm(A))
