"""Oracle: the coarse solve by eigendecomposition, reused across lambda.

Test infrastructure only.

Section 4 notes that the Cholesky factor of the coarse operator has to be
recomputed whenever beta (lambda here) changes, while a decomposition of the
coarse matrix X_c = X P can be reused. With the Galerkin operator
A_c(lambda) = X_c^T X_c + lambda I (Section 3.2), the symmetric
eigendecomposition of the lambda-free part

    G_s = X_c^T X_c = D_s G D_s = Q diag(mu) Q^T      (Q orthogonal)

gives every coarse inverse at once:

    A_c(lambda)^{-1} = Q diag(1 / (mu + lambda)) Q^T.

(X_c's right singular vectors are Q's columns and its squared singular values
are mu; the eigendecomposition of G_s is the same object without forming an
SVD of the N x k matrix.)

The eigendecomposition is computed by the cyclic Jacobi method (Jacobi 1846;
the cyclic-by-row sweep of Golub & Van Loan, Matrix Computations, Section
8.5): each step annihilates one off-diagonal entry (p, q) by a plane rotation
J with tan(phi) = t, t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
tau = (a_qq - a_pp) / (2 a_pq), c = 1 / sqrt(1 + t^2), s = t c, applied as
A <- J^T A J and accumulated as Q <- Q J; sweeps over all pairs p < q repeat
until the off-diagonal Frobenius norm is below tol times that of A. Plain
loops over the pairs, vectorised along the rows: for small k only.
"""
from __future__ import annotations

import numpy as np


def jacobi_eigh(S, tol=1e-15, max_sweeps=50):
    """(mu, Q, sweeps) with S = Q diag(mu) Q^T, S symmetric (k x k)."""
    A = np.array(S, dtype=np.float64, copy=True)
    n = A.shape[0]
    Q = np.eye(n)
    norm = np.linalg.norm(A)
    sweeps = 0
    for sweeps in range(1, max_sweeps + 1):
        off = np.linalg.norm(A - np.diag(np.diag(A)))   # directly, not by cancellation
        if off <= tol * norm:
            sweeps -= 1
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                tau = (A[q, q] - A[p, p]) / (2.0 * apq)
                t = (1.0 if tau >= 0.0 else -1.0) / (abs(tau) + np.sqrt(1.0 + tau * tau))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = t * c
                # A <- J^T A J: rows p and q, then columns p and q
                rp, rq = A[p, :].copy(), A[q, :].copy()
                A[p, :] = c * rp - s * rq
                A[q, :] = s * rp + c * rq
                cp, cq = A[:, p].copy(), A[:, q].copy()
                A[:, p] = c * cp - s * cq
                A[:, q] = s * cp + c * cq
                A[p, q] = A[q, p] = 0.0
                # Q <- Q J
                qp, qq = Q[:, p].copy(), Q[:, q].copy()
                Q[:, p] = c * qp - s * qq
                Q[:, q] = s * qp + c * qq
    return np.diag(A).copy(), Q, sweeps


def coarse_gram_scaled(G, s):
    """G_s = D_s G D_s with D_s = diag(1/sqrt(n_S)): the coarse operator without
    its lambda (lower triangle (G[S,T] s_S) s_T, mirrored, as the Cholesky path
    forms A_c)."""
    A = (np.asarray(G, np.float64) * s[:, None]) * s[None, :]
    return np.tril(A) + np.tril(A, -1).T


def coarse_inverse(mu, Q, lam):
    """A_c(lambda)^{-1} = Q diag(1 / (mu + lambda)) Q^T."""
    return (Q * (1.0 / (mu + lam))[None, :]) @ Q.T


def coarse_solve(mu, Q, lam, rc):
    """e_c = A_c(lambda)^{-1} r_c as Q (diag(1 / (mu + lambda)) (Q^T r_c))."""
    return Q @ ((Q.T @ rc) / (mu + lam))
