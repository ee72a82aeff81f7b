"""Oracle: the clustering-based two-level preconditioner (Section 3).

Test infrastructure only.

  P            Eq. (prolong): P(i, S) = 1/sqrt(n_S) for feature i in cluster S,
               so P^T P = I (Section 3.2).
  coarse op    Section 3.2: A_c = P^T (X^T X + lambda I) P = X_c^T X_c + lambda I,
               X_c = X P. For binary X, X_c = C D_s with the integer counts
               C = X (one-hot cluster matrix) and D_s = diag(1/sqrt(n_S)), so
               A_c[S,T] = (G[S,T] s_S) s_T + lambda delta_ST with G = C^T C exact.
  coarse solve Section 4: Cholesky factor of A_c, forward then back substitution.
  smoother     Section 3.1's Richardson step generalised to damped Jacobi
               w D^{-1}, D = diag(A); w = 1/L with L the Gershgorin bound on the
               spectrum of D^{-1} A, so w * lambda_max(D^{-1}A) <= 1 and the
               symmetric cycle below is SPD.
  cycle        Section 3.1: T = (I - S A)(I - P A_c^{-1} P^T A)(I - S A), i.e.
               z1 = S r; r1 = r - A z1; e_c = A_c^{-1} P^T r1; z2 = z1 + P e_c;
               r2 = r - A z2; z = z2 + S r2, with S = w D^{-1}.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from . import kmeans as km
from . import sparse as osp


class NotSPD(ValueError):
    pass


def prolong_scale(n_S):
    """s_S = 1/sqrt(n_S): an IEEE square root, then an IEEE division."""
    return 1.0 / np.sqrt(np.asarray(n_S, dtype=np.float64))


def restrict(labels, s, r):
    """r_c = P^T r: r_c[S] = s_S * (sum of r[i] over i in S, ascending i)."""
    return s * np.bincount(labels, weights=r, minlength=len(s))


def prolong(labels, s, e_c):
    """P e_c: (P e_c)[i] = s_{S(i)} e_c[S(i)]."""
    return s[labels] * e_c[labels]


def prolongation_dense(labels, s):
    """P as an explicit F x k matrix (tiny inputs only)."""
    F, k = len(labels), len(s)
    P = np.zeros((F, k))
    P[np.arange(F), labels] = s[labels]
    return P


def averaging_dense(labels, n_S):
    """The plain averaging operator P~ with entries 1/n_S (Section 3.2), tiny inputs only."""
    F, k = len(labels), len(n_S)
    P = np.zeros((F, k))
    P[np.arange(F), labels] = 1.0 / np.asarray(n_S, np.float64)[labels]
    return P


def coarse_counts(n_rows, n_cols, row_ptr, col_idx, labels, k):
    """C = X * onehot(labels): C[r, S] = number of features of cluster S in row r."""
    X = sp.csr_matrix((np.ones(len(col_idx), np.int64), np.asarray(col_idx, np.int64),
                       np.asarray(row_ptr, np.int64)), shape=(n_rows, n_cols))
    A = sp.csr_matrix((np.ones(n_cols, np.int64), np.asarray(labels, np.int64),
                       np.arange(n_cols + 1)), shape=(n_cols, k))
    return (X @ A).tocsr()


def coarse_gram_binary(n_rows, n_cols, row_ptr, col_idx, labels, k):
    """G = C^T C in exact int64 (dense k x k)."""
    C = coarse_counts(n_rows, n_cols, row_ptr, col_idx, labels, k)
    return np.asarray((C.T @ C).toarray(), dtype=np.int64)


def coarse_operator_binary(G, s, lam):
    """A_c from the exact Gram: lower triangle (G[S,T] s_S) s_T, mirrored; + lambda I."""
    A = (np.asarray(G, np.float64) * s[:, None]) * s[None, :]
    A = np.tril(A) + np.tril(A, -1).T
    A[np.diag_indices_from(A)] += lam
    return A


def coarse_operator_dense(X, labels, s, lam):
    """A_c = X_c^T X_c + lambda I with X_c = X P (dense X)."""
    Xc = X @ prolongation_dense(labels, s)
    return Xc.T @ Xc + lam * np.eye(len(s))


def cholesky(A):
    """Unblocked Cholesky A = L L^T (column by column); raises NotSPD on a pivot <= 0."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    L = np.zeros_like(A)
    for j in range(n):
        piv = A[j, j] - L[j, :j] @ L[j, :j]
        if not piv > 0.0:
            raise NotSPD(f"pivot {j} = {piv}")
        L[j, j] = np.sqrt(piv)
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def forward_sub(L, b):
    y = np.zeros_like(b, dtype=np.float64)
    for i in range(len(b)):
        y[i] = (b[i] - L[i, :i] @ y[:i]) / L[i, i]
    return y


def back_sub_t(L, y):
    """Solve L^T x = y."""
    n = len(y)
    x = np.zeros_like(y, dtype=np.float64)
    for i in range(n - 1, -1, -1):
        x[i] = (y[i] - L[i + 1:, i] @ x[i + 1:]) / L[i, i]
    return x


def chol_solve(L, b):
    return back_sub_t(L, forward_sub(L, b))


@dataclasses.dataclass
class TwoLevel:
    M: osp.Matrix
    lam: float
    labels: np.ndarray        # int32[F], compacted cluster of each feature
    n_S: np.ndarray           # int64[k_eff]
    s: np.ndarray             # 1/sqrt(n_S)
    G: np.ndarray | None      # exact Gram (binary X) or None
    Ac: np.ndarray
    L: np.ndarray
    d: np.ndarray             # diag(A)
    omega: float
    centers: np.ndarray       # the initial centres used by Lloyd
    kmeans_iters: int

    @property
    def k_eff(self):
        return len(self.n_S)

    def A(self, v):
        return osp.apply_A(self.M, self.lam, v)

    def coarse_correction(self, r1):
        """e_c = A_c^{-1} P^T r1."""
        return chol_solve(self.L, restrict(self.labels, self.s, r1))

    def apply(self, r):
        """z = M^{-1} r for the symmetric two-level cycle of Section 3.1."""
        z1 = self.omega * r / self.d
        r1 = r - self.A(z1)
        e_c = self.coarse_correction(r1)
        z2 = z1 + prolong(self.labels, self.s, e_c)
        r2 = r - self.A(z2)
        return z2 + self.omega * r2 / self.d

    def apply_tlfcg(self, r, steps=2):
        """The cycle the paper recommends for FCG (Section 3.1 and Section 4's
        smoothing study): `steps` iterations of CG on A z = r from z = 0 as a
        pre-smoother (the "rougher"), then the coarse correction of what is
        left: z = z1 + P A_c^-1 P^T r1, with r1 = r - A z1 carried by the CG
        recurrence. No post-smoothing. z depends non-linearly on r (CG), so the
        outer method is flexible CG."""
        r = np.asarray(r, np.float64)
        z1 = np.zeros_like(r)
        res = r.copy()
        rho = float(res @ res)
        p = res.copy()
        for j in range(steps):
            if rho == 0.0:
                break
            if j > 0:
                p = res + (rho / rho_old) * p
            q = self.A(p)
            alpha = rho / float(p @ q)
            z1 += alpha * p
            res -= alpha * q
            rho_old, rho = rho, float(res @ res)
        return z1 + prolong(self.labels, self.s, self.coarse_correction(res))

    def with_lambda(self, lam):
        """The same clustering at another lambda: the coarse factor and the
        smoother are rebuilt, the clustering is reused (Section 4: the
        Cholesky factor must be recomputed when beta changes)."""
        d = osp.col_sq_norms(self.M) + lam
        omega = jacobi_omega(self.M, d, lam)
        if self.G is not None:
            Ac = coarse_operator_binary(self.G, self.s, lam)
        else:
            Ac = coarse_operator_dense(self.M.X, self.labels, self.s, lam)
        return dataclasses.replace(self, lam=lam, Ac=Ac, L=cholesky(Ac), d=d, omega=omega)


def jacobi_omega(M, d, lam):
    """w = 1 / max_i ((|X|^T |X| 1)_i + lambda) / d_i (Gershgorin bound on D^{-1} A)."""
    return 1.0 / float(np.max((osp.gershgorin_rowsums(M) + lam) / d))


def setup_binary(n_rows, n_cols, row_ptr, col_idx, lam, k, seed=0, centers=None,
                 kmeans_max_iter=50):
    """Clustering, prolongation, Galerkin coarse operator and its Cholesky
    factor, and the Jacobi smoother, for binary X given as a CSR pattern."""
    col_ptr, row_idx = osp.csc_pattern(n_rows, n_cols, row_ptr, col_idx)
    if centers is None:
        centers = km.kmeanspp_binary(n_rows, n_cols, row_ptr, col_idx, col_ptr, row_idx, k, seed)
    raw, iters = km.lloyd_binary(n_rows, n_cols, row_ptr, col_idx, col_ptr, row_idx,
                                 centers, kmeans_max_iter)
    return from_labels(n_rows, n_cols, row_ptr, col_idx, lam, raw, centers, iters)


def from_labels(n_rows, n_cols, row_ptr, col_idx, lam, raw_labels, centers=(), iters=0):
    """The steps of setup_binary after the clustering, from given (raw) cluster
    labels: compaction, P, the exact Gram, A_c and its factor, the smoother."""
    M = osp.from_csr(n_rows, n_cols, row_ptr, col_idx)
    labels, n_S = km.compact(raw_labels)
    s = prolong_scale(n_S)
    G = coarse_gram_binary(n_rows, n_cols, row_ptr, col_idx, labels, len(n_S))
    Ac = coarse_operator_binary(G, s, lam)
    d = osp.col_sq_norms(M) + lam
    return TwoLevel(M, lam, labels, n_S, s, G, Ac, cholesky(Ac), d, jacobi_omega(M, d, lam),
                    np.asarray(centers, np.int32), iters)


def setup_dense(X, lam, k, seed=0, centers=None, kmeans_max_iter=50):
    """The same for dense X (N x F)."""
    M = osp.from_dense(X)
    if centers is None:
        centers = km.kmeanspp_dense(X, k, seed)
    raw, iters = km.lloyd_dense(X, centers, kmeans_max_iter)
    labels, n_S = km.compact(raw)
    s = prolong_scale(n_S)
    Ac = coarse_operator_dense(M.X, labels, s, lam)
    d = osp.col_sq_norms(M) + lam
    return TwoLevel(M, lam, labels, n_S, s, None, Ac, cholesky(Ac), d, jacobi_omega(M, d, lam),
                    np.asarray(centers, np.int32), iters)
