"""Oracle: the matrix-free operator of Eq. (1) on binary CSR or dense X.

Test infrastructure only. The system matrix A = X^T X + lambda I is never
formed: it is applied as two mat-vecs, u = X v then X^T u, plus lambda v
(Section 1: Krylov methods only need the mat-vec).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass
class Matrix:
    """X as a scipy CSR matrix (binary pattern, FP64 ones) or a dense FP64 array."""
    X: object
    binary: bool

    @property
    def shape(self):
        return self.X.shape


def from_csr(n_rows, n_cols, row_ptr, col_idx) -> Matrix:
    data = np.ones(len(col_idx), dtype=np.float64)
    X = sp.csr_matrix((data, np.asarray(col_idx, np.int64), np.asarray(row_ptr, np.int64)),
                      shape=(n_rows, n_cols))
    return Matrix(X, True)


def from_dense(X) -> Matrix:
    return Matrix(np.asarray(X, dtype=np.float64), False)


def csc_pattern(n_rows, n_cols, row_ptr, col_idx):
    """CSC of a CSR pattern by a stable counting sort on the column index:
    rows stay in ascending order within each column. Returns (col_ptr, row_idx)."""
    col_idx = np.asarray(col_idx, np.int64)
    rows = np.repeat(np.arange(n_rows, dtype=np.int64), np.diff(np.asarray(row_ptr)))
    order = np.argsort(col_idx, kind="stable")
    col_ptr = np.zeros(n_cols + 1, dtype=np.int64)
    np.cumsum(np.bincount(col_idx, minlength=n_cols), out=col_ptr[1:])
    return col_ptr, rows[order].astype(np.int32)


def X_mv(M: Matrix, v):
    return M.X @ v


def Xt_mv(M: Matrix, u):
    return M.X.T @ u


def apply_A(M: Matrix, lam: float, v):
    """(X^T X + lambda I) v, Eq. (1)."""
    return Xt_mv(M, X_mv(M, v)) + lam * v


def rhs(M: Matrix, y):
    """b = X^T y, the right-hand side of Eq. (1)."""
    return Xt_mv(M, y)


def dense_A(M: Matrix, lam: float):
    """A formed explicitly: only for tiny test inputs."""
    X = M.X.toarray() if M.binary else M.X
    return X.T @ X + lam * np.eye(X.shape[1])


def col_sq_norms(M: Matrix):
    """diag(X^T X): column nnz for binary X, sum of squares for dense X."""
    if M.binary:
        return np.asarray(M.X.getnnz(axis=0), dtype=np.float64)
    return np.einsum("ij,ij->j", M.X, M.X)


def gershgorin_rowsums(M: Matrix):
    """Row sums of |X^T X|: |X|^T (|X| 1)."""
    absX = abs(M.X)
    return absX.T @ (absX @ np.ones(M.shape[1]))
