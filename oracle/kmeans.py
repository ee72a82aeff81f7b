"""Oracle: k-means++ clustering of the features (Section 3.4, "K-means++").

Test infrastructure only. Thin ctypes wrappers over kmeans_exact.c, which
holds the arithmetic (exact integer arithmetic for binary X, fixed-order
FP64 for dense X); see that file's header for every rule (draws, ties, empty
clusters, stopping).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _clib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> int:
    """Threads of the Lloyd assignment step (n < 1: all cores); returns the count."""
    return int(_clib.lib().oracle_set_threads(int(n)))


def splitmix64(seed: int, t: int) -> int:
    """Output t (from 0) of SplitMix64 seeded with `seed`."""
    return int(_clib.lib().oracle_splitmix64(seed & 0xFFFFFFFFFFFFFFFF, t))


def kmeanspp_binary(n_rows, n_cols, row_ptr, col_idx, col_ptr, row_idx, k, seed):
    """K-means++ seeding: k distinct feature ids (Section 3.4)."""
    rp, ci = np.ascontiguousarray(row_ptr, np.int64), np.ascontiguousarray(col_idx, np.int32)
    cp, ri = np.ascontiguousarray(col_ptr, np.int64), np.ascontiguousarray(row_idx, np.int32)
    out = np.empty(k, dtype=np.int32)
    rc = _clib.lib().oracle_kmeanspp_binary(n_rows, n_cols, _p(rp), _p(ci), _p(cp), _p(ri),
                                            k, seed & 0xFFFFFFFFFFFFFFFF, _p(out))
    if rc != 0:
        raise ValueError("k-means++ seeding failed (k out of range)")
    return out


def lloyd_binary(n_rows, n_cols, row_ptr, col_idx, col_ptr, row_idx, centers, max_iter):
    """Lloyd iterations from the given centres. Returns (labels int32[F], iterations)."""
    rp, ci = np.ascontiguousarray(row_ptr, np.int64), np.ascontiguousarray(col_idx, np.int32)
    cp, ri = np.ascontiguousarray(col_ptr, np.int64), np.ascontiguousarray(row_idx, np.int32)
    centers = np.ascontiguousarray(centers, np.int32)
    labels = np.empty(n_cols, dtype=np.int32)
    iters = np.zeros(1, dtype=np.int32)
    rc = _clib.lib().oracle_lloyd_binary(n_rows, n_cols, _p(rp), _p(ci), _p(cp), _p(ri),
                                         len(centers), _p(centers), max_iter, _p(labels),
                                         _p(iters))
    if rc != 0:
        raise ValueError("invalid centres (out of range or repeated)")
    return labels, int(iters[0])


def kmeanspp_dense(X, k, seed):
    X = np.ascontiguousarray(X, np.float32)
    out = np.empty(k, dtype=np.int32)
    rc = _clib.lib().oracle_kmeanspp_dense(X.shape[0], X.shape[1], _p(X), k,
                                           seed & 0xFFFFFFFFFFFFFFFF, _p(out))
    if rc != 0:
        raise ValueError("k-means++ seeding failed")
    return out


def lloyd_dense(X, centers, max_iter):
    X = np.ascontiguousarray(X, np.float32)
    centers = np.ascontiguousarray(centers, np.int32)
    labels = np.empty(X.shape[1], dtype=np.int32)
    iters = np.zeros(1, dtype=np.int32)
    rc = _clib.lib().oracle_lloyd_dense(X.shape[0], X.shape[1], _p(X), len(centers),
                                        _p(centers), max_iter, _p(labels), _p(iters))
    if rc != 0:
        raise ValueError("invalid centres")
    return labels, int(iters[0])


def compact(labels):
    """Drop empty clusters, keeping the order of the others.
    Returns (labels in [0, k_eff), sizes n_S int64[k_eff])."""
    labels = np.asarray(labels, np.int64)
    used = np.unique(labels)
    remap = np.full(int(labels.max()) + 1, -1, dtype=np.int64)
    remap[used] = np.arange(len(used))
    new = remap[labels]
    return new.astype(np.int32), np.bincount(new, minlength=len(used)).astype(np.int64)
