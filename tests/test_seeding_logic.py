"""Two facts the GPU clustering relies on, checked on the CPU.

(1) The k-means++ rounds skip the overlap count of a feature whose distance
cannot drop: D2(i, c) = |x_i XOR x_c| >= |n_i - n_c|, so a feature with
d2_i <= |n_i - n_c| keeps d2_i, and its overlap may be taken as 0 (the update's
n_i + n_c - 2 * 0 >= d2_i leaves d2_i unchanged). A numpy restatement of the
rounds with that skip must give the same d2 and the same nearest centres as the
rounds without it, on every round.

(2) The first Lloyd step from singleton clusters {c_S} assigns each feature to
its nearest centre (score n_{c_S} - 2 |x_i AND x_{c_S}| = D2(i, c_S) - n_i, ties
to the smallest S), so the GPU takes those labels from the seeding: the oracle's
own Lloyd step from the oracle's centres must give exactly the nearest centres.
"""
import numpy as np

from gen import synth
from oracle import kmeans as okm
from oracle import sparse as osp


def dense_binary(X):
    A = np.zeros((X.n_rows, X.n_cols), dtype=np.int64)
    for r in range(X.n_rows):
        A[r, X.col_idx[X.row_ptr[r]:X.row_ptr[r + 1]]] = 1
    return A


def rounds(A, centers, skip):
    """d2 and nearest centre after each round, with or without the size skip."""
    n = A.sum(axis=0)
    d2 = near = None
    out = []
    for t, c in enumerate(centers):
        ov = A.T @ A[:, c]
        if skip and t > 0:
            ov = np.where(d2 > np.abs(n - n[c]), ov, 0)
        dist = n + n[c] - 2 * ov
        if t == 0:
            d2, near = dist.copy(), np.zeros(len(n), np.int64)
        else:
            better = dist < d2
            near = np.where(better, t, near)
            d2 = np.minimum(d2, dist)
        out.append((d2.copy(), near.copy()))
    return out


def test_size_bound_skip_changes_no_distance():
    for seed, (N, F, dens, k) in enumerate([(300, 200, 0.05, 20), (500, 120, 0.2, 30),
                                             (80, 400, 0.03, 60)]):
        X = synth.zipf_binary(N, F, dens, 1.1, seed)
        A = dense_binary(X)
        cp, ri = osp.csc_pattern(N, F, X.row_ptr, X.col_idx)
        centers = okm.kmeanspp_binary(N, F, X.row_ptr, X.col_idx, cp, ri, k, seed)
        full, skipped = rounds(A, centers, False), rounds(A, centers, True)
        for t, ((d_f, n_f), (d_s, n_s)) in enumerate(zip(full, skipped)):
            assert np.array_equal(d_f, d_s), (seed, t)
            assert np.array_equal(n_f, n_s), (seed, t)
        # the skip did prune: some overlaps were not needed
        n = A.sum(axis=0)
        assert any((full[t - 1][0] <= np.abs(n - n[c])).any() for t, c in enumerate(centers) if t)


def test_first_lloyd_step_is_the_nearest_centre():
    for seed, (N, F, dens, k) in enumerate([(2000, 1000, 0.01, 50), (600, 300, 0.05, 40)]):
        X = synth.zipf_binary(N, F, dens, 1.1, seed)
        A = dense_binary(X)
        cp, ri = osp.csc_pattern(N, F, X.row_ptr, X.col_idx)
        centers = okm.kmeanspp_binary(N, F, X.row_ptr, X.col_idx, cp, ri, k, seed)
        labels, iters = okm.lloyd_binary(N, F, X.row_ptr, X.col_idx, cp, ri, centers, 1)
        assert iters == 1
        # nearest centre by D2, ties to the smallest S (argmin takes the first)
        n = A.sum(axis=0)
        ov = A.T @ A[:, centers]                      # F x k overlaps
        d2 = n[:, None] + n[centers][None, :] - 2 * ov
        assert np.array_equal(labels, np.argmin(d2, axis=1)), seed
