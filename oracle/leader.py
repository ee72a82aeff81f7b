"""Oracle: leader-follower clustering of the features (Section 3.4, Algorithm 1).

Test infrastructure only.

Algorithm 1 visits the samples in order and keeps a growing set of leaders:
each sample is compared with every leader, and joins the nearest one when
that distance is below the tolerance, else it becomes a leader itself. Here
the samples are the F features (columns of the binary X), in index order, and
the leaders are never updated (Section 3.4: the paper's experiments keep the
leaders as they are, so that they stay sparse). Readings where the algorithm
leaves a choice:
  - the initial set of leaders is empty (feature 0 is the first leader);
  - the distance is Euclidean between binary columns, compared squared and
    exactly: d(i, c)^2 = n_i + n_c - 2 |R_i and R_c| (an integer; R_j the rows
    of column j, n_j = |R_j|), against tol2, the squared tolerance, as
    d^2 < tol2 in double precision (exact for every integer d^2 < 2^53);
  - the nearest leader is the one of smallest d^2, the earliest leader on ties.
Returns the leaders (feature ids, in creation order) and every feature's
cluster index (the position of its leader in that list).

Plain numpy: a dense 0/1 membership of the leaders' rows (N x leaders) gives
every overlap of a feature with all leaders as one column sum over its rows.
For small inputs only.
"""
from __future__ import annotations

import numpy as np

from . import sparse as osp


def leader_follower_binary(n_rows, n_cols, row_ptr, col_idx, tol2, max_leaders=None):
    col_ptr, row_idx = osp.csc_pattern(n_rows, n_cols, row_ptr, col_idx)
    col_ptr = np.asarray(col_ptr, np.int64)
    row_idx = np.asarray(row_idx, np.int64)
    cap = n_cols if max_leaders is None else max_leaders
    member = np.zeros((n_rows, min(cap, n_cols)), dtype=np.uint8)   # member[r, s]: r in R_leader(s)
    n_lead = np.zeros(min(cap, n_cols), dtype=np.int64)
    leaders = []
    labels = np.empty(n_cols, dtype=np.int32)
    for i in range(n_cols):
        rows = row_idx[col_ptr[i]:col_ptr[i + 1]]
        n_i = len(rows)
        L = len(leaders)
        if L:
            overlap = member[rows, :L].sum(axis=0, dtype=np.int64)
            d2 = n_i + n_lead[:L] - 2 * overlap
            s = int(np.argmin(d2))            # the first minimum: the earliest leader
            if float(d2[s]) < tol2:
                labels[i] = s
                continue
        if L == cap:
            raise ValueError(f"leader-follower: more than {cap} leaders at tol2 = {tol2}")
        leaders.append(i)
        member[rows, L] = 1
        n_lead[L] = n_i
        labels[i] = L
    return np.array(leaders, dtype=np.int32), labels
