"""GPU parity of leader-follower clustering (rr_options.clustering =
RR_CLUSTER_LEADER; Section 3.4, Algorithm 1) against the oracle's
sequential loop (oracle/leader.py): the leaders and every label bit for bit
(integer distances, strict comparison with tol2, the earliest leader on
ties), on cases with a ragged last step of 64 features, tolerances from
"every feature leads" to a few large clusters; then a two-level solve on
that clustering against the exact solution, and the capacity error.
"""
import numpy as np
import pytest

from gen import synth
from oracle import leader, twolevel
from oracle import sparse as osp

import solution_ref

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_05826_gb300 import build
    build.build_library()
    from paper_1806_05826_gb300 import rr as rrmod
    rrmod.load()
    return rrmod


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


CASES = [("zipf_2000x1000", 2000, 1000, 0.01, 0, (0.0, 2.0, 5.0, 10.0, 20.0)),
         ("ragged_3001x1777", 3001, 1777, 0.006, 5, (3.0, 8.5)),
         ("dense_rows_800x333", 800, 333, 0.2, 7, (30.0, 80.0, 200.0)),
         ("zipf_12000x4000", 12000, 4000, 0.004, 9, (12.0,))]


@pytest.mark.parametrize("name,N,F,dens,seed,tols", CASES, ids=[c[0] for c in CASES])
def test_leaders_and_labels_bit_exact(rr, name, N, F, dens, seed, tols):
    X = synth.zipf_binary(N, F, dens, 1.1, seed)
    for tol2 in tols:
        L, lab = leader.leader_follower_binary(N, F, X.row_ptr, X.col_idx, tol2)
        h = rr.rr_setup(X.row_ptr, X.col_idx, N, F, 1e-2, F, seed=seed,
                        clustering=rr.RR_CLUSTER_LEADER, lf_tol2=tol2)
        q = rr.rr_query(h)
        assert q["k_eff"] == len(L), (tol2, q["k_eff"], len(L))
        centers = rr.rr_get_centers(h, F)
        assert np.array_equal(centers[:len(L)], L), tol2
        assert np.all(centers[len(L):] == -1)
        assert np.array_equal(rr.rr_get_labels(h), lab), tol2
        rr.rr_free(h)


def test_solve_on_leader_clusters(rr):
    """The two-level PCG on the leader-follower clustering: within the
    solution bar of the exact solution, and the oracle's cycle on the same
    clusters needs the same iterations."""
    N, F, lam, tol2 = 2000, 1000, 1e-2, 10.0
    X = synth.zipf_binary(N, F, 0.01, 1.1, 0)
    y, _ = synth.ridge_targets(X, 0)
    L, lab = leader.leader_follower_binary(N, F, X.row_ptr, X.col_idx, tol2)
    ref = twolevel.from_labels(N, F, X.row_ptr, X.col_idx, lam, lab, centers=L)
    for prec in (rr.RR_PREC_FP64, rr.RR_PREC_MIXED):
        h = rr.rr_setup(X.row_ptr, X.col_idx, N, F, lam, F, clustering=rr.RR_CLUSTER_LEADER,
                        lf_tol2=tol2, precision=prec)
        w = torch.empty(F, dtype=torch.float64, device="cuda")
        info = rr.rr_solve(h, dev(y), w, tol=1e-8)
        assert info["status"] == "RR_OK" and info["true_rel_res"] <= 1e-8
        b = osp.rhs(ref.M, y)
        w_ref, snaps = solution_ref.exact_solution(ref, b)
        solution_ref.check(w.cpu().numpy(), w_ref, snaps[1e-8], f"leader-follower, prec {prec}")
        rr.rr_free(h)


def test_leader_capacity_error(rr):
    X = synth.zipf_binary(2000, 1000, 0.01, 1.1, 0)
    L, _ = leader.leader_follower_binary(2000, 1000, X.row_ptr, X.col_idx, 5.0)
    with pytest.raises(rr.RRError) as e:
        rr.rr_setup(X.row_ptr, X.col_idx, 2000, 1000, 1e-2, len(L) - 1,
                    clustering=rr.RR_CLUSTER_LEADER, lf_tol2=5.0)
    assert e.value.status == rr.RR_UNSUPPORTED
    h = rr.rr_setup(X.row_ptr, X.col_idx, 2000, 1000, 1e-2, len(L),
                    clustering=rr.RR_CLUSTER_LEADER, lf_tol2=5.0)
    assert rr.rr_query(h)["k_eff"] == len(L)
