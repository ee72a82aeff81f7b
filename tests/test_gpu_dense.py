"""GPU parity for dense X (row-major FP32 values, the AR(1) design of the
dense experiments, Sec. 5): k-means++ centres and Lloyd labels bit-exact
against the oracle (both sum rows in blocks of 64, in FP64, in the same order),
the Galerkin coarse operator and the Jacobi weight to rounding, the operator
and right-hand side, and two-level solves (FP64 and mixed precision) against
the oracle's solves. Definition 1's duplicated-feature design checks the
clustering against a property that does not depend on the oracle."""
import numpy as np
import pytest

from gen import synth
from oracle import krylov, twolevel
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


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


# (N, F, k, lambda, seed): several 64-row blocks with a ragged tail, F not a
# multiple of the thread blocks, k above and below 8
CASES = {"ar1_3000x400": (3000, 400, 12, 1e-2, 0),
         "ar1_1037x211": (1037, 211, 5, 1.0, 1),
         "ar1_700x96": (700, 96, 96 // 4, 1e-3, 2)}


@pytest.fixture(scope="module", params=list(CASES))
def case(request, rr):
    N, F, k, lam, seed = CASES[request.param]
    X = synth.dense_ar1(N, F, 0.9, seed)
    y, _ = synth.ridge_targets(X, seed)
    ref = twolevel.setup_dense(X, lam, k, seed=seed)
    h = rr.rr_setup_dense(X, lam, k, seed=seed)
    return dict(X=X, y=y, ref=ref, h=h, lam=lam, k=k, seed=seed)


def test_dense_kmeanspp_centres_bit_exact(case, rr):
    assert np.array_equal(rr.rr_get_centers(case["h"], case["k"]), case["ref"].centers)


def test_dense_lloyd_labels_bit_exact(case, rr):
    assert np.array_equal(rr.rr_get_labels(case["h"]), case["ref"].labels)
    assert rr.rr_query(case["h"])["k_eff"] == case["ref"].k_eff
    w = torch.empty(case["X"].shape[1], dtype=torch.float64, device="cuda")
    info = rr.rr_solve(case["h"], dev(case["y"]), w, tol=1e-8)
    assert info["kmeans_iters"] == case["ref"].kmeans_iters


def test_dense_coarse_operator_and_omega(case, rr):
    """A_c = P^T X^T X P + lambda I: sums of N products in FP64 in another
    order, so equal to ~N eps relative to the largest entry."""
    Ac, G = rr.rr_get_coarse(case["h"])
    assert G is None
    want = case["ref"].Ac
    assert np.max(np.abs(Ac - want)) <= 1e-12 * np.abs(want).max()
    om = rr.rr_query(case["h"])["omega"]
    assert abs(om - case["ref"].omega) <= 1e-13 * case["ref"].omega


def test_dense_operator_rhs_matvec(case, rr):
    X, ref = case["X"], case["ref"]
    F = X.shape[1]
    v = np.random.default_rng(1).standard_normal(F)
    out = torch.empty(F, dtype=torch.float64, device="cuda")
    rr.rr_apply(case["h"], dev(v), out)
    want = ref.A(v)
    assert np.max(np.abs(out.cpu().numpy() - want)) <= 1e-12 * np.abs(want).max()
    b = torch.empty(F, dtype=torch.float64, device="cuda")
    rr.rr_rhs(case["h"], dev(case["y"]), b)
    bw = osp.rhs(ref.M, case["y"])
    assert np.max(np.abs(b.cpu().numpy() - bw)) <= 1e-12 * np.abs(bw).max()
    u = torch.empty(X.shape[0], dtype=torch.float64, device="cuda")
    rr.rr_matvec(case["h"], dev(v), u)
    uw = X.astype(np.float64) @ v
    assert np.max(np.abs(u.cpu().numpy() - uw)) <= 1e-12 * np.abs(uw).max()


@pytest.mark.parametrize("F", [8192, 8196, 8200])
def test_dense_operator_one_and_two_pass(rr, F):
    """F = 8192 takes the one-pass kernel with 8 column groups per thread;
    8196 and 8200 have too many groups and take the two-pass form (and 8196
    is a multiple of 4, 8200 too: the group count decides). Both precisions
    against X^T (X v) + lambda v in FP64."""
    X = synth.dense_ar1(333, F, 0.9, 6)
    v = np.random.default_rng(3).standard_normal(F)
    want = X.T.astype(np.float64) @ (X.astype(np.float64) @ v) + 0.5 * v
    for prec, tol in ((rr.RR_PREC_FP64, 1e-12), (rr.RR_PREC_MIXED, 1e-5)):
        h = rr.rr_setup_dense(X, 0.5, 2, seed=0, precision=prec)
        out = torch.empty(F, dtype=torch.float64, device="cuda")
        rr.rr_apply(h, dev(v), out)
        assert np.linalg.norm(out.cpu().numpy() - want) <= tol * np.linalg.norm(want)


def test_dense_operator_mixed_precision(case, rr):
    """FP32 products and sums inside each block, FP64 across blocks: relative
    error of a few FP32 roundings per term times the growth of the sums."""
    X, ref = case["X"], case["ref"]
    h = rr.rr_setup_dense(X, case["lam"], case["k"], seed=case["seed"], precision=rr.RR_PREC_MIXED)
    v = np.random.default_rng(4).standard_normal(X.shape[1])
    out = torch.empty(X.shape[1], dtype=torch.float64, device="cuda")
    rr.rr_apply(h, dev(v), out)
    want = ref.A(v)
    assert np.linalg.norm(out.cpu().numpy() - want) <= 1e-5 * np.linalg.norm(want)


def test_dense_preconditioner(case, rr):
    ref = case["ref"]
    r = np.random.default_rng(2).standard_normal(case["X"].shape[1])
    z = torch.empty(len(r), dtype=torch.float64, device="cuda")
    rr.rr_precondition(case["h"], dev(r), z)
    want = ref.apply(r)
    tol = max(1e-12, 1e-15 * np.linalg.cond(ref.Ac))
    assert np.linalg.norm(z.cpu().numpy() - want) / np.linalg.norm(want) <= tol


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_dense_two_level_solve(case, rr, prec):
    """Residual 1e-8 (recomputed by the oracle's operator) and a solution
    within the solution bar of the exact one (tests/solution_ref.py)."""
    X, ref = case["X"], case["ref"]
    b = osp.rhs(ref.M, case["y"])
    if prec == "fp64":
        h = case["h"]
    else:
        h = rr.rr_setup_dense(X, case["lam"], case["k"], seed=case["seed"],
                              precision=rr.RR_PREC_MIXED, max_restarts=20)
    w = torch.empty(X.shape[1], dtype=torch.float64, device="cuda")
    info = rr.rr_solve(h, dev(case["y"]), w, tol=1e-8)
    assert info["status"] == "RR_OK"
    wg = w.cpu().numpy()
    want = krylov.pcg(ref.A, ref.apply, b, tol=1e-8)
    r_gpu = np.linalg.norm(b - ref.A(wg))
    assert r_gpu / np.linalg.norm(b) <= 1e-8
    w_ref, _ = solution_ref.exact_solution(ref, b, snap_tols=())
    solution_ref.check(wg, w_ref, want.w, f"dense {prec}")
    if prec == "fp64":
        assert abs(info["iters"] - want.iters) <= max(2, 0.05 * want.iters)
    else:
        assert info["iters"] <= 2 * want.iters + 20


def test_dense_duplicated_features_recover_groups(rr):
    """Definition 1: with every column of a 16-column base repeated 3..9 times
    and k = 16, k-means++ never picks a copy of a chosen column (its distance
    is zero), so each group holds one centre and Lloyd puts every copy with its
    own group's centre: the labels are the groups up to renaming, and the
    coarse space holds the exact solution's group structure."""
    base = synth.dense_ar1(900, 16, 0.5, 7)
    counts = 3 + (np.arange(16) * 5) % 7
    X, groups = synth.duplicated_features(base, counts)
    h = rr.rr_setup_dense(X, 1e-2, 16, seed=3)
    labels = rr.rr_get_labels(h)
    assert rr.rr_query(h)["k_eff"] == 16
    pairs = set(zip(groups.tolist(), labels.tolist()))
    assert len(pairs) == 16 and len({g for g, _ in pairs}) == 16 and len({l for _, l in pairs}) == 16
    y, _ = synth.ridge_targets(X, 5)
    w = torch.empty(X.shape[1], dtype=torch.float64, device="cuda")
    info = rr.rr_solve(h, dev(y), w, tol=1e-8)
    assert info["status"] == "RR_OK" and info["true_rel_res"] <= 1e-8


def test_dense_given_centres_match_oracle(rr):
    X = synth.dense_ar1(1500, 300, 0.9, 4)
    centers = np.array([0, 37, 150, 151, 299, 64, 200], np.int32)
    ref = twolevel.setup_dense(X, 1e-2, len(centers), centers=centers)
    h = rr.rr_setup_dense(X, 1e-2, len(centers), init_centers=centers)
    assert np.array_equal(rr.rr_get_labels(h), ref.labels)


def test_dense_device_input_and_rejections(rr):
    X = synth.dense_ar1(500, 64, 0.9, 5)
    h = rr.rr_setup_dense(dev(X, torch.float32), 1e-2, 4, seed=0)
    ref = twolevel.setup_dense(X, 1e-2, 4, seed=0)
    assert np.array_equal(rr.rr_get_labels(h), ref.labels)
    Y = dev(np.zeros((1, 500)))
    W = torch.empty((1, 1, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(rr.RRError):
        rr.rr_solve_batch(h, Y, [1e-2], W)


def test_many_mixes_dense_and_binary(rr):
    """rr_solve_many over dense and binary problems in one graph equals the
    single solves bit for bit."""
    hs, ys, ws = [], [], []
    for i, (N, F) in enumerate([(2000, 300), (800, 150)]):
        X = synth.dense_ar1(N, F, 0.9, 10 + i)
        y, _ = synth.ridge_targets(X, 10 + i)
        hs.append(rr.rr_setup_dense(X, 1e-2, 6, seed=i))
        ys.append(dev(y))
        ws.append(torch.empty(F, dtype=torch.float64, device="cuda"))
    Xb = synth.zipf_binary(3000, 900, 0.01, 1.1, 3)
    yb, _ = synth.ridge_targets(Xb, 3)
    hs.append(rr.rr_setup(Xb.row_ptr, Xb.col_idx, 3000, 900, 1e-2, 9, seed=3))
    ys.append(dev(yb))
    ws.append(torch.empty(900, dtype=torch.float64, device="cuda"))
    out = rr.rr_solve_many(hs, ys, ws, tol=1e-8)
    assert out["status"] == "RR_OK"
    for h, y, w, info in zip(hs, ys, ws, out["infos"]):
        w1 = torch.empty_like(w)
        single = rr.rr_solve(h, y, w1, tol=1e-8)
        assert torch.equal(w1, w) and single["iters"] == info["iters"]
