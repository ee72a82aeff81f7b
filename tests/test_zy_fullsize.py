"""GPU parity at the bench workload's full size: 200,000 x 100,000 binary Zipf
(density 0.2%, s = 1.1, seed 1), k = 1000, at every lambda of the workload
(1e-3, 1e-1, 10), in the configuration bench.py times (mixed precision, CUDA
graph loops, automatic gather choice, Lloyd until no label changes, up to 20
refinement restarts).

Every oracle quantity is computed by the oracle from the oracle's own
clustering (k-means++ and every Lloyd step, its assignment step on all host
cores):
- all k k-means++ centres, the number of Lloyd steps and the final labels:
  bit-exact (the steps whose update work passes the pull threshold run the
  per-feature pull kernel, the others the push; both are covered here);
- the integer Gram G = C^T C, every entry: exact (the oracle forms C by row
  blocks and multiplies in FP64, exact for these integers below 2^53);
- A_c and omega: bit-exact (the same IEEE operations on both sides);
- the operator: the FP64 handle to 1e-13 of the largest entry, the mixed
  handle within the FP32 summation bound;
- the preconditioner (FP64 handle) to cond(A_c) * 1e-15;
- the solves against the exact solution w_ref (the oracle's PCG to relative
  residual 1e-12, run in background processes while the GPU tests run): at
  tolerance 1e-8, mixed precision (as timed) and FP64, the true residual
  recomputed by the oracle is <= 1e-8 and ||w - w_ref|| / ||w_ref|| is within
  the bar of tests/solution_ref.py (max(1e-6, 25 x the oracle's own error at
  1e-8)); at tolerance 1e-10 (mixed precision) the error is <= 1e-6.
"""
import numpy as np
import pytest

from gen import synth
from oracle import kmeans as okm
from oracle import reference
from oracle import sparse as osp
from oracle import twolevel

import solution_ref

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

WORKLOAD = "zipf_200000x100000"
EPS = 2.0 ** -53


def oracle_state(X, p):
    """The oracle's setup: k-means++ centres, Lloyd labels (until no label
    changes, at most 50 steps, as on the GPU), the integer Gram (by blocks of
    rows, dense FP64 products), A_c, its factor, the Jacobi diagonal and
    omega."""
    N, F, lam, k, seed = X.n_rows, X.n_cols, p["lambdas"][0], p["k"], p["seed"]
    M = osp.from_csr(N, F, X.row_ptr, X.col_idx)
    cp, ri = osp.csc_pattern(N, F, X.row_ptr, X.col_idx)
    spec = (N, F, p["density"], p["s"], p["seed"])
    centers, raw, iters = solution_ref.oracle_clustering(spec, k, seed)
    labels, n_S = okm.compact(raw)
    k_eff = len(n_S)
    C = twolevel.coarse_counts(N, F, X.row_ptr, X.col_idx, labels, k_eff)
    G = np.zeros((k_eff, k_eff))
    for r0 in range(0, N, 20000):
        Cb = C[r0:r0 + 20000].toarray().astype(np.float64)
        G += Cb.T @ Cb
    assert G.max() < 2.0 ** 53
    G = G.astype(np.int64)
    s = twolevel.prolong_scale(n_S)
    Ac = twolevel.coarse_operator_binary(G, s, lam)
    d = osp.col_sq_norms(M) + lam
    omega = twolevel.jacobi_omega(M, d, lam)
    two = twolevel.TwoLevel(M, lam, labels, n_S, s, G, Ac, twolevel.cholesky(Ac), d, omega,
                            np.asarray(centers, np.int32), iters)
    return dict(two=two, centers=np.asarray(centers, np.int32), raw=raw, cmax=int(C.max()),
                col_len=int(np.diff(cp).max()), row_len=int(np.diff(X.row_ptr).max()))


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


TOLS = (1e-8, 1e-10)


@pytest.fixture(scope="module")
def full(rr):
    X, y, _, p = synth.workload(WORKLOAD)
    ref = oracle_state(X, p)
    # the exact solutions, one process per lambda, while the GPU tests run
    spec = (X.n_rows, X.n_cols, p["density"], p["s"], p["seed"])
    pool, pending = reference.start(spec, ref["raw"], [(lam, y) for lam in p["lambdas"]],
                                    snap_tols=TOLS)
    rp = torch.as_tensor(X.row_ptr, device="cuda")
    ci = torch.as_tensor(X.col_idx, device="cuda")
    lam, k, seed = p["lambdas"][0], p["k"], p["seed"]
    hm = rr.rr_setup(rp, ci, X.n_rows, X.n_cols, lam, k, seed=seed, precision=rr.RR_PREC_MIXED,
                     max_restarts=20)
    h64 = rr.rr_setup(rp, ci, X.n_rows, X.n_cols, lam, k, seed=seed, precision=rr.RR_PREC_FP64,
                      max_restarts=20)
    yield dict(X=X, y=y, p=p, ref=ref, hm=hm, h64=h64, pending=pending)
    pool.terminate()


def test_full_centres_and_labels_bit_exact(full, rr):
    ref = full["ref"]
    y = dev(full["y"])
    w = torch.empty(full["X"].n_cols, dtype=torch.float64, device="cuda")
    for h in (full["hm"], full["h64"]):
        assert np.array_equal(rr.rr_get_centers(h, full["p"]["k"]), ref["centers"])
        assert np.array_equal(rr.rr_get_labels(h), ref["two"].labels)
        assert rr.rr_query(h)["k_eff"] == ref["two"].k_eff
    info = rr.rr_solve(full["hm"], y, w, tol=1e-2)
    assert info["kmeans_iters"] == ref["two"].kmeans_iters


def test_full_gram_coarse_operator_and_omega(full, rr):
    two = full["ref"]["two"]
    Ac, G = rr.rr_get_coarse(full["hm"])
    assert np.array_equal(G, two.G)
    assert np.array_equal(Ac, two.Ac)
    assert rr.rr_query(full["hm"])["omega"] == two.omega


def test_full_operator(full, rr):
    X, two = full["X"], full["ref"]["two"]
    v = np.random.default_rng(1).standard_normal(X.n_cols)
    want = two.A(v)
    out = torch.empty(X.n_cols, dtype=torch.float64, device="cuda")
    rr.rr_apply(full["h64"], dev(v), out)
    assert np.max(np.abs(out.cpu().numpy() - want)) <= 1e-13 * np.abs(want).max()
    # FP32 gathers: v and u rounded to FP32 and summed in FP32 over at most
    # row_len + col_len terms per output; |error_i| <= gamma (|X|^T |X| |v|)_i
    rr.rr_apply(full["hm"], dev(v), out)
    n = full["ref"]["row_len"] + full["ref"]["col_len"] + 4
    gamma = n * 2.0 ** -24 / (1 - n * 2.0 ** -24)
    bound = gamma * osp.apply_A(two.M, 0.0, np.abs(v)) + 1e-13 * np.abs(want).max()
    assert np.all(np.abs(out.cpu().numpy() - want) <= bound)


def test_full_preconditioner(full, rr):
    X, two = full["X"], full["ref"]["two"]
    r = np.random.default_rng(2).standard_normal(X.n_cols)
    z = torch.empty(X.n_cols, dtype=torch.float64, device="cuda")
    rr.rr_precondition(full["h64"], dev(r), z)
    want = two.apply(r)
    tol = max(1e-12, 1e-15 * np.linalg.cond(two.Ac))
    rel = np.linalg.norm(z.cpu().numpy() - want) / np.linalg.norm(want)
    assert rel <= tol, (rel, tol)


def test_full_solves_match_exact_solution(full, rr):
    X, y, p, two = full["X"], full["y"], full["p"], full["ref"]["two"]
    M = two.M
    b = osp.rhs(M, y)
    bn = np.linalg.norm(b)
    n = full["ref"]["row_len"] + full["ref"]["col_len"] + 4
    w = torch.empty(X.n_cols, dtype=torch.float64, device="cuda")
    yd = dev(y)
    exact = full["pending"].get()
    for lam, (w_ref, snaps, it_ref, rel_ref) in zip(p["lambdas"], exact):
        assert rel_ref <= reference.TOL_REF
        for h, tol in ((full["hm"], 1e-8), (full["h64"], 1e-8), (full["hm"], 1e-10)):
            rr.rr_set_lambda(h, lam)
            info = rr.rr_solve(h, yd, w, tol=tol)
            assert info["status"] == "RR_OK" and info["true_rel_res"] <= tol
            wg = w.cpu().numpy()
            res = np.linalg.norm(b - osp.apply_A(M, lam, wg))
            # two FP64 evaluations of b - A w in different orders differ by at
            # most about n eps (|X|^T |X| |w| + lambda |w| + |b|) per entry
            slack = 2 * n * EPS * np.linalg.norm(osp.apply_A(M, lam, np.abs(wg)) + np.abs(b))
            assert res <= tol * bn + slack, (lam, res / bn, slack / bn)
            if tol == 1e-8:
                solution_ref.check(wg, w_ref, snaps[1e-8], f"lambda {lam}")
            else:
                assert solution_ref.rel_err(wg, w_ref) <= 1e-6, lam
