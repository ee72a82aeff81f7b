"""GPU parity of the coarse solve by eigendecomposition (RR_COARSE_EIGEN):
X_c^T X_c = Q diag(mu) Q^T once per clustering, A_c(lambda)^-1 =
Q diag(1/(mu + lambda)) Q^T for every lambda (Section 4's decomposition of
X_c reused across beta).

Against the oracle (oracle/eigen.py, cyclic Jacobi in its textbook
row-cyclic order; the GPU uses the parallel round-robin order, so rounding
differs): the spectrum to 1e-12 of its largest eigenvalue (Jacobi is
backward stable: each eigenvalue moves by at most ~k eps ||G_s||); Q
orthogonal and Q diag(mu) Q^T = G_s to 1e-12 relative; the preconditioner
M^-1 r of an eigen handle against the oracle's (Cholesky) cycle to
cond(A_c) 1e-15; solves at several lambda within the solution bar of
tests/solution_ref.py; the batched solve with the eigen factors.
"""
import numpy as np
import pytest

from gen import synth
from oracle import eigen, krylov, twolevel
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


CASES = {"zipf_2000x1000": (2000, 1000, 0.01, 50, 1e-2, 0),
         "ragged_3001x1777_k37": (3001, 1777, 0.006, 37, 1e-3, 5)}


@pytest.fixture(scope="module", params=list(CASES))
def case(request, rr):
    N, F, dens, k, lam, seed = CASES[request.param]
    X = synth.zipf_binary(N, F, dens, 1.1, seed)
    y, _ = synth.ridge_targets(X, seed)
    ref = twolevel.setup_binary(N, F, X.row_ptr, X.col_idx, lam, k, seed=seed)
    h = rr.rr_setup(X.row_ptr, X.col_idx, N, F, lam, k, seed=seed, coarse=rr.RR_COARSE_EIGEN)
    Gs = eigen.coarse_gram_scaled(ref.G, ref.s)
    mu_o, Q_o, sweeps_o = eigen.jacobi_eigh(Gs)
    return dict(X=X, y=y, ref=ref, h=h, lam=lam, k=k, seed=seed, Gs=Gs, mu_o=mu_o)


def test_eigen_spectrum_and_vectors(case, rr):
    mu, Q, sweeps = rr.rr_get_eigen(case["h"])
    mu_o, Gs = case["mu_o"], case["Gs"]
    assert 1 <= sweeps <= 30
    assert np.allclose(np.sort(mu), np.sort(mu_o), rtol=0, atol=1e-12 * np.abs(mu_o).max())
    k = len(mu)
    assert np.abs(Q.T @ Q - np.eye(k)).max() <= 1e-12
    assert np.abs((Q * mu) @ Q.T - Gs).max() <= 1e-12 * np.abs(Gs).max()


def test_eigen_preconditioner_matches_oracle(case, rr):
    ref = case["ref"]
    r = np.random.default_rng(4).standard_normal(case["X"].n_cols)
    z = torch.empty_like(dev(r))
    rr.rr_precondition(case["h"], dev(r), z)
    want = ref.apply(r)
    tol = max(1e-12, 1e-15 * np.linalg.cond(ref.Ac))
    assert np.linalg.norm(z.cpu().numpy() - want) / np.linalg.norm(want) <= tol


def test_eigen_solves_at_several_lambda(case, rr):
    """rr_set_lambda on an eigen handle forms A_c^-1 from the kept
    decomposition; every solve is within the solution bar of the exact one."""
    X, ref = case["X"], case["ref"]
    w = torch.empty(X.n_cols, dtype=torch.float64, device="cuda")
    for lam in (case["lam"], 1e-3, 0.3, 30.0):
        rr.rr_set_lambda(case["h"], lam)
        refl = ref.with_lambda(lam)
        b = osp.rhs(refl.M, case["y"])
        w_ref, snaps = solution_ref.exact_solution(refl, b)
        info = rr.rr_solve(case["h"], dev(case["y"]), w, tol=1e-8)
        assert info["status"] == "RR_OK" and info["true_rel_res"] <= 1e-8
        solution_ref.check(w.cpu().numpy(), w_ref, snaps[1e-8], f"eigen, lambda {lam}")
        # the same preconditioner as the Cholesky form: the same iteration count
        want = krylov.pcg(refl.A, refl.apply, b, tol=1e-8)
        assert abs(info["iters"] - want.iters) <= max(2, 0.05 * want.iters)
    rr.rr_set_lambda(case["h"], case["lam"])


def test_eigen_batched_solve(case, rr):
    X = case["X"]
    Y, _ = synth.ridge_targets_many(X, [300, 301])
    lams = (1e-3, 1e-1, 3.0)
    W = torch.empty((len(lams), 2, X.n_cols), dtype=torch.float64, device="cuda")
    out = rr.rr_solve_batch(case["h"], dev(Y), lams, W, tol=1e-8)
    assert out["status"] == "RR_OK"
    Wh = W.cpu().numpy()
    for l, lam in enumerate(lams):
        refl = case["ref"].with_lambda(lam)
        for j in range(2):
            b = osp.rhs(refl.M, Y[j])
            w_ref, snaps = solution_ref.exact_solution(refl, b)
            solution_ref.check(Wh[l, j], w_ref, snaps[1e-8], f"batched eigen ({l}, {j})")


def test_eigen_dense_handle(rr):
    """Dense X: the same decomposition of its coarse Gram."""
    Xd = synth.dense_ar1(1500, 120, 0.9, 2)
    lam, k = 1e-2, 12
    h = rr.rr_setup_dense(Xd, lam, k, seed=2, coarse=rr.RR_COARSE_EIGEN)
    ref = twolevel.setup_dense(Xd, lam, k, seed=2)
    mu, Q, _ = rr.rr_get_eigen(h)
    Gs = ref.Ac - lam * np.eye(ref.k_eff)
    assert np.abs((Q * mu) @ Q.T - Gs).max() <= 1e-12 * np.abs(Gs).max()
    y = np.random.default_rng(3).standard_normal(1500)
    w = torch.empty(120, dtype=torch.float64, device="cuda")
    info = rr.rr_solve(h, dev(y), w, tol=1e-10)
    b = osp.rhs(ref.M, y)
    exact = np.linalg.solve(osp.dense_A(ref.M, lam), b)
    assert info["status"] == "RR_OK"
    assert solution_ref.rel_err(w.cpu().numpy(), exact) <= 1e-6
