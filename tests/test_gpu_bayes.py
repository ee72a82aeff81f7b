"""GPU parity of the Gibbs sampler with noise injection (rr_bayes, Section 2,
Eq. (ni_xtx)) against the oracle's chain (oracle/bayes.py) on the same
counter-based draws.

The chain is a smooth function of its solves: the Gamma draws accept or
reject on the shape alone (fixed per chain), so a draw moves with its rate,
rate0 + ||v||^2 / 2, and a relative error e in a solution moves lambda and
tau by at most about 2 e. Step t inherits the earlier steps' errors through
lambda / tau and the noise scales, so the bar on the traces at step t is
(t + 1) 2 e_bar, e_bar the solution bar of tests/solution_ref.py
(max(1e-6, 25 e_oracle) at tol 1e-8, 1e-6 at tol 1e-10); the mean of w gets
n e_bar.
"""
import numpy as np
import pytest

from gen import synth
from oracle import bayes, twolevel
from oracle import sparse as osp

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


N, F, K, SEED = 2000, 1000, 50, 0
PARAMS = dict(alpha=1.0, beta=1.0, a_tau=1.0, b_tau=1.0, lambda0=1.0, tau0=1.0, seed=9)


@pytest.fixture(scope="module")
def problem():
    X = synth.zipf_binary(N, F, 0.01, 1.1, SEED)
    y, _ = synth.ridge_targets(X, SEED)
    ref = twolevel.setup_binary(N, F, X.row_ptr, X.col_idx, 1e-2, K, seed=SEED)
    return X, y, ref


def oracle_chain(ref, y, n, burnin, tol):
    p = bayes.Params(tol=tol, **PARAMS)
    return bayes.gibbs(ref, y, p, n, burnin)


def oracle_solution_errors(ref, y, lams, taus, tol):
    """The oracle's own solution error at each step against the dense solve."""
    A0 = osp.dense_A(ref.M, 0.0)
    lam, tau = PARAMS["lambda0"], PARAMS["tau0"]
    errs = []
    for t in range(len(lams)):
        res = bayes.noise_sample(ref, y, lam, tau, PARAMS["seed"], t, tol)
        e1 = synth.normal(PARAMS["seed"], 2 * t, N) / np.sqrt(tau)
        e2 = synth.normal(PARAMS["seed"], 2 * t + 1, F) * np.sqrt(lam)
        b = osp.rhs(ref.M, y + e1) + e2 / tau
        w = np.linalg.solve(A0 + (lam / tau) * np.eye(F), b)
        errs.append(np.linalg.norm(res.w - w) / np.linalg.norm(w))
        lam, tau = lams[t], taus[t]
    return np.array(errs)


def check_chain(got, want, e_bar, what):
    (lg, tg, wg, ig), (lw, tw, ww, iw) = got, want
    n = len(lw)
    for t in range(n):
        bar = (t + 1) * 2 * e_bar
        assert abs(lg[t] - lw[t]) <= bar * lw[t], f"{what}: lambda at step {t}"
        assert abs(tg[t] - tw[t]) <= bar * tw[t], f"{what}: tau at step {t}"
    err_w = np.linalg.norm(wg - ww) / np.linalg.norm(ww)
    assert err_w <= n * e_bar, f"{what}: mean of w {err_w:.3g}"
    print(f"{what}: lambda {np.max(np.abs(lg / lw - 1)):.3g} tau {np.max(np.abs(tg / tw - 1)):.3g} "
          f"w {err_w:.3g} iters {list(ig)} vs {list(iw)}")


@pytest.mark.parametrize("coarse", ["cholesky", "eigen"])
def test_bayes_chain_fp64(rr, problem, coarse):
    X, y, ref = problem
    n, burnin, tol = 6, 2, 1e-10
    c = rr.RR_COARSE_EIGEN if coarse == "eigen" else rr.RR_COARSE_CHOLESKY
    h = rr.rr_setup(X.row_ptr, X.col_idx, N, F, 1e-2, K, seed=SEED, coarse=c)
    wm = torch.empty(F, dtype=torch.float64, device="cuda")
    lg, tg, ig = rr.rr_bayes(h, dev(y), n, burnin, wm, tol=tol, **PARAMS)
    want = oracle_chain(ref, y, n, burnin, tol)
    check_chain((lg, tg, wm.cpu().numpy(), ig), want, 1e-6, f"FP64 {coarse}")
    assert np.all(np.abs(ig - np.array(want[3])) <= 2)
    # the handle's lambda is back
    assert rr.rr_query(h)["lambda"] == 1e-2


def test_bayes_chain_mixed_eigen(rr, problem):
    """The configuration the benchmark times: mixed precision, eigen coarse
    solve, tol 1e-8."""
    X, y, ref = problem
    n, burnin, tol = 6, 2, 1e-8
    h = rr.rr_setup(X.row_ptr, X.col_idx, N, F, 1e-2, K, seed=SEED, coarse=rr.RR_COARSE_EIGEN,
                    precision=rr.RR_PREC_MIXED)
    wm = torch.empty(F, dtype=torch.float64, device="cuda")
    lg, tg, ig = rr.rr_bayes(h, dev(y), n, burnin, wm, tol=tol, **PARAMS)
    want = oracle_chain(ref, y, n, burnin, tol)
    e_orc = oracle_solution_errors(ref, y, want[0], want[1], tol)
    check_chain((lg, tg, wm.cpu().numpy(), ig), want, max(1e-6, 25 * e_orc.max()), "mixed eigen")


def test_bayes_fixed_tau_and_arguments(rr, problem):
    X, y, ref = problem
    h = rr.rr_setup(X.row_ptr, X.col_idx, N, F, 1e-2, K, seed=SEED)
    p = dict(PARAMS, a_tau=0.0, tau0=50.0)
    lg, tg, _ = rr.rr_bayes(h, dev(y), 3, 0, None, tol=1e-10, **p)
    assert np.all(tg == 50.0)
    lw, tw, _, _ = bayes.gibbs(ref, y, bayes.Params(tol=1e-10, **p), 3)
    assert np.allclose(lg, lw, rtol=6e-6, atol=0)
    for bad in (dict(n_samples=0), dict(burnin=3), dict(burnin=-1), dict(alpha=0.0),
                dict(lambda0=-1.0), dict(tol=1.5)):
        kw = dict(n_samples=3, burnin=0)
        kw.update(bad)
        n_s, b_i = kw.pop("n_samples"), kw.pop("burnin")
        with pytest.raises((rr.RRError, ValueError)):
            rr.rr_bayes(h, dev(y), n_s, b_i, None, **dict(PARAMS, **kw))
