"""GPU parity of rr_solve_many: independent problems of uneven sizes in one
graph. Each problem is Eq. (1) for its own X, clustering and lambda, so the
oracle is the single-problem oracle (dense Cholesky solve on these sizes), and
rr_solve on the same handle is the same kernels in the same order: the
solutions must be identical bit for bit, whatever runs beside them."""
import numpy as np
import pytest

from gen import synth
from oracle import sparse as osp

import solution_ref
from oracle import twolevel

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


# uneven problems: (n, d, density, seed); k = max(2, d // 100), lambda = 1e-2
PROBLEMS = [(1200, 300, 0.02, 0), (5000, 1900, 0.004, 1), (800, 650, 0.01, 2),
            (3000, 1100, 0.007, 3), (9000, 400, 0.003, 4)]


@pytest.fixture(scope="module", params=[0, 1], ids=["fp64", "mixed"])
def many(request, rr):
    prec = rr.RR_PREC_FP64 if request.param == 0 else rr.RR_PREC_MIXED
    probs = []
    for (n, d, dens, seed) in PROBLEMS:
        X = synth.zipf_binary(n, d, dens, 1.1, seed)
        y, _ = synth.ridge_targets(X, 100 + seed)
        h = rr.rr_setup(X.row_ptr, X.col_idx, n, d, 1e-2, max(2, d // 100), seed=seed,
                        precision=prec, max_restarts=20)
        probs.append(dict(X=X, y=y, h=h, seed=seed))
    ys = [dev(p["y"]) for p in probs]
    ws = [torch.empty(p["X"].n_cols, dtype=torch.float64, device="cuda") for p in probs]
    out = rr.rr_solve_many([p["h"] for p in probs], ys, ws, tol=1e-8)
    for p, w in zip(probs, ws):
        p["w"] = w.cpu().numpy()
    return dict(probs=probs, out=out)


def test_many_equals_single_solves(many, rr):
    assert many["out"]["status"] == "RR_OK"
    for p, info in zip(many["probs"], many["out"]["infos"]):
        w = torch.empty(p["X"].n_cols, dtype=torch.float64, device="cuda")
        single = rr.rr_solve(p["h"], dev(p["y"]), w, tol=1e-8)
        assert np.array_equal(w.cpu().numpy(), p["w"])
        assert single["iters"] == info["iters"] and single["restarts"] == info["restarts"]


def test_many_matches_exact_solutions(many):
    for p, info in zip(many["probs"], many["out"]["infos"]):
        X = p["X"]
        M = osp.from_csr(X.n_rows, X.n_cols, X.row_ptr, X.col_idx)
        b = osp.rhs(M, p["y"])
        r = np.linalg.norm(b - osp.apply_A(M, 1e-2, p["w"]))
        assert r <= 1e-8 * np.linalg.norm(b) and info["true_rel_res"] <= 1e-8
        w_ref, snaps = solution_ref.for_problem(X, p["y"], 1e-2, max(2, X.n_cols // 100),
                                                p["seed"])
        solution_ref.check(p["w"], w_ref, snaps[1e-8], f"problem {p['seed']}")


def test_many_rejects_shared_handles(many, rr):
    p = many["probs"][0]
    w = torch.empty(p["X"].n_cols, dtype=torch.float64, device="cuda")
    with pytest.raises(rr.RRError):
        rr.rr_solve_many([p["h"], p["h"]], [dev(p["y"])] * 2, [w, w], tol=1e-8)


def test_capped_problem_keeps_its_cap_when_others_restart(rr):
    """A problem that stops on its iteration cap is left as it is while the
    graph is relaunched for the refinement restarts of the others: its
    iterate and count equal those of rr_solve with the same cap."""
    hs, ys, ws, Xs = [], [], [], []
    for j, (n, d, dens, seed) in enumerate(PROBLEMS[:2]):
        X = synth.zipf_binary(n, d, dens, 1.1, seed)
        y, _ = synth.ridge_targets(X, 100 + seed)
        hs.append(rr.rr_setup(X.row_ptr, X.col_idx, n, d, 1e-2, max(2, d // 100), seed=seed,
                              precision=rr.RR_PREC_MIXED, max_restarts=20,
                              max_iter=5 if j == 0 else 20000))
        ys.append(dev(y))
        ws.append(torch.empty(d, dtype=torch.float64, device="cuda"))
        Xs.append(X)
    out = rr.rr_solve_many(hs, ys, ws, tol=1e-8)
    capped, free = out["infos"]
    assert out["status"] == "RR_NOT_CONVERGED"
    assert capped["iters"] == 5 and free["true_rel_res"] <= 1e-8
    w = torch.empty(Xs[0].n_cols, dtype=torch.float64, device="cuda")
    single = rr.rr_solve(hs[0], ys[0], w, tol=1e-8)
    assert single["status"] == "RR_NOT_CONVERGED" and single["iters"] == 5
    assert np.array_equal(w.cpu().numpy(), ws[0].cpu().numpy())
    if free["restarts"] == 0:
        pytest.skip("the uncapped problem took no restart, so the graph was not relaunched")


def test_many_tight_tolerance_within_1e6(many, rr):
    """At relative residual 1e-10 every problem of the graph is within 1e-6 of
    its exact solution."""
    probs = many["probs"]
    ws = [torch.empty(p["X"].n_cols, dtype=torch.float64, device="cuda") for p in probs]
    out = rr.rr_solve_many([p["h"] for p in probs], [dev(p["y"]) for p in probs], ws, tol=1e-10)
    assert out["status"] == "RR_OK"
    for p, w in zip(probs, ws):
        X = p["X"]
        M = osp.from_csr(X.n_rows, X.n_cols, X.row_ptr, X.col_idx)
        exact = np.linalg.solve(osp.dense_A(M, 1e-2), osp.rhs(M, p["y"]))
        assert solution_ref.rel_err(w.cpu().numpy(), exact) <= 1e-6, p["seed"]
