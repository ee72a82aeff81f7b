"""rr_apply_noalloc: the operator without device allocation, for callers that
may not call cudaMalloc (a framework that owns all device memory through its
own pool, a path that cannot take cudaMalloc's implicit synchronisation).

Its output must equal the FP64 oracle's operator and the handle-based
rr_apply on two calls in a row with different matrices, so no state from one
call leaks into the next; after a warm-up call, a call must leave the device's
free memory and torch's allocation count unchanged. This file is collected
last on purpose: if it fails, a run that stops at the first failure has
already run every other test."""
import numpy as np
import pytest

from gen import synth
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


def _device_patterns(X):
    cp, ri = osp.csc_pattern(X.n_rows, X.n_cols, X.row_ptr, X.col_idx)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    return t(X.row_ptr), t(X.col_idx), t(cp), t(ri)


CASES = ((3001, 1777, 0.006, 5), (2000, 1000, 0.01, 0))


def test_noalloc_matches_oracle_and_handle_apply_twice(rr):
    lam = 0.37
    for N, F, dens, seed in CASES:          # two calls in a row, different matrices
        X = synth.zipf_binary(N, F, dens, 1.1, seed)
        v_np = np.random.default_rng(seed).standard_normal(F)
        ref = osp.apply_A(osp.from_csr(N, F, X.row_ptr, X.col_idx), lam, v_np)
        h = rr.rr_setup(X.row_ptr, X.col_idx, N, F, lam, 8, seed=seed)
        v = torch.as_tensor(v_np, device="cuda")
        want = torch.empty(F, dtype=torch.float64, device="cuda")
        rr.rr_apply(h, v, want)
        rp, ci, cp, ri = _device_patterns(X)
        got = torch.full((F,), np.nan, dtype=torch.float64, device="cuda")
        rr.rr_apply_noalloc(N, F, rp, ci, cp, ri, lam, v, got)
        torch.cuda.synchronize()
        w, g = want.cpu().numpy(), got.cpu().numpy()
        # FP64 sums of the same terms in another order: the handle path's
        # parity tolerance, against the oracle and against rr_apply
        assert np.max(np.abs(g - ref)) <= 1e-13 * np.abs(ref).max()
        assert np.max(np.abs(g - w)) <= 1e-13 * np.abs(w).max()
        rr.rr_free(h)


def test_noalloc_leaves_device_memory_unchanged(rr):
    lam = 0.5
    mats = []
    for N, F, dens, seed in CASES:
        X = synth.zipf_binary(N, F, dens, 1.1, seed)
        v = torch.as_tensor(np.random.default_rng(seed + 1).standard_normal(F), device="cuda")
        mats.append((N, F, _device_patterns(X), v, torch.empty(F, dtype=torch.float64,
                                                                device="cuda")))
    N, F, pat, v, out = mats[0]
    rr.rr_apply_noalloc(N, F, *pat, lam, v, out)       # warm-up: loads the module
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    N, F, pat, v, out = mats[1]                         # another matrix, other sizes
    rr.rr_apply_noalloc(N, F, *pat, lam, v, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.isfinite(out).all()


def test_noalloc_rejects_bad_arguments(rr):
    lib = rr.load()
    z = torch.zeros(4, dtype=torch.float64, device="cuda")
    z2 = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = torch.zeros(2, dtype=torch.int64, device="cuda")
    # the library's own row limit, through the C ABI directly: it refuses before
    # touching any buffer (the binding already refuses pointer arrays this short)
    st = lib.rr_apply_noalloc((1 << 22) + 1, 4, p.data_ptr(), p.data_ptr(), p.data_ptr(),
                              p.data_ptr(), 1.0, z.data_ptr(), z2.data_ptr(), None)
    assert st == rr.RR_UNSUPPORTED
    with pytest.raises(ValueError):
        rr.rr_apply_noalloc((1 << 22) + 1, 4, p, p.to(torch.int32), p, p.to(torch.int32), 1.0,
                            z, z2)
    # NULL index arrays are refused whatever nnz the pointer arrays imply
    for ci, ri in ((None, p.data_ptr()), (p.data_ptr(), None)):
        st = lib.rr_apply_noalloc(1, 4, p.data_ptr(), ci, p.data_ptr(), ri, 1.0, z.data_ptr(),
                                  z2.data_ptr(), None)
        assert st == rr.RR_INVALID_ARG
        assert b"NULL" in lib.rr_last_error()
