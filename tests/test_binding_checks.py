"""The Python binding refuses arguments that would let the library read or
write outside a buffer, or take a host address for a device one, before it
calls into the library. CPU only: every check fires before the first call."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_1806_05826_gb300 import rr  # noqa: E402


def handle(N=20, F=10, k=3):
    return rr.Handle(None, F, N, (), k)   # no library handle behind it


def test_vectors_must_be_cuda_tensors():
    h = handle()
    y, w = torch.zeros(20, dtype=torch.float64), torch.zeros(10, dtype=torch.float64)
    calls = [lambda: rr.rr_solve(h, y, w), lambda: rr.rr_solve_fcg(h, None, y, w),
             lambda: rr.rr_apply(h, w, w.clone()), lambda: rr.rr_precondition(h, w, w.clone()),
             lambda: rr.rr_rhs(h, y, w), lambda: rr.rr_matvec(h, w, y),
             lambda: rr.rr_solve_many([h], [y], [w]),
             lambda: rr.rr_solve_batch(h, y[None], [0.1], w[None, None]),
             lambda: rr.rr_harvest(h, y[None], 0.1, w[None], 1e-8, 3, 4, 3),
             lambda: rr.rr_solve(h, np.zeros(20), np.zeros(10))]
    for call in calls:
        with pytest.raises(TypeError, match="CUDA tensor"):
            call()


def test_tensor_checks_dtype_layout_and_size():
    t = torch.zeros(6, dtype=torch.float64)
    assert rr._dev(t, torch.float64, 6, "t", device="cpu") == t.data_ptr()
    with pytest.raises(TypeError, match="dtype"):
        rr._dev(t.float(), torch.float64, 6, "t", device="cpu")
    with pytest.raises(ValueError, match="contiguous"):
        rr._dev(torch.zeros(6, 2, dtype=torch.float64).t(), torch.float64, 6, "t", device="cpu")
    with pytest.raises(ValueError, match="at least 7"):
        rr._dev(t, torch.float64, 7, "t", device="cpu")


def test_setup_checks_host_csr_sizes():
    rp = np.array([0, 2, 3], np.int64)
    with pytest.raises(ValueError, match="row_ptr"):
        rr.rr_setup(rp, np.array([0, 1, 2], np.int32), 3, 3, 1.0, 1)       # N + 1 = 4 entries
    with pytest.raises(ValueError, match="col_idx"):
        rr.rr_setup(rp, np.array([0, 1], np.int32), 2, 3, 1.0, 1)          # nnz = 3
    with pytest.raises(TypeError, match="CUDA tensor"):
        rr.rr_setup(torch.as_tensor(rp), torch.tensor([0, 1, 2], dtype=torch.int32), 2, 3, 1.0, 1)
    with pytest.raises(ValueError, match="two-dimensional"):
        rr.rr_setup_dense(np.zeros(5, np.float32), 1.0, 1)
    with pytest.raises(TypeError, match="CUDA tensor"):
        rr.rr_setup_dense(torch.zeros((4, 3)), 1.0, 1)


def test_counts_and_shapes_match_the_handle():
    h = handle(k=3)
    with pytest.raises(ValueError, match="k = 3"):
        rr.rr_get_centers(h, 2)          # a 2-entry buffer for 3 centres
    with pytest.raises(ValueError, match="same length"):
        rr.rr_solve_many([h, handle()], [torch.zeros(20, dtype=torch.float64)], [])
    m = rr.Mlp(None, 5, 128)
    with pytest.raises(ValueError, match="shape"):
        rr.mlp_forward(m, torch.zeros((2, 4)))
    with pytest.raises(ValueError, match="shape"):
        rr.mlp_grad(m, torch.zeros((2, 5)), torch.zeros((3, 5)))
    with pytest.raises(ValueError, match="shape"):
        rr.mlp_train(m, torch.zeros((8, 5)), torch.zeros((8, 4)))


def test_noalloc_checks_pattern_lengths():
    # 3 rows, 2 columns, nnz = 3; the length checks fire before the device
    # checks, so host tensors reach them here
    rp = torch.tensor([0, 1, 2, 3], dtype=torch.int64)
    cp = torch.tensor([0, 2, 3], dtype=torch.int64)
    idx = torch.tensor([0, 1, 0], dtype=torch.int32)
    short = idx[:2].clone()
    v, out = torch.zeros(2, dtype=torch.float64), torch.zeros(2, dtype=torch.float64)
    with pytest.raises(ValueError, match="col_idx"):
        rr.rr_apply_noalloc(3, 2, rp, short, cp, idx, 1.0, v, out)
    with pytest.raises(ValueError, match="row_idx"):
        rr.rr_apply_noalloc(3, 2, rp, idx, cp, short, 1.0, v, out)
    with pytest.raises(ValueError, match="same pattern"):
        rr.rr_apply_noalloc(3, 2, rp, idx, torch.tensor([0, 2, 4]), idx, 1.0, v, out)
    with pytest.raises(ValueError, match="row_ptr"):
        rr.rr_apply_noalloc(4, 2, rp, idx, cp, idx, 1.0, v, out)
    with pytest.raises(TypeError, match="CUDA tensor"):   # lengths right: the device check
        rr.rr_apply_noalloc(3, 2, rp, idx, cp, idx, 1.0, v, out)
