"""The seeded input generators: the shapes and distributions the workloads
claim (binary Zipf columns, AR(1) dense features, targets y = X w* + noise),
and that every array is a pure function of its seed."""
import math

import numpy as np

from gen import synth


def test_uniform_and_normal_moments():
    u = synth.uniform(3, 0, 200_000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / u.size)
    z = synth.normal(3, 1, 200_000)
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2 / z.size)
    # the tails of a normal: P(|z| > 2) = 0.0455
    assert abs(np.mean(np.abs(z) > 2) - 0.0455) < 0.003


def test_draws_are_functions_of_seed_stream_and_index():
    a = synth.uniform(7, 2, 1000)
    assert np.array_equal(a, synth.uniform(7, 2, 1000))
    assert np.array_equal(a[300:], synth.uniform(7, 2, 700, offset=300))
    assert not np.array_equal(a, synth.uniform(8, 2, 1000))
    assert not np.array_equal(a, synth.uniform(7, 3, 1000))


def test_zipf_probs_sum_to_density_and_follow_the_power_law():
    F, dens, s = 5000, 0.002, 1.1
    q = synth.zipf_column_probs(F, dens, s)
    assert abs(q.sum() - dens * F) < 1e-9 * dens * F
    assert np.all(np.diff(q) <= 0) and q.max() <= 1.0
    # below the cap, q_j (j + 1)^s is one constant
    free = q < 1.0
    c = q[free] * (np.arange(1, F + 1)[free] ** s)
    assert np.allclose(c, c[0], rtol=1e-12)


def test_zipf_probs_saturate_at_one_for_dense_heads():
    q = synth.zipf_column_probs(100, 0.3, 1.1)
    assert q[0] == 1.0 and abs(q.sum() - 30.0) < 1e-9


def test_zipf_binary_is_a_valid_pattern_with_the_stated_column_frequencies():
    N, F, dens, s = 20_000, 3000, 0.005, 1.1
    X = synth.zipf_binary(N, F, dens, s, seed=5)
    rp, ci = X.row_ptr, X.col_idx
    assert rp[0] == 0 and rp[-1] == ci.size and np.all(np.diff(rp) >= 0)
    assert ci.dtype == np.int32 and ci.min() >= 0 and ci.max() < F
    # strictly increasing within each row (no repeated entry)
    rows = np.repeat(np.arange(N), np.diff(rp))
    same_row = rows[1:] == rows[:-1]
    assert np.all(np.diff(ci.astype(np.int64))[same_row] > 0)
    # each column's count is Binomial(N, q_rank): standardised residuals ~ N(0, 1)
    q = synth.zipf_column_probs(F, dens, s)
    perm = np.argsort(synth.raw64(5, 1, F), kind="stable")
    counts = np.bincount(ci, minlength=F)[perm]
    var = N * q * (1 - q)
    ok = var > 0
    zs = (counts[ok] - N * q[ok]) / np.sqrt(var[ok])
    assert abs(zs.mean()) < 5 / math.sqrt(zs.size)
    assert abs(zs.var() - 1.0) < 0.2
    assert np.abs(zs).max() < 6.0
    # and the whole matrix has the requested density
    assert abs(X.nnz - dens * N * F) < 5 * math.sqrt(dens * N * F)


def test_zipf_binary_rows_of_a_column_are_independent_of_the_row_index():
    # geometric skipping places a column's rows uniformly: the head column's
    # members split evenly between the two halves of the rows
    N = 40_000
    X = synth.zipf_binary(N, 500, 0.02, 1.1, seed=2)
    rows = np.repeat(np.arange(N), np.diff(X.row_ptr))
    head = np.argsort(synth.raw64(2, 1, 500), kind="stable")[0]
    r = rows[X.col_idx == head]
    m = r.size
    assert m > 1000
    assert abs(np.sum(r < N // 2) - m / 2) < 5 * math.sqrt(m / 4)


def test_zipf_binary_is_a_function_of_its_seed():
    a = synth.zipf_binary(3000, 400, 0.01, 1.1, seed=9)
    b = synth.zipf_binary(3000, 400, 0.01, 1.1, seed=9)
    c = synth.zipf_binary(3000, 400, 0.01, 1.1, seed=10)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col_idx, b.col_idx)
    assert not (a.nnz == c.nnz and np.array_equal(a.col_idx, c.col_idx))


def test_dense_ar1_has_unit_variance_and_geometric_correlation():
    rho = 0.9
    X = synth.dense_ar1(20_000, 12, rho, seed=1).astype(np.float64)
    assert X.dtype == np.float64 and X.shape == (20_000, 12)
    v = X.var(axis=0)
    assert np.all(np.abs(v - 1.0) < 0.06)
    C = np.corrcoef(X, rowvar=False)
    for lag in (1, 2, 5):
        c = np.diag(C, lag)
        assert np.all(np.abs(c - rho ** lag) < 0.03), (lag, c)


def test_ridge_targets_noise_level_and_signal():
    X = synth.zipf_binary(10_000, 800, 0.01, 1.1, seed=3)
    y, w_star = synth.ridge_targets(X, seed=3)
    assert w_star.shape == (800,) and y.shape == (10_000,)
    e = y - synth.csr_matvec(X, w_star)
    assert abs(e.std() - 0.1) < 0.005
    assert abs(e.mean()) < 5 * 0.1 / math.sqrt(e.size)
    # dense X takes the same w* and noise streams
    D = synth.dense_ar1(500, 40, 0.9, seed=4)
    yd, wd = synth.ridge_targets(D, seed=4)
    assert np.allclose(yd - D.astype(np.float64) @ wd, 0.1 * synth.normal(4, 11, 500))


def test_ridge_targets_many_matches_one_seed_at_a_time():
    X = synth.zipf_binary(2000, 300, 0.02, 1.1, seed=6)
    Y, W = synth.ridge_targets_many(X, [4, 5])
    for j, sd in enumerate([4, 5]):
        y, w = synth.ridge_targets(X, sd)
        assert np.array_equal(W[j], w)
        assert np.allclose(Y[j], y, rtol=0, atol=1e-12)


def test_duplicated_features_repeats_columns_by_group():
    base = np.arange(12.0).reshape(4, 3)
    X, groups = synth.duplicated_features(base, [2, 0, 3])
    assert groups.tolist() == [0, 0, 2, 2, 2]
    assert np.array_equal(X[:, 1], base[:, 0]) and np.array_equal(X[:, 4], base[:, 2])


def test_many_problem_parameters_lie_in_their_ranges():
    spec = synth.MANY_WORKLOADS["uneven_12_dense4"]
    ps = synth.many_params("uneven_12_dense4")
    assert len(ps) == spec["n_problems"] + spec["n_dense"]
    binary, dense = ps[:spec["n_problems"]], ps[spec["n_problems"]:]
    for q in binary:
        assert spec["n"][0] <= q["n"] < spec["n"][1]
        assert spec["d"][0] <= q["d"] < spec["d"][1]
        assert spec["density"][0] <= q["density"] < spec["density"][1]
        assert q["k"] == max(2, q["d"] // 100) and q["lam"] == spec["lam"]
    assert [q["seed"] for q in ps] == list(range(len(ps)))
    for q in dense:
        assert q["dense"] and (q["n"], q["d"]) == spec["dense"] and q["k"] == 40
    # the binary problems differ from one another
    assert len({(q["n"], q["d"]) for q in binary}) == len(binary)
    # the binary part of the set with dense problems is the plain set
    assert binary == synth.many_params("uneven_12")


def test_mlp_init_he_uniform_bounds():
    p = synth.mlp_init(64, 128, seed=1)
    assert p["W1"].shape == (128, 64) and p["W2"].shape == (128, 128) and p["W3"].shape == (64, 128)
    for name, fan_in in (("W1", 64), ("W2", 128), ("W3", 128)):
        bound = math.sqrt(6.0 / fan_in)
        W = p[name]
        assert np.abs(W).max() <= bound
        # uniform on [-bound, bound]: variance bound^2 / 3
        assert abs(W.var() - bound ** 2 / 3) < 0.05 * bound ** 2
    assert not np.any(p["b1"]) and not np.any(p["b2"]) and not np.any(p["b3"])
