"""Strength of the oracle's pins (CPU only).

Each case plants one plausible mistake in the oracle (a dropped term, a wrong
scale, sign, index or orientation, a missing step) by patching it for the
duration of the test, then runs the pins that guard that part of the oracle:
at least one of them must fail. The mistakes live here, in the tests, and
only while a case runs; the oracle itself is untouched.
"""
import dataclasses
import importlib.util
import os

import numpy as np
import pytest

from oracle import kmeans as km
from oracle import krylov, mlp
from oracle import sparse as osp
from oracle import twolevel as tl

_spec = importlib.util.spec_from_file_location(
    "_oracle_pins", os.path.join(os.path.dirname(__file__), "test_oracle_pins.py"))
pins = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(pins)


def _some_pin_fails(checks):
    for check in checks:
        try:
            check()
        except Exception:   # an assertion, or an error the mistake provokes
            return True
    return False


# ---- the planted mistakes -------------------------------------------------

def _apply_A_without_lambda(mp):
    mp.setattr(osp, "apply_A", lambda M, lam, v: osp.Xt_mv(M, osp.X_mv(M, v)))


def _dcg_without_diagonal(mp):
    mp.setattr(krylov, "dcg", lambda A, d, b, **kw: krylov.cg(A, b, **kw))


def _csc_rows_reversed(mp):
    orig = osp.csc_pattern

    def bad(n_rows, n_cols, row_ptr, col_idx):
        cp, ri = orig(n_rows, n_cols, row_ptr, col_idx)
        ri = ri.copy()
        for j in range(n_cols):
            ri[cp[j]:cp[j + 1]] = ri[cp[j]:cp[j + 1]][::-1]
        return cp, ri
    mp.setattr(osp, "csc_pattern", bad)


def _scale_without_sqrt(mp):
    mp.setattr(tl, "prolong_scale", lambda n_S: 1.0 / np.asarray(n_S, np.float64))


def _restrict_without_scale(mp):
    mp.setattr(tl, "restrict", lambda labels, s, r: np.bincount(labels, weights=r,
                                                                minlength=len(s)))


def _prolong_wrong_cluster(mp):
    mp.setattr(tl, "prolong", lambda labels, s, e: s[labels] * e[(labels + 1) % len(s)])


def _coarse_operator_without_lambda(mp):
    orig = tl.coarse_operator_binary
    mp.setattr(tl, "coarse_operator_binary", lambda G, s, lam: orig(G, s, 0.0) + 1e-12 * np.eye(len(s)))


def _gram_without_diagonal(mp):
    orig = tl.coarse_gram_binary

    def bad(*a):
        G = orig(*a)
        return G - np.diag(np.diag(G)) + np.eye(len(G), dtype=G.dtype)
    mp.setattr(tl, "coarse_gram_binary", bad)


def _cholesky_transposed(mp):
    orig = tl.cholesky
    mp.setattr(tl, "cholesky", lambda A: orig(A).T)


def _coarse_solve_forward_only(mp):
    mp.setattr(tl, "chol_solve", lambda L, b: tl.forward_sub(L, b))


def _gershgorin_diagonal_only(mp):
    mp.setattr(osp, "gershgorin_rowsums", lambda M: osp.col_sq_norms(M))


def _cycle_without_coarse_correction(mp):
    mp.setattr(tl.TwoLevel, "coarse_correction", lambda self, r1: np.zeros(self.k_eff))


def _cycle_without_post_smoothing(mp):
    def pre_only(self, r):
        z1 = self.omega * r / self.d
        e_c = self.coarse_correction(r - self.A(z1))
        return z1 + tl.prolong(self.labels, self.s, e_c)
    mp.setattr(tl.TwoLevel, "apply", pre_only)


def _pcg_steepest_descent(mp):
    def core(A, Minv, b, target, max_iter, history, bnorm):
        x, r = np.zeros_like(b), b.copy()
        if np.linalg.norm(r) <= target:
            return x, r, 0
        for it in range(1, max_iter + 1):
            p = Minv(r)          # the mistake: no conjugation against the last direction
            q = A(p)
            alpha = (r @ p) / (p @ q)
            x += alpha * p
            r -= alpha * q
            rn = np.linalg.norm(r)
            history.append(rn / bnorm)
            if rn <= target:
                return x, r, it
        return x, r, max_iter
    mp.setattr(krylov, "_pcg_core", core)


def _rougher_one_step(mp):
    orig = tl.TwoLevel.apply_tlfcg
    mp.setattr(tl.TwoLevel, "apply_tlfcg", lambda self, r, steps=2: orig(self, r, steps=1))


def _with_lambda_keeps_factor(mp):
    mp.setattr(tl.TwoLevel, "with_lambda", lambda self, lam: dataclasses.replace(self, lam=lam))


def _splitmix_counter_off_by_one(mp):
    orig = km.splitmix64
    mp.setattr(km, "splitmix64", lambda seed, t: orig(seed, t + 1))


def _lloyd_one_step(mp):
    orig = km.lloyd_binary
    mp.setattr(km, "lloyd_binary", lambda *a: orig(*a[:-1], 1))


def _lloyd_dense_one_step(mp):
    orig = km.lloyd_dense
    mp.setattr(km, "lloyd_dense", lambda X, centers, max_iter: orig(X, centers, 1))


def _seeding_uniform(mp):
    def uniform(n, f, rp, ci, cp, ri, k, seed):
        return np.random.default_rng(seed).choice(f, size=k, replace=False).astype(np.int32)
    mp.setattr(km, "kmeanspp_binary", uniform)


def _compact_reversed(mp):
    def bad(labels):
        labels = np.asarray(labels, np.int64)
        used = np.unique(labels)[::-1]
        remap = np.full(int(labels.max()) + 1, -1, np.int64)
        remap[used] = np.arange(len(used))
        new = remap[labels]
        return new.astype(np.int32), np.bincount(new, minlength=len(used)).astype(np.int64)
    mp.setattr(km, "compact", bad)


def _mlp_gradient_sign(mp):
    orig = mlp.backward

    def bad(p, X, T):
        g = orig(p, X, T)
        g["b2"] = -g["b2"]
        return g
    mp.setattr(mlp, "backward", bad)


def _adam_without_bias_correction(mp):
    def bad(p, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        for name in p:
            m = state.setdefault("m_" + name, np.zeros_like(p[name]))
            v = state.setdefault("v_" + name, np.zeros_like(p[name]))
            m *= b1
            m += (1.0 - b1) * g[name]
            v *= b2
            v += (1.0 - b2) * g[name] ** 2
            p[name] -= lr * m / (np.sqrt(v) + eps)
    mp.setattr(mlp, "adam_step", bad)


def _correction_not_rescaled(mp):
    mp.setattr(mlp, "coarse_correction", lambda p, rc: mlp.forward(p, rc[None, :])[0][0])


def _fcg_without_orthogonalisation(mp):
    def bad(A, Minv, b, m=1, tol=1e-8, max_iter=10000, on_step=None):
        b = np.asarray(b, np.float64)
        bnorm = float(np.linalg.norm(b))
        x, r, hist, it = np.zeros_like(b), b.copy(), [], 0
        while it < max_iter and np.linalg.norm(r) > tol * bnorm:
            p = Minv(r, it)      # the mistake: p is not A-orthogonalised against earlier p
            q = A(p)
            alpha = (p @ r) / (p @ q)
            x += alpha * p
            r -= alpha * q
            it += 1
            hist.append(float(np.linalg.norm(r)) / bnorm)
        return krylov.Result(x, it, float(np.linalg.norm(r)) / bnorm,
                             float(np.linalg.norm(b - A(x))) / bnorm, hist)
    mp.setattr(krylov, "fcg", bad)


def _harvest_target_without_smoothing(mp):
    from oracle import learned

    def bad(two, b, w_ref, n_iter):
        b = np.asarray(b, np.float64)
        w, r, xs, ts, p, rho_old = np.zeros_like(b), b.copy(), [], [], None, None
        for _ in range(n_iter):
            z1 = two.omega * r / two.d
            xs.append(tl.restrict(two.labels, two.s, r - two.A(z1)))
            ts.append(tl.restrict(two.labels, two.s, w_ref - w))   # the mistake: z1 not removed
            z = two.apply(r)
            rho = r @ z
            p = z.copy() if p is None else z + (rho / rho_old) * p
            q = two.A(p)
            alpha = rho / (p @ q)
            w, r, rho_old = w + alpha * p, r - alpha * q, rho
        return np.array(xs), np.array(ts)
    mp.setattr(learned, "harvest_pairs", bad)


def _dense_seeding_uniform(mp):
    def uniform(X, k, seed):
        return np.random.default_rng(seed).choice(np.shape(X)[1], size=k,
                                                  replace=False).astype(np.int32)
    mp.setattr(km, "kmeanspp_dense", uniform)


def _dense_coarse_operator_with_averaging(mp):
    def bad(X, labels, s, lam):
        n_S = np.rint(1.0 / s ** 2).astype(np.int64)
        Xc = X @ tl.averaging_dense(labels, n_S)     # the mistake: P~ (1/n_S) in place of P
        return Xc.T @ Xc + lam * np.eye(len(s))
    mp.setattr(tl, "coarse_operator_dense", bad)


def _eigen_inverse_without_lambda(mp):
    from oracle import eigen
    mp.setattr(eigen, "coarse_solve", lambda mu, Q, lam, rc: Q @ ((Q.T @ rc) / mu))
    mp.setattr(eigen, "coarse_inverse", lambda mu, Q, lam: (Q / mu[None, :]) @ Q.T)


def _jacobi_stops_on_cancelled_norm(mp):
    """The off-diagonal norm taken as ||A||^2 - sum diag^2 (cancellation: a
    premature stop), a mistake the oracle once made: the oracle's own loop,
    with that one line changed."""
    import inspect
    import textwrap
    from oracle import eigen
    src = textwrap.dedent(inspect.getsource(eigen.jacobi_eigh))
    good = "off = np.linalg.norm(A - np.diag(np.diag(A)))"
    assert good in src
    src = src.replace(good, "off = np.sqrt(max(0.0, np.sum(A * A) - np.sum(np.diag(A) ** 2)))")
    ns = {"np": np}
    exec(src, ns)
    mp.setattr(eigen, "jacobi_eigh", ns["jacobi_eigh"])


def _jacobi_rotation_sign(mp):
    from oracle import eigen
    orig_sqrt = np.sqrt

    def bad(S, tol=1e-15, max_sweeps=50):
        A = np.array(S, dtype=np.float64, copy=True)
        n = A.shape[0]
        Q = np.eye(n)
        for _ in range(max_sweeps):
            for p in range(n - 1):
                for q in range(p + 1, n):
                    if A[p, q] == 0.0:
                        continue
                    tau = (A[q, q] - A[p, p]) / (2.0 * A[p, q])
                    t = -(1.0 if tau >= 0.0 else -1.0) / (abs(tau) + orig_sqrt(1.0 + tau * tau))
                    c = 1.0 / orig_sqrt(1.0 + t * t)
                    s = t * c
                    J = np.eye(n)
                    J[p, p] = J[q, q] = c
                    J[p, q], J[q, p] = s, -s
                    A = J.T @ A @ J
                    Q = Q @ J
        return np.diag(A).copy(), Q, max_sweeps
    mp.setattr(eigen, "jacobi_eigh", lambda S, tol=1e-15, max_sweeps=50: bad(S, tol, 3))


def _bayes_patched(mp, fn_name, good, bad):
    """One line of an oracle/bayes.py function changed, the rest as it is."""
    import inspect
    import textwrap
    from oracle import bayes
    src = textwrap.dedent(inspect.getsource(getattr(bayes, fn_name)))
    assert good in src
    ns = dict(vars(bayes))
    exec(src.replace(good, bad), ns)
    mp.setattr(bayes, fn_name, ns[fn_name])


def _gamma_times_rate(mp):
    _bayes_patched(mp, "gamma_draw", "return d * v / rate", "return d * v * rate")


def _gamma_without_cube(mp):
    _bayes_patched(mp, "gamma_draw", "v = t * t * t", "v = t * t")


def _noise_e2_times_tau(mp):
    _bayes_patched(mp, "noise_sample", "+ e2 / tau", "+ e2 * tau")


def _noise_e1_unscaled(mp):
    _bayes_patched(mp, "noise_sample", "synth.normal(seed, 2 * step, N) / math.sqrt(tau)",
                   "synth.normal(seed, 2 * step, N)")


def _lambda_rate_without_half(mp):
    _bayes_patched(mp, "gibbs", "p.beta + 0.5 * float(w @ w)", "p.beta + float(w @ w)")


def _tau_shape_without_half_n(mp):
    _bayes_patched(mp, "gibbs", "p.a_tau + 0.5 * N", "p.a_tau + N")


def _metric_gradient_ignored(mp):
    _orig = mlp.backward
    mp.setattr(mlp, "backward", lambda p, X, T, W=None: _orig(p, X, T))


def _metric_loss_transposed_side(mp):
    _orig = mlp.loss

    def bad(p, X, T, W=None):
        if W is None:
            return _orig(p, X, T)
        o, _ = mlp.forward(p, X)
        D = o - T
        return 0.5 * np.sum(D @ W) / X.shape[0]   # sums W's rows instead of the quadratic form
    mp.setattr(mlp, "loss", bad)


def _leader_patched(mp, good, bad):
    import inspect
    import textwrap
    from oracle import leader
    src = textwrap.dedent(inspect.getsource(leader.leader_follower_binary))
    assert good in src
    ns = dict(vars(leader))
    exec(src.replace(good, bad), ns)
    mp.setattr(leader, "leader_follower_binary", ns["leader_follower_binary"])


def _leader_non_strict(mp):
    _leader_patched(mp, "if float(d2[s]) < tol2:", "if float(d2[s]) <= tol2:")


def _leader_last_minimum(mp):
    _leader_patched(mp, "s = int(np.argmin(d2))", "s = int(len(d2) - 1 - np.argmin(d2[::-1]))")


def _leader_without_overlap(mp):
    _leader_patched(mp, "d2 = n_i + n_lead[:L] - 2 * overlap", "d2 = n_i + n_lead[:L] - overlap")


P = pins
CASES = [
    ("leader-follower joins at d^2 = tol^2", _leader_non_strict,
     [lambda: P.test_leader_follower_worked_example(2.0, [0, 2, 4], [0, 0, 1, 0, 2])]),
    ("leader-follower takes the last of tied leaders", _leader_last_minimum,
     [P.test_leader_follower_characterisation]),
    ("leader-follower distance with a single overlap term", _leader_without_overlap,
     [P.test_leader_follower_characterisation, P.test_leader_follower_recovers_duplicated_features]),
    ("gamma draw multiplied by the rate", _gamma_times_rate, [P.test_gamma_draw_distribution]),
    ("gamma draw with (1 + c x)^2", _gamma_without_cube, [P.test_gamma_draw_distribution]),
    ("noise e2 multiplied by tau", _noise_e2_times_tau,
     [P.test_noise_injected_sample_has_the_conditional_posterior_moments]),
    ("noise e1 without the tau^-1/2 scale", _noise_e1_unscaled,
     [P.test_noise_injected_sample_has_the_conditional_posterior_moments]),
    ("lambda rate without the 1/2", _lambda_rate_without_half,
     [P.test_gibbs_chain_recovers_the_generating_precisions]),
    ("tau shape with N instead of N/2", _tau_shape_without_half_n,
     [P.test_gibbs_chain_recovers_the_generating_precisions]),
    ("eigen coarse inverse without lambda", _eigen_inverse_without_lambda,
     [P.test_eigen_coarse_inverse_equals_cholesky_solve_at_every_lambda]),
    ("Jacobi stops on a cancelled off-diagonal norm", _jacobi_stops_on_cancelled_norm,
     [P.test_jacobi_eigh_against_library_eigh,
      P.test_eigen_coarse_inverse_equals_cholesky_solve_at_every_lambda]),
    ("Jacobi rotation angle of the wrong sign", _jacobi_rotation_sign,
     [P.test_jacobi_eigh_against_library_eigh, P.test_eigen_theorem1_spectrum]),
    ("dense seeding uniform instead of D^2", _dense_seeding_uniform,
     [P.test_kmeanspp_dense_draw_follows_d2_weights]),
    ("dense coarse operator from the averaging operator", _dense_coarse_operator_with_averaging,
     [lambda: P.test_galerkin_coarse_operator(0)]),
    ("FCG without A-orthogonalisation", _fcg_without_orthogonalisation,
     [P.test_fcg_truncation_rule, P.test_fcg_matches_pcg_for_fixed_spd_preconditioner]),
    ("harvest target without the smoothing step", _harvest_target_without_smoothing,
     [P.test_harvest_pairs_first_two_iterations_closed_form]),
    ("apply_A drops lambda", _apply_A_without_lambda,
     [P.test_apply_A_matches_dense, P.test_single_feature_closed_form]),
    ("DCG without the diagonal", _dcg_without_diagonal,
     [P.test_disjoint_supports_diagonal_system]),
    ("CSC rows out of order", _csc_rows_reversed, [P.test_csc_is_stable_transpose]),
    ("P scaled by 1/n_S", _scale_without_sqrt,
     [P.test_prolongation_orthonormal_and_averaging, lambda: P.test_galerkin_coarse_operator(0)]),
    ("restriction without the scale", _restrict_without_scale,
     [P.test_prolongation_orthonormal_and_averaging, P.test_coarse_correction_exact_on_coarse_space]),
    ("prolongation from the wrong cluster", _prolong_wrong_cluster,
     [P.test_prolongation_orthonormal_and_averaging, P.test_cycle_error_propagation_is_T]),
    ("coarse operator without lambda", _coarse_operator_without_lambda,
     [lambda: P.test_galerkin_coarse_operator(0)]),
    ("Gram without its diagonal", _gram_without_diagonal,
     [P.test_coarse_counts_and_integer_gram_by_brute_force,
      lambda: P.test_galerkin_coarse_operator(0)]),
    ("Cholesky factor transposed", _cholesky_transposed, [P.test_cholesky_against_library]),
    ("coarse solve without the back substitution", _coarse_solve_forward_only,
     [P.test_cholesky_against_library, P.test_coarse_correction_exact_on_coarse_space]),
    ("damping bound from the diagonal only", _gershgorin_diagonal_only,
     [P.test_gershgorin_rowsums_by_brute_force, P.test_omega_below_spectral_bound]),
    ("cycle without the coarse correction", _cycle_without_coarse_correction,
     [P.test_coarse_correction_exact_on_coarse_space, P.test_cycle_error_propagation_is_T]),
    ("cycle without post-smoothing", _cycle_without_post_smoothing,
     [P.test_cycle_error_propagation_is_T, lambda: P.test_preconditioner_spd(0)]),
    ("PCG without conjugation", _pcg_steepest_descent,
     [P.test_fcg_matches_pcg_for_fixed_spd_preconditioner]),
    ("rougher with one CG step", _rougher_one_step, [P.test_rougher_is_two_step_krylov_minimiser]),
    ("lambda change keeps the old factor", _with_lambda_keeps_factor,
     [P.test_with_lambda_equals_fresh_setup_with_same_clustering]),
    ("SplitMix64 counter off by one", _splitmix_counter_off_by_one,
     [P.test_splitmix64_published_output]),
    ("Lloyd stops after one step", _lloyd_one_step,
     [P.test_lloyd_fixed_point_at_exit, lambda: P.test_lloyd_matches_brute_force(0)]),
    ("dense Lloyd stops after one step", _lloyd_dense_one_step,
     [lambda: P.test_lloyd_dense_matches_exact_arithmetic(0), P.test_dense_kmeans_recovers_groups]),
    ("seeding uniform instead of D^2", _seeding_uniform,
     [P.test_kmeanspp_picks_other_group, P.test_kmeanspp_draw_follows_d2_weights]),
    ("compaction reverses the cluster order", _compact_reversed,
     [P.test_compact_drops_empty_clusters_in_order]),
    ("metric ignored in the gradient", _metric_gradient_ignored,
     [P.test_mlp_metric_gradients_finite_differences]),
    ("metric loss without the quadratic form", _metric_loss_transposed_side,
     [P.test_mlp_metric_loss_is_plain_loss_of_transformed_output]),
    ("a bias gradient with the wrong sign", _mlp_gradient_sign,
     [P.test_mlp_gradients_finite_differences]),
    ("Adam without bias correction", _adam_without_bias_correction,
     [P.test_adam_first_step_is_lr_times_sign]),
    ("learned correction not rescaled by ||r_c||", _correction_not_rescaled,
     [P.test_learned_correction_positively_homogeneous]),
]


@pytest.mark.parametrize("name,plant,checks", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_a_pin(name, plant, checks, monkeypatch):
    # the guarding pins pass on the oracle as it is ...
    for check in checks:
        check()
    # ... and at least one of them fails once the mistake is planted
    with monkeypatch.context() as mp:
        plant(mp)
        assert _some_pin_fails(checks), f"no pin caught: {name}"
