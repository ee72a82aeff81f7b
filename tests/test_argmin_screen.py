"""The Lloyd assignment's FP32 screen (CPU emulation of its arithmetic).

The GPU argmin compares a cluster's exact score (Q_S - 2 n_S D_iS) / n_S^2 by
128-bit cross multiplication only when an FP32 bracket around it does not lie
wholly above the least upper bound seen so far (the warp-wide U). That is exact
only if every bracket [s - 16u m, s + 16u m] contains its exact score, with
s = fl(q - r d), m = fl(q + r d), q = fl(fl(Q) / fl(n n)), r = fl(2 / n),
u = 2^-24. This test rebuilds those FP32 values with numpy (the fused
multiply-adds through float64, where the FP32 product is exact) on random and
deliberately tied scores, runs the same screen, and checks against exact
integer arithmetic that the exact argmin (ties to the smallest S) always
survives, so the result equals the exact argmin.
"""
import numpy as np

U = 2.0 ** -24
TOL = np.float32(2.0 ** -20)


def f32(x):
    return np.float32(x)


def fma32(a, b, c):
    """fl32(a*b + c): the product of two FP32 values is exact in FP64."""
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def exact_better(x, y):
    """Is cluster x = (a, w, s) strictly preferable to y (score a/w, ties to smaller s)?"""
    if x[1] == 0:
        return False
    if y[1] == 0:
        return True
    lhs, rhs = x[0] * y[1], y[0] * x[1]
    return lhs < rhs if lhs != rhs else x[2] < y[2]


def screened_argmin(Q, n, D, lanes=32, batch=8):
    k = len(Q)
    q = [f32(np.inf) if n[s] == 0 else f32(f32(Q[s]) / (f32(n[s]) * f32(n[s]))) for s in range(k)]
    r = [f32(0.0) if n[s] == 0 else f32(f32(2.0) / f32(n[s])) for s in range(k)]
    best = [(0, 0, 1 << 30)] * lanes
    Ub = f32(np.inf)
    for s0 in range(0, k, lanes * batch):
        lo, hi = {}, f32(np.inf)
        for lane in range(lanes):
            for u in range(batch):
                s = s0 + lane + lanes * u
                if s >= k:
                    continue
                df = f32(D[s])
                with np.errstate(invalid="ignore"):
                    sc = fma32(-r[s], df, q[s])
                    m = fma32(r[s], df, q[s])
                    lo[s] = fma32(-TOL, m, sc)
                    hi = np.fmin(hi, fma32(TOL, m, sc))
        Ub = np.fmin(Ub, hi)
        for lane in range(lanes):
            for u in range(batch):
                s = s0 + lane + lanes * u
                if s >= k or not (lo[s] <= Ub) or n[s] == 0:
                    continue
                c = (Q[s] - 2 * n[s] * D[s], n[s] * n[s], s)
                if exact_better(c, best[lane]):
                    best[lane] = c
    out = best[0]
    for b in best[1:]:
        if exact_better(b, out):
            out = b
    return out[2]


def exact_argmin(Q, n, D):
    best = (0, 0, 1 << 30)
    for s in range(len(Q)):
        if n[s] == 0:
            continue
        c = (Q[s] - 2 * n[s] * D[s], n[s] * n[s], s)
        if exact_better(c, best):
            best = c
    return best[2]


def random_clusters(rng, k, tied):
    n = [int(v) for v in rng.integers(1, 100000, size=k)]
    n[int(rng.integers(k))] = 0                      # an empty cluster
    Q = [int(v) * nv + nv for v, nv in zip(rng.integers(1, 1000, size=k), n)]
    ni = int(rng.integers(1, 5000))
    D = [int(rng.integers(0, min(nv, ni) * 50 + 1)) for nv in n]
    if tied:   # copies of one cluster at later indices: equal exact scores
        src = int(rng.integers(k))
        for dst in rng.choice(k, size=4, replace=False):
            n[dst], Q[dst], D[dst] = n[src], Q[src], D[src]
    return Q, n, D


def test_screen_keeps_the_exact_argmin():
    rng = np.random.default_rng(7)
    for trial in range(300):
        k = int(rng.integers(1, 700))
        Q, n, D = random_clusters(rng, k, tied=trial % 3 == 0)
        if not any(n):
            continue
        assert screened_argmin(Q, n, D) == exact_argmin(Q, n, D), trial


def test_screen_with_scores_one_ulp_apart():
    """Scores that differ far below FP32 resolution must still be ordered
    exactly: the bracket lets every such cluster through to the exact test."""
    rng = np.random.default_rng(11)
    for trial in range(100):
        k = 300
        n = [int(rng.integers(50000, 60000))] * k
        base = int(rng.integers(10 ** 9, 10 ** 10))
        Q = [base + int(d) for d in rng.integers(0, 3, size=k)]   # scores within 2 / n^2
        D = [int(rng.integers(1000, 1001))] * k
        assert screened_argmin(Q, n, D) == exact_argmin(Q, n, D), trial


def test_screen_with_near_ties_of_different_clusters():
    """Clusters of different sizes whose exact scores differ by less than FP32
    resolution (so FP32 rounding can order them either way): the bracket must
    let the exact minimiser through. A bracket of width 0, or of 2^-26 (a
    quarter of u), drops it in some of these cases."""
    from fractions import Fraction
    rng = np.random.default_rng(13)
    for trial in range(400):
        k = 64
        n = [int(v) for v in rng.integers(20000, 100000, size=k)]
        D = [int(rng.integers(0, 2 * nv)) for nv in n]
        Q0 = int(rng.integers(10 ** 11, 10 ** 12))
        score0 = Fraction(Q0 - 2 * n[0] * D[0], n[0] * n[0])
        Q = [Q0]
        for s in range(1, k):
            # the smallest Q_s whose score is at least score0, then a few units either way
            t = score0 * n[s] * n[s] + 2 * n[s] * D[s]
            q = -((-t.numerator) // t.denominator) + int(rng.integers(-2, 3))
            Q.append(max(q, 1))
        assert screened_argmin(Q, n, D) == exact_argmin(Q, n, D), trial
