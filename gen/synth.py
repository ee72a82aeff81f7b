"""Seeded synthetic inputs shaped like the paper's feature matrices.

This module only makes inputs: it holds none of the solver's arithmetic, and
both the CUDA path's tests and the CPU oracle draw their inputs from it.

The paper's datasets (Table 1) are not available, so two stand-ins are made:

* binary sparse X with power-law column frequencies (Zipf exponent s), the
  shape of the ChEMBL / news20-like binary data of Table 1;
* dense X with AR(1)-correlated features, the shape of the dense
  gisette / DrivFace / SNP-like data of Table 1.

All randomness comes from one counter-based generator, SplitMix64
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), evaluated on (seed, stream, index) so every array is a pure
function of its seed and no draw depends on the order of the others.
"""
from __future__ import annotations

import dataclasses
import math
import os

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (wrapping uint64 arithmetic)."""
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _stream_base(seed: int, stream: int) -> np.uint64:
    s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    t = np.array([(stream * 0xD1B54A32D192ED03) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(_mix64(s) ^ t)[0]


def raw64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """The n SplitMix64 outputs offset..offset+n-1 of stream `stream` of `seed`."""
    base = _stream_base(seed, stream)
    idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(base + idx * _GAMMA)


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniforms in [0, 1) with 53 random bits."""
    return (raw64(seed, stream, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _normal_range(seed: int, stream: int, offset: int, n: int) -> np.ndarray:
    u1 = 1.0 - uniform(seed, stream, n, offset)          # (0, 1]
    u2 = uniform(seed, stream, n, (1 << 40) + offset)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """Standard normals by the Box-Muller transform of two uniform streams
    (normal i from uniforms i and 2^40 + i). Large draws are split into
    ranges computed on several threads (numpy releases the GIL in its
    element-wise loops); the values do not depend on the split."""
    chunk = 1 << 22
    if n <= 2 * chunk:
        return _normal_range(seed, stream, 0, n)
    import concurrent.futures as cf
    out = np.empty(n, dtype=np.float64)

    def fill(a):
        out[a:a + min(chunk, n - a)] = _normal_range(seed, stream, a, min(chunk, n - a))

    workers = max(1, min(16, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        list(ex.map(fill, range(0, n, chunk)))
    return out


# --------------------------------------------------------------------------
# Binary sparse X with Zipf column frequencies
# --------------------------------------------------------------------------

@dataclasses.dataclass
class CSR:
    """Binary CSR pattern (values are all one): row_ptr int64[N+1], col_idx int32[nnz]."""
    n_rows: int
    n_cols: int
    row_ptr: np.ndarray
    col_idx: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def zipf_column_probs(n_cols: int, density: float, s: float) -> np.ndarray:
    """Inclusion probability of the column of frequency rank j: min(1, c (j+1)^-s),
    with c fixed by bisection so that the probabilities sum to density * n_cols."""
    target = density * n_cols
    base = np.arange(1, n_cols + 1, dtype=np.float64) ** (-s)
    lo, hi = 0.0, 1.0
    while np.minimum(1.0, hi * base).sum() < target:
        hi *= 2.0
        if hi > 1e300:
            raise ValueError("density too high")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.minimum(1.0, mid * base).sum() < target:
            lo = mid
        else:
            hi = mid
    return np.minimum(1.0, hi * base)


def zipf_binary(n_rows: int, n_cols: int, density: float, s: float = 1.1,
                seed: int = 0) -> CSR:
    """Binary N x F matrix whose column of frequency rank j holds each row
    independently with probability q_j (zipf_column_probs). Column ranks are
    mapped to column indices by a seeded permutation. Rows of a column are
    drawn by geometric skipping, so the cost is O(nnz)."""
    q = zipf_column_probs(n_cols, density, s)
    perm = np.argsort(raw64(seed, 1, n_cols), kind="stable").astype(np.int64)

    rows_parts = []
    cols_parts = []
    full = q >= 1.0
    for j in np.nonzero(full)[0]:
        rows_parts.append(np.arange(n_rows, dtype=np.int64))
        cols_parts.append(np.full(n_rows, perm[j], dtype=np.int64))

    part = np.nonzero(~full)[0]
    pending = part
    attempt = 0
    while pending.size:
        qp = q[pending]
        m = qp * n_rows
        budget = np.ceil(m + 8.0 * np.sqrt(m * (1.0 - qp)) + 16.0).astype(np.int64) << attempt
        budget = np.minimum(budget, n_rows + 1)
        starts = np.zeros(pending.size + 1, dtype=np.int64)
        np.cumsum(budget, out=starts[1:])
        total = int(starts[-1])
        u = 1.0 - uniform(seed, 2 + attempt, total)       # (0, 1]
        logq = np.log1p(-np.repeat(qp, budget))
        gaps = np.floor(np.log(u) / logq).astype(np.int64) + 1
        gaps = np.minimum(gaps, n_rows + 1)
        cs = np.cumsum(gaps)
        seg_off = np.repeat(cs[starts[:-1]] - gaps[starts[:-1]], budget)
        pos = cs - seg_off - 1                               # 0-based row positions
        last = pos[starts[1:] - 1]
        done = last >= n_rows
        keep = (pos < n_rows) & np.repeat(done, budget)
        colrep = np.repeat(perm[pending], budget)
        rows_parts.append(pos[keep])
        cols_parts.append(colrep[keep])
        pending = pending[~done]
        attempt += 1
        if attempt > 8:
            raise RuntimeError("geometric skipping did not terminate")

    rows = np.concatenate(rows_parts) if rows_parts else np.zeros(0, np.int64)
    cols = np.concatenate(cols_parts) if cols_parts else np.zeros(0, np.int64)
    key = np.sort(rows * np.int64(n_cols) + cols)
    rows = key // n_cols
    cols = (key - rows * n_cols).astype(np.int32)
    row_ptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n_rows), out=row_ptr[1:])
    return CSR(n_rows, n_cols, row_ptr, cols)


def csr_matvec(X: CSR, v: np.ndarray) -> np.ndarray:
    """X v for a binary pattern (used only to make targets y = X w* + noise)."""
    rows = np.repeat(np.arange(X.n_rows), np.diff(X.row_ptr))
    return np.bincount(rows, weights=v[X.col_idx], minlength=X.n_rows)


def ridge_targets(X, seed: int, noise_sigma: float = 0.1):
    """w* ~ N(0, 1) per feature and y = X w* + N(0, noise_sigma^2) per sample.
    X is a CSR pattern or a dense (N, F) array."""
    if isinstance(X, CSR):
        n, f = X.n_rows, X.n_cols
        w_star = normal(seed, 10, f)
        y = csr_matvec(X, w_star)
    else:
        n, f = X.shape
        w_star = normal(seed, 10, f)
        y = X.astype(np.float64) @ w_star
    return y + noise_sigma * normal(seed, 11, n), w_star


def ridge_targets_many(X: CSR, seeds, noise_sigma: float = 0.1):
    """Targets y_j = X w*_j + noise for each seed j (as ridge_targets, one seed
    per target). Returns Y (len(seeds), N) and W* (len(seeds), F)."""
    import scipy.sparse as sp
    A = sp.csr_matrix((np.ones(X.nnz), X.col_idx, X.row_ptr), shape=(X.n_rows, X.n_cols))
    W = np.stack([normal(sd, 10, X.n_cols) for sd in seeds])
    Y = np.asarray((A @ W.T).T)
    for j, sd in enumerate(seeds):
        Y[j] += noise_sigma * normal(sd, 11, X.n_rows)
    return np.ascontiguousarray(Y), W


def mlp_init(k: int, hidden: int, seed: int, stream: int = 30) -> dict:
    """Initial weights of the learned correction's network (k -> hidden ->
    hidden -> k): He-uniform draws (2u - 1) sqrt(6 / fan_in) from this module's
    uniforms, taken in the order W1, W2, W3; biases zero."""
    draws = uniform(seed, stream, 2 * hidden * k + hidden * hidden)
    out, o = {}, 0
    for name, fo, fi in (("W1", hidden, k), ("W2", hidden, hidden), ("W3", k, hidden)):
        n = fo * fi
        out[name] = (2.0 * draws[o:o + n] - 1.0).reshape(fo, fi) * np.sqrt(6.0 / fi)
        o += n
    out["b1"], out["b2"], out["b3"] = np.zeros(hidden), np.zeros(hidden), np.zeros(k)
    return out


def dense_ar1(n_rows: int, n_cols: int, rho: float = 0.9, seed: int = 0) -> np.ndarray:
    """Dense float32 X with X[:,0] ~ N(0,1) and X[:,j] = rho X[:,j-1] + sqrt(1-rho^2) eps_j."""
    eps = normal(seed, 20, n_rows * n_cols).reshape(n_cols, n_rows)
    out = np.empty((n_cols, n_rows), dtype=np.float64)
    out[0] = eps[0]
    c = math.sqrt(1.0 - rho * rho)
    for j in range(1, n_cols):
        out[j] = rho * out[j - 1] + c * eps[j]
    # X = out^T rounded to float32, by blocks of rows on several threads
    X = np.empty((n_rows, n_cols), dtype=np.float32)

    def put(r0):
        X[r0:r0 + 256] = out[:, r0:r0 + 256].T

    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:
        list(ex.map(put, range(0, n_rows, 256)))
    return X


def duplicated_features(base: np.ndarray, counts) -> tuple[np.ndarray, np.ndarray]:
    """Definition 1's ideal data set: column g of `base` repeated counts[g] times.
    Returns the (N, sum(counts)) matrix and the group of each column."""
    counts = np.asarray(counts, dtype=np.int64)
    groups = np.repeat(np.arange(len(counts)), counts)
    return base[:, groups], groups


# --------------------------------------------------------------------------
# The workloads, by name
# --------------------------------------------------------------------------

WORKLOADS = {
    # small case: 2,000 x 1,000 binary, 1% dense, k = 50, lambda = 1e-2
    "zipf_2000x1000": dict(n_rows=2000, n_cols=1000, density=0.01, s=1.1, seed=0,
                           k=50, lambdas=(1e-2,)),
    # full size: 200,000 x 100,000 binary, 0.2% dense, k = 1000, three lambdas
    "zipf_200000x100000": dict(n_rows=200_000, n_cols=100_000, density=0.002, s=1.1,
                               seed=1, k=1000, lambdas=(1e-3, 1e-1, 10.0)),
}

# many targets x many weights over the 200,000 x 100,000 matrix: 64 targets
# (seeds 0..63), 8 weights log-spaced from 1e-3 to 10 -> 512 systems
BATCH_WORKLOADS = {
    "zipf_200000x100000_64x8": dict(base="zipf_200000x100000", target_seeds=tuple(range(64)),
                                    lambdas=tuple(float(v) for v in np.logspace(-3, 1, 8))),
}


# independent problems of uneven sizes (Zipf s = 1.1 binary X, lambda = 1e-2,
# k = d // 100), problem i drawn from seed i, density ~ U[0.1%, 1%]:
#   "uneven_28_dense4": 28 binary problems, n ~ U[10k, 400k], d ~ U[5k, 150k]
#     (about 2.55e9 nonzeros in all: minutes of host generation), and four
#     dense problems of 50,000 x 4,000 float32 AR(1) (rho = 0.9), k = 40,
#     seeds 28..31;
#   "uneven_12_dense4": a scaled stand-in, 12 binary problems with
#     n ~ U[10k, 100k], d ~ U[5k, 40k], and the same four dense problems
#     (seeds 12..15).
MANY_WORKLOADS = {"uneven_12": dict(n_problems=12, n=(10_000, 100_000), d=(5_000, 40_000),
                                    density=(0.001, 0.01), lam=1e-2),
                  "uneven_12_dense4": dict(n_problems=12, n=(10_000, 100_000), d=(5_000, 40_000),
                                           density=(0.001, 0.01), lam=1e-2,
                                           n_dense=4, dense=(50_000, 4_000), rho=0.9),
                  "uneven_28_dense4": dict(n_problems=28, n=(10_000, 400_000),
                                           d=(5_000, 150_000), density=(0.001, 0.01), lam=1e-2,
                                           n_dense=4, dense=(50_000, 4_000), rho=0.9)}


def many_params(name: str):
    """The parameters of each problem of a named set of independent problems:
    n, d and density drawn uniformly in their ranges from seed i (binary
    problems), then the dense problems; k = max(2, d // 100)."""
    p = MANY_WORKLOADS[name]
    out = []
    for i in range(p["n_problems"]):
        u = uniform(i, 40, 3)
        n = int(p["n"][0] + u[0] * (p["n"][1] - p["n"][0]))
        d = int(p["d"][0] + u[1] * (p["d"][1] - p["d"][0]))
        dens = p["density"][0] + u[2] * (p["density"][1] - p["density"][0])
        out.append(dict(n=n, d=d, density=dens, k=max(2, d // 100), lam=p["lam"], seed=i))
    for j in range(p.get("n_dense", 0)):
        n, d = p["dense"]
        out.append(dict(n=n, d=d, density=1.0, k=max(2, d // 100), lam=p["lam"],
                        seed=p["n_problems"] + j, dense=True, rho=p["rho"]))
    return out


def many_problem(q):
    """(X, y) of one problem of a set (params from many_params)."""
    if q.get("dense"):
        X = dense_ar1(q["n"], q["d"], q["rho"], q["seed"])
    else:
        X = zipf_binary(q["n"], q["d"], q["density"], 1.1, q["seed"])
    y, _ = ridge_targets(X, q["seed"])
    return X, y


def many_workload(name: str):
    """[(X, y, params)] of a named set of independent problems (X a CSR
    pattern, or a dense float32 array when params["dense"])."""
    return [many_problem(q) + (q,) for q in many_params(name)]


def batch_workload(name: str):
    """(X, Y, W*, params) of a named batched workload."""
    p = dict(BATCH_WORKLOADS[name])
    base = WORKLOADS[p["base"]]
    X = zipf_binary(base["n_rows"], base["n_cols"], base["density"], base["s"], base["seed"])
    Y, Ws = ridge_targets_many(X, p["target_seeds"])
    p.update(k=base["k"], seed=base["seed"])
    return X, Y, Ws, p


def workload(name: str):
    """(X, y, w_star, params) of a named workload; seed as listed."""
    p = WORKLOADS[name]
    X = zipf_binary(p["n_rows"], p["n_cols"], p["density"], p["s"], p["seed"])
    y, w_star = ridge_targets(X, p["seed"])
    return X, y, w_star, p
