"""Python binding of include/rr.h (ctypes): argument marshalling only.

Every computation happens in librr.so's CUDA kernels. Device vectors are
torch CUDA tensors (FP64) passed by pointer on the current torch stream.
Without a built librr.so every call raises at once (the first one loads the
library): there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librr.so")

RR_OK, RR_INVALID_ARG, RR_CUDA_ERROR, RR_OOM, RR_NOT_SPD = 0, 1, 2, 3, 4
RR_NOT_CONVERGED, RR_NONFINITE, RR_TIMEOUT, RR_UNSUPPORTED = 5, 6, 7, 8
RR_CSR_BINARY, RR_DENSE_F32_ROWMAJOR = 0, 1
RR_SOLVER_TWOLEVEL, RR_SOLVER_CG, RR_SOLVER_DCG, RR_SOLVER_TLFCG = 0, 1, 2, 3
RR_PREC_FP64, RR_PREC_MIXED = 0, 1
RR_GRAM_AUTO, RR_GRAM_CUDA_CORES = 0, 1
RR_GATHER_AUTO, RR_GATHER_LANES, RR_GATHER_STAGED, RR_GATHER_LANES_STAGED = 0, 1, 2, 3
RR_COARSE_CHOLESKY, RR_COARSE_EIGEN = 0, 1
RR_CLUSTER_KMEANS, RR_CLUSTER_LEADER = 0, 1

_STATUS = {0: "RR_OK", 1: "RR_INVALID_ARG", 2: "RR_CUDA_ERROR", 3: "RR_OOM", 4: "RR_NOT_SPD",
           5: "RR_NOT_CONVERGED", 6: "RR_NONFINITE", 7: "RR_TIMEOUT", 8: "RR_UNSUPPORTED"}


class rr_matrix(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
                ("values", ctypes.c_void_p), ("layout", ctypes.c_int32),
                ("on_device", ctypes.c_int32)]


class rr_options(ctypes.Structure):
    _fields_ = [("kmeans_max_iter", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("init_centers", ctypes.c_void_p),
                ("solver", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("max_restarts", ctypes.c_int32),
                ("use_graphs", ctypes.c_int32), ("gram", ctypes.c_int32),
                ("gather", ctypes.c_int32), ("wait_limit", ctypes.c_int32),
                ("lloyd_pull_work", ctypes.c_int64), ("coarse", ctypes.c_int32),
                ("split_head", ctypes.c_int32), ("clustering", ctypes.c_int32),
                ("lf_tol2", ctypes.c_double), ("seed_pull_work", ctypes.c_int64),
                ("stream", ctypes.c_void_p)]


class rr_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("k_eff", ctypes.c_int32), ("kmeans_iters", ctypes.c_int32),
                ("rel_res", ctypes.c_double), ("true_rel_res", ctypes.c_double),
                ("omega", ctypes.c_double), ("setup_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("launches", ctypes.c_int64),
                ("gram_tensor_cores", ctypes.c_int32), ("fallbacks", ctypes.c_int32),
                ("gather_staged", ctypes.c_int32), ("setup_phase_ms", ctypes.c_double * 8)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["setup_phase_ms"] = list(self.setup_phase_ms)
        return d


class rr_bayes_params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("a_tau", ctypes.c_double), ("b_tau", ctypes.c_double),
                ("lambda0", ctypes.c_double), ("tau0", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("tol", ctypes.c_double)]


class RRError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None

# the C ABI: name -> (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "rr_default_options": (None, [ctypes.POINTER(rr_options)]),
    "rr_setup": (ctypes.c_int, [ctypes.POINTER(rr_matrix), ctypes.c_double, ctypes.c_int32,
                                ctypes.POINTER(rr_options), ctypes.POINTER(_P)]),
    "rr_set_lambda": (ctypes.c_int, [_P, ctypes.c_double]),
    "rr_prepare_lambdas": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "rr_fork_lambda": (ctypes.c_int, [_P, ctypes.c_double, _P]),
    "rr_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.POINTER(rr_info)]),
    "rr_solve_batch": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32, _P, _P,
                                      ctypes.c_double, _P]),
    "rr_solve_fcg": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_double, ctypes.POINTER(rr_info)]),
    "rr_solve_many": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, ctypes.c_double, _P, _P]),
    "rr_harvest": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_double, _P, ctypes.c_double,
                                  ctypes.c_int32, _P, _P, ctypes.c_int64,
                                  ctypes.POINTER(ctypes.c_int64)]),
    "rr_mlp_param_count": (ctypes.c_int64, [ctypes.c_int32, ctypes.c_int32]),
    "rr_mlp_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P,
                                     ctypes.POINTER(_P)]),
    "rr_mlp_set_params": (ctypes.c_int, [_P, _P]),
    "rr_mlp_set_metric": (ctypes.c_int, [_P, _P]),
    "rr_mlp_get_params": (ctypes.c_int, [_P, _P]),
    "rr_mlp_forward": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "rr_mlp_grad": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, _P]),
    "rr_mlp_train": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_float, ctypes.c_uint64, _P]),
    "rr_mlp_free": (None, [_P]),
    "rr_apply": (ctypes.c_int, [_P, _P, _P]),
    "rr_precondition": (ctypes.c_int, [_P, _P, _P]),
    "rr_rhs": (ctypes.c_int, [_P, _P, _P]),
    "rr_matvec": (ctypes.c_int, [_P, _P, _P]),
    "rr_get_labels": (ctypes.c_int, [_P, _P]),
    "rr_get_centers": (ctypes.c_int, [_P, _P]),
    "rr_get_coarse": (ctypes.c_int, [_P, _P, _P]),
    "rr_query": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "rr_free": (None, [_P]),
    "rr_last_error": (ctypes.c_char_p, []),
    "rr_query_batch": (ctypes.c_int, [_P, _P, _P, _P]),
    "rr_get_eigen": (ctypes.c_int, [_P, _P, _P, _P]),
    "rr_bayes": (ctypes.c_int, [_P, _P, ctypes.POINTER(rr_bayes_params), ctypes.c_int32,
                                ctypes.c_int32, _P, _P, _P, _P]),
    "rr_launch_count": (ctypes.c_int64, []),
    "rr_apply_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, _P, _P, _P, _P,
                                        ctypes.c_double, _P, _P, _P]),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads librr.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1806_05826_gb300/build.py "
                               "(or __graft_entry__.build()); there is no CPU fallback")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def rr_launch_count() -> int:
    return int(load().rr_launch_count())


def rr_last_error() -> str:
    return load().rr_last_error().decode()


def _check(status):
    if status != RR_OK:
        raise RRError(status, rr_last_error())


def _ptr(t):
    """Device or host pointer of a torch tensor or numpy array."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _dev(t, dtype, n, name, device="cuda"):
    """Device pointer of a contiguous CUDA tensor of `dtype` holding at least
    n elements. Anything else raises here, before the library could read or
    write past a buffer or treat a host address as a device one."""
    import torch
    if not isinstance(t, torch.Tensor) or t.device.type != device:
        raise TypeError(f"{name}: a {device.upper()} tensor is required, got {type(t).__name__}"
                        + ("" if not isinstance(t, torch.Tensor) else f" on {t.device}"))
    if t.dtype != dtype:
        raise TypeError(f"{name}: dtype {t.dtype}, {dtype} required")
    if not t.is_contiguous():
        raise ValueError(f"{name}: a contiguous tensor is required")
    if t.numel() < n:
        raise ValueError(f"{name}: {t.numel()} elements, at least {n} required")
    return t.data_ptr()


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def rr_default_options(**kw) -> rr_options:
    o = rr_options()
    load().rr_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Handle:
    """Owns an rr_handle; the functions below take it as their first argument."""

    def __init__(self, ptr, F, N, keepalive, k=None):
        self.ptr = ptr
        self.F, self.N, self.k = F, N, k
        self.dense = False
        self._keep = keepalive

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "ptr", None):
            load().rr_free(self.ptr)
            self.ptr = None


def rr_setup(row_ptr, col_idx, n_rows, n_cols, lam, k, *, seed=0, init_centers=None,
             kmeans_max_iter=50, max_iter=20000, solver=RR_SOLVER_TWOLEVEL, check_every=8,
             max_restarts=5, use_graphs=1, gram=RR_GRAM_AUTO, gather=RR_GATHER_AUTO,
             precision=RR_PREC_FP64, wait_limit=0, lloyd_pull_work=0, split_head=0,
             coarse=0, clustering=RR_CLUSTER_KMEANS, lf_tol2=1.0, seed_pull_work=0,
             stream=None) -> Handle:
    """rr_setup on a binary CSR pattern given as numpy arrays (host) or torch
    CUDA tensors (device): row_ptr int64[N+1], col_idx int32[nnz]. With
    clustering = RR_CLUSTER_LEADER, k is the largest number of leaders."""
    on_device = 0 if isinstance(row_ptr, np.ndarray) else 1
    if on_device == 0:
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        if row_ptr.ndim != 1 or row_ptr.size != n_rows + 1:
            raise ValueError(f"row_ptr: {row_ptr.size} entries, n_rows + 1 = {n_rows + 1} required")
        nnz = int(row_ptr[-1])
        if col_idx.size < nnz:
            raise ValueError(f"col_idx: {col_idx.size} entries, row_ptr[-1] = {nnz} required")
        rp, ci = _ptr(row_ptr), _ptr(col_idx)
    else:
        torch = _torch()
        rp = _dev(row_ptr, torch.int64, n_rows + 1, "row_ptr")
        ci = _dev(col_idx, torch.int32, 0, "col_idx")
        nnz = int(col_idx.numel())
    lib = load()
    X = rr_matrix(n_rows, n_cols, nnz, rp, ci, None, RR_CSR_BINARY, on_device)
    ic = None
    if init_centers is not None:
        ic = np.ascontiguousarray(init_centers, dtype=np.int32)
    o = rr_default_options(kmeans_max_iter=kmeans_max_iter, max_iter=max_iter, seed=seed,
                           init_centers=_ptr(ic), solver=solver, check_every=check_every,
                           max_restarts=max_restarts, use_graphs=use_graphs, gram=gram,
                           gather=gather, wait_limit=wait_limit, lloyd_pull_work=lloyd_pull_work,
                           split_head=split_head, coarse=coarse, clustering=clustering,
                           lf_tol2=float(lf_tol2), seed_pull_work=int(seed_pull_work),
                           precision=precision, stream=_stream_ptr(stream))
    out = _P()
    _check(lib.rr_setup(ctypes.byref(X), float(lam), int(k), ctypes.byref(o), ctypes.byref(out)))
    return Handle(out, n_cols, n_rows, (ic,), int(k))


def rr_setup_dense(X, lam, k, *, seed=0, init_centers=None, kmeans_max_iter=50, max_iter=20000,
                   solver=RR_SOLVER_TWOLEVEL, check_every=8, max_restarts=5, use_graphs=1,
                   precision=RR_PREC_FP64, coarse=RR_COARSE_CHOLESKY, stream=None) -> Handle:
    """rr_setup on a dense X (N x F, float32 row-major) given as a numpy array
    (host) or a torch CUDA tensor (device)."""
    on_device = 0 if isinstance(X, np.ndarray) else 1
    if on_device == 0:
        X = np.ascontiguousarray(X, dtype=np.float32)
    if X.ndim != 2:
        raise ValueError("X: a two-dimensional (N, F) array is required")
    n_rows, n_cols = int(X.shape[0]), int(X.shape[1])
    xp = _ptr(X) if on_device == 0 else _dev(X, _torch().float32, n_rows * n_cols, "X")
    lib = load()
    M = rr_matrix(n_rows, n_cols, n_rows * n_cols, None, None, xp, RR_DENSE_F32_ROWMAJOR,
                  on_device)
    ic = None
    if init_centers is not None:
        ic = np.ascontiguousarray(init_centers, dtype=np.int32)
    o = rr_default_options(kmeans_max_iter=kmeans_max_iter, max_iter=max_iter, seed=seed,
                           init_centers=_ptr(ic), solver=solver, check_every=check_every,
                           max_restarts=max_restarts, use_graphs=use_graphs,
                           precision=precision, stream=_stream_ptr(stream), coarse=coarse)
    out = _P()
    _check(lib.rr_setup(ctypes.byref(M), float(lam), int(k), ctypes.byref(o), ctypes.byref(out)))
    h = Handle(out, n_cols, n_rows, (ic,), int(k))
    h.dense = True
    return h


def rr_prepare_lambdas(h: Handle, lambdas):
    """Coarse levels of further lambdas built ahead on a second stream."""
    lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64).ravel())
    _check(load().rr_prepare_lambdas(h.ptr, lam.ctypes.data, int(lam.size)))


def rr_set_lambda(h: Handle, lam: float):
    _check(load().rr_set_lambda(h.ptr, float(lam)))


def rr_solve(h: Handle, y, w, tol=1e-8) -> dict:
    f64 = _torch().float64
    yp, wp = _dev(y, f64, h.N, "y"), _dev(w, f64, h.F, "w")
    info = rr_info()
    st = load().rr_solve(h.ptr, yp, wp, float(tol), ctypes.byref(info))
    d = info.as_dict()
    d["status"] = _STATUS[st]
    if st not in (RR_OK, RR_NOT_CONVERGED):
        raise RRError(st, rr_last_error())
    return d


def rr_solve_batch(h: Handle, Y, lambdas, W, tol=1e-8) -> dict:
    """rr_solve_batch: Y device float64 (nrhs, N); W device float64 (nlam, nrhs, F).
    Returns {"status": ..., "infos": [[info of (j, l) for j] for l]}."""
    nrhs = int(Y.shape[0])
    lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64).ravel())
    nlam = int(lam.size)
    f64 = _torch().float64
    yp = _dev(Y, f64, nrhs * h.N, "Y")
    wp = _dev(W, f64, nlam * nrhs * h.F, "W")
    infos = (rr_info * (nrhs * nlam))()
    st = load().rr_solve_batch(h.ptr, nrhs, yp, nlam, lam.ctypes.data, wp, float(tol),
                               ctypes.cast(infos, _P))
    if st not in (RR_OK, RR_NOT_CONVERGED):
        raise RRError(st, rr_last_error())
    return {"status": _STATUS[st],
            "infos": [[infos[l * nrhs + j].as_dict() for j in range(nrhs)] for l in range(nlam)]}


def rr_fork_lambda(h: Handle, lam) -> Handle:
    """rr_fork_lambda: a handle for weight lam sharing h's X-dependent setup
    (h must outlive it; rr_free it before h)."""
    out = _P()
    _check(load().rr_fork_lambda(h.ptr, float(lam), ctypes.byref(out)))
    return Handle(out, h.F, h.N, (h,), h.k)


def rr_solve_many(hs, ys, ws, tol=1e-8, stream=None) -> dict:
    """rr_solve_many over handles hs, device targets ys and solutions ws (lists)."""
    n = len(hs)
    if len(ys) != n or len(ws) != n:
        raise ValueError("hs, ys and ws must have the same length")
    f64 = _torch().float64
    H = (_P * n)(*[h.ptr for h in hs])
    Y = (_P * n)(*[_dev(y, f64, h.N, f"ys[{i}]") for i, (h, y) in enumerate(zip(hs, ys))])
    W = (_P * n)(*[_dev(w, f64, h.F, f"ws[{i}]") for i, (h, w) in enumerate(zip(hs, ws))])
    infos = (rr_info * n)()
    st = load().rr_solve_many(n, ctypes.cast(H, _P), ctypes.cast(Y, _P), ctypes.cast(W, _P),
                              float(tol), _stream_ptr(stream), ctypes.cast(infos, _P))
    if st not in (RR_OK, RR_NOT_CONVERGED):
        raise RRError(st, rr_last_error())
    return {"status": _STATUS[st], "infos": [infos[i].as_dict() for i in range(n)]}


def rr_solve_fcg(h: Handle, net, y, w, tol=1e-8) -> dict:
    """rr_solve_fcg: flexible CG with the Cholesky coarse solve (net None) or the
    learned correction of an Mlp."""
    f64 = _torch().float64
    yp, wp = _dev(y, f64, h.N, "y"), _dev(w, f64, h.F, "w")
    info = rr_info()
    st = load().rr_solve_fcg(h.ptr, net.ptr if net is not None else None, yp, wp,
                             float(tol), ctypes.byref(info))
    d = info.as_dict()
    d["status"] = _STATUS[st]
    if st not in (RR_OK, RR_NOT_CONVERGED):
        raise RRError(st, rr_last_error())
    return d


def rr_harvest(h: Handle, Y, lam, Wref, tol, max_iter, max_pairs, k):
    """rr_harvest into new device float32 tensors (max_pairs, k); returns the
    (Xp, Tp) rows written."""
    torch = _torch()
    nrhs = int(Y.shape[0])
    yp = _dev(Y, torch.float64, nrhs * h.N, "Y")
    wp = _dev(Wref, torch.float64, nrhs * h.F, "Wref")
    k_eff = rr_query(h)["k_eff"]
    if k != k_eff:
        raise ValueError(f"k = {k}: the pairs have the handle's k_eff = {k_eff} entries")
    Xp = torch.empty((max_pairs, k), dtype=torch.float32, device=Y.device)
    Tp = torch.empty((max_pairs, k), dtype=torch.float32, device=Y.device)
    n = ctypes.c_int64()
    _check(load().rr_harvest(h.ptr, nrhs, yp, float(lam), wp, float(tol),
                             int(max_iter), _ptr(Xp), _ptr(Tp), int(max_pairs), ctypes.byref(n)))
    return Xp[:n.value], Tp[:n.value]


# ---- the learned correction's network

MLP_KEYS = ("W1", "b1", "W2", "b2", "W3", "b3")


def mlp_pack(p: dict) -> np.ndarray:
    """Flat float32 parameters in the documented order (W1, b1, W2, b2, W3, b3)."""
    return np.concatenate([np.asarray(p[n], dtype=np.float32).ravel() for n in MLP_KEYS])


def mlp_unpack(flat, k: int, H: int) -> dict:
    shapes = {"W1": (H, k), "b1": (H,), "W2": (H, H), "b2": (H,), "W3": (k, H), "b3": (k,)}
    out, o = {}, 0
    for n in MLP_KEYS:
        size = int(np.prod(shapes[n]))
        out[n] = np.asarray(flat[o:o + size]).reshape(shapes[n])
        o += size
    return out


class Mlp:
    def __init__(self, ptr, k, H):
        self.ptr, self.k, self.H = ptr, k, H

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "ptr", None):
            load().rr_mlp_free(self.ptr)
            self.ptr = None


def mlp_param_count(k: int, H: int) -> int:
    return int(load().rr_mlp_param_count(k, H))


def mlp_create(k: int, H: int, params: dict, max_batch=512, stream=None) -> Mlp:
    flat = np.ascontiguousarray(mlp_pack(params))
    assert flat.size == mlp_param_count(k, H)
    out = _P()
    _check(load().rr_mlp_create(k, H, max_batch, flat.ctypes.data, _stream_ptr(stream),
                                ctypes.byref(out)))
    return Mlp(out, k, H)


def mlp_get_params(m: Mlp) -> dict:
    flat = np.empty(mlp_param_count(m.k, m.H), dtype=np.float32)
    _check(load().rr_mlp_get_params(m.ptr, flat.ctypes.data))
    return mlp_unpack(flat, m.k, m.H)


def mlp_set_params(m: Mlp, params: dict):
    flat = np.ascontiguousarray(mlp_pack(params))
    _check(load().rr_mlp_set_params(m.ptr, flat.ctypes.data))


def mlp_set_metric(m: Mlp, W=None):
    """Loss metric W (symmetric k x k, host array) or None for the plain loss."""
    if W is None:
        _check(load().rr_mlp_set_metric(m.ptr, None))
        return
    Wf = np.ascontiguousarray(W, dtype=np.float32)
    if Wf.shape != (m.k, m.k):
        raise ValueError(f"W: shape ({m.k}, {m.k}) required, got {Wf.shape}")
    _check(load().rr_mlp_set_metric(m.ptr, Wf.ctypes.data))


def mlp_forward(m: Mlp, X):
    """X: device float32 (B, k) -> device float32 (B, k)."""
    torch = _torch()
    B = int(X.shape[0])
    if X.ndim != 2 or int(X.shape[1]) != m.k:
        raise ValueError(f"X: shape (B, {m.k}) required, got {tuple(X.shape)}")
    xp = _dev(X, torch.float32, B * m.k, "X")
    out = torch.empty_like(X)
    _check(load().rr_mlp_forward(m.ptr, B, xp, _ptr(out)))
    return out


def mlp_grad(m: Mlp, X, T):
    """Loss and gradients (dict of numpy arrays) for device float32 rows X, T."""
    f32 = _torch().float32
    B = int(X.shape[0])
    for name, t in (("X", X), ("T", T)):
        if t.ndim != 2 or tuple(t.shape) != (B, m.k):
            raise ValueError(f"{name}: shape ({B}, {m.k}) required, got {tuple(t.shape)}")
    xp, tp = _dev(X, f32, B * m.k, "X"), _dev(T, f32, B * m.k, "T")
    flat = np.empty(mlp_param_count(m.k, m.H), dtype=np.float32)
    loss = ctypes.c_float()
    _check(load().rr_mlp_grad(m.ptr, B, xp, tp, flat.ctypes.data, ctypes.byref(loss)))
    return float(loss.value), mlp_unpack(flat, m.k, m.H)


def mlp_train(m: Mlp, Xp, Tp, batch=256, steps=100, lr=1e-3, seed=0):
    """Adam steps on pairs (device float32 (n, k)); returns the batch losses."""
    f32 = _torch().float32
    n = int(Xp.shape[0])
    for name, t in (("Xp", Xp), ("Tp", Tp)):
        if t.ndim != 2 or tuple(t.shape) != (n, m.k):
            raise ValueError(f"{name}: shape ({n}, {m.k}) required, got {tuple(t.shape)}")
    xp, tp = _dev(Xp, f32, n * m.k, "Xp"), _dev(Tp, f32, n * m.k, "Tp")
    losses = np.empty(max(1, steps), dtype=np.float32)
    _check(load().rr_mlp_train(m.ptr, n, xp, tp, int(batch),
                               int(steps), float(lr), int(seed), losses.ctypes.data))
    return losses[:steps]


def rr_apply(h: Handle, v, out):
    f64 = _torch().float64
    vp, op = _dev(v, f64, h.F, "v"), _dev(out, f64, h.F, "out")
    _check(load().rr_apply(h.ptr, vp, op))


def rr_precondition(h: Handle, r, z):
    f64 = _torch().float64
    rp, zp = _dev(r, f64, h.F, "r"), _dev(z, f64, h.F, "z")
    _check(load().rr_precondition(h.ptr, rp, zp))


def rr_rhs(h: Handle, y, b):
    f64 = _torch().float64
    yp, bp = _dev(y, f64, h.N, "y"), _dev(b, f64, h.F, "b")
    _check(load().rr_rhs(h.ptr, yp, bp))


def rr_matvec(h: Handle, v, u):
    f64 = _torch().float64
    vp, up = _dev(v, f64, h.F, "v"), _dev(u, f64, h.N, "u")
    _check(load().rr_matvec(h.ptr, vp, up))


def rr_apply_noalloc(n_rows, n_cols, row_ptr, col_idx, col_ptr, row_idx, lam, v, out,
                     stream=None):
    """out = (X^T X + lam I) v from device CSR/CSC tensors; allocates nothing.

    The pattern's lengths are checked before anything reaches the library:
    row_ptr and col_ptr must end at the same nnz, which must equal the
    lengths of col_idx and row_idx (reading the two end entries waits for the
    device, but allocates nothing on it)."""
    torch = _torch()
    for name, t, n in (("row_ptr", row_ptr, n_rows + 1), ("col_ptr", col_ptr, n_cols + 1)):
        if not isinstance(t, torch.Tensor) or t.ndim != 1 or t.numel() != n:
            raise ValueError(f"{name}: a one-dimensional tensor of {n} entries is required")
    nnz_r, nnz_c = int(row_ptr[n_rows]), int(col_ptr[n_cols])
    for name, t in (("col_idx", col_idx), ("row_idx", row_idx)):
        if not isinstance(t, torch.Tensor) or t.numel() != nnz_r:
            raise ValueError(f"{name}: row_ptr ends at nnz = {nnz_r}, so {nnz_r} entries are "
                             f"required, got {getattr(t, 'numel', lambda: None)()}")
    if nnz_c != nnz_r:
        raise ValueError(f"col_ptr ends at {nnz_c}, row_ptr at {nnz_r}: not the same pattern")
    ptrs = (_dev(row_ptr, torch.int64, n_rows + 1, "row_ptr"),
            _dev(col_idx, torch.int32, nnz_r, "col_idx"),
            _dev(col_ptr, torch.int64, n_cols + 1, "col_ptr"),
            _dev(row_idx, torch.int32, nnz_r, "row_idx"))
    vp, op = _dev(v, torch.float64, n_cols, "v"), _dev(out, torch.float64, n_cols, "out")
    _check(load().rr_apply_noalloc(int(n_rows), int(n_cols), *ptrs, float(lam), vp, op,
                                   _stream_ptr(stream)))


def rr_get_labels(h: Handle) -> np.ndarray:
    out = np.empty(h.F, dtype=np.int32)
    _check(load().rr_get_labels(h.ptr, out.ctypes.data))
    return out


def rr_get_centers(h: Handle, k: int) -> np.ndarray:
    if h.k is not None and k != h.k:
        raise ValueError(f"k = {k}: the handle was set up with k = {h.k} centres")
    out = np.empty(k, dtype=np.int32)
    _check(load().rr_get_centers(h.ptr, out.ctypes.data))
    return out


def rr_query(h: Handle) -> dict:
    n, f = ctypes.c_int64(), ctypes.c_int64()
    k, om, lam = ctypes.c_int32(), ctypes.c_double(), ctypes.c_double()
    _check(load().rr_query(h.ptr, ctypes.byref(n), ctypes.byref(f), ctypes.byref(k),
                           ctypes.byref(om), ctypes.byref(lam)))
    return {"n_rows": n.value, "n_cols": f.value, "k_eff": k.value, "omega": om.value,
            "lambda": lam.value}


def rr_query_batch(h: Handle) -> dict:
    """The batched engine's autotuned SpMM variant and its apply time."""
    w, u, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(load().rr_query_batch(h.ptr, ctypes.byref(w), ctypes.byref(u), ctypes.byref(ms)))
    return {"slab_width": w.value, "unroll": u.value, "apply_ms": ms.value}


def rr_get_eigen(h: Handle):
    """(mu, Q, sweeps) of an RR_COARSE_EIGEN handle: X_c^T X_c = Q diag(mu) Q^T."""
    k = rr_query(h)["k_eff"]
    mu = np.empty(k, dtype=np.float64)
    Q = np.empty((k, k), dtype=np.float64)
    sw = ctypes.c_int32()
    _check(load().rr_get_eigen(h.ptr, mu.ctypes.data, Q.ctypes.data, ctypes.byref(sw)))
    return mu, Q, sw.value


def rr_bayes(h: Handle, y, n_samples, burnin=0, w_mean=None, alpha=1.0, beta=1.0, a_tau=1.0,
             b_tau=1.0, lambda0=1.0, tau0=1.0, seed=0, tol=1e-8):
    """Gibbs sampling with noise injection: returns (lambda trace, tau trace,
    iterations per solve); w_mean (device float64[F] or None) receives the
    mean of w over the samples after burnin."""
    f64 = _torch().float64
    yp = _dev(y, f64, h.N, "y")
    wp = None if w_mean is None else _dev(w_mean, f64, h.F, "w_mean")
    n = int(n_samples)
    if n < 1:
        raise ValueError("n_samples must be >= 1")
    p = rr_bayes_params(float(alpha), float(beta), float(a_tau), float(b_tau), float(lambda0),
                        float(tau0), int(seed), float(tol))
    lam, tau = np.zeros(n), np.zeros(n)
    iters = np.zeros(n, dtype=np.int32)
    _check(load().rr_bayes(h.ptr, yp, ctypes.byref(p), n, int(burnin), wp, lam.ctypes.data,
                           tau.ctypes.data, iters.ctypes.data))
    return lam, tau, iters


def rr_get_coarse(h: Handle):
    """(A_c, G): G is the exact integer Gram for binary X, None for dense X."""
    k = rr_query(h)["k_eff"]
    Ac = np.empty((k, k), dtype=np.float64)
    G = None if h.dense else np.empty((k, k), dtype=np.int64)
    _check(load().rr_get_coarse(h.ptr, Ac.ctypes.data, None if G is None else G.ctypes.data))
    return Ac, G


def rr_free(h: Handle):
    h.close()
