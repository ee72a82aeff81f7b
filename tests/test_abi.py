"""CPU-only checks of the C boundary: librr.so builds, loads, and exports
every entry point include/rr.h declares (no compute call without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "rr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rr_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1806_05826_gb300 import build
    path = build.build_library()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("rr_setup", "rr_solve", "rr_free", "rr_set_lambda", "rr_apply",
                     "rr_get_labels", "rr_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_1806_05826_gb300 import rr
    assert set(header_functions()) <= set(rr.exported_symbols())


def test_default_options_and_invalid_args_without_gpu(lib):
    from paper_1806_05826_gb300 import rr
    o = rr.rr_default_options()
    assert o.kmeans_max_iter == 50 and o.max_iter == 20000 and o.check_every == 8
    L = rr.load()
    # argument checks happen on the host before any device work
    out = ctypes.c_void_p()
    assert L.rr_setup(None, 1.0, 1, None, ctypes.byref(out)) == rr.RR_INVALID_ARG
    assert "NULL" in rr.rr_last_error()
    X = rr.rr_matrix(4, 3, 0, None, None, None, rr.RR_CSR_BINARY, 0)
    assert L.rr_setup(ctypes.byref(X), 1.0, 1, None, ctypes.byref(out)) == rr.RR_INVALID_ARG
    import numpy as np
    rp = np.zeros(5, np.int64)
    X = rr.rr_matrix(4, 3, 0, rp.ctypes.data, None, None, rr.RR_CSR_BINARY, 0)
    assert L.rr_setup(ctypes.byref(X), -1.0, 1, None, ctypes.byref(out)) == rr.RR_INVALID_ARG
    assert L.rr_setup(ctypes.byref(X), 1.0, 0, None, ctypes.byref(out)) == rr.RR_INVALID_ARG
    assert L.rr_setup(ctypes.byref(X), 1.0, 4, None, ctypes.byref(out)) == rr.RR_INVALID_ARG
    o_bad = rr.rr_default_options(gather=4)
    assert L.rr_setup(ctypes.byref(X), 1.0, 1, ctypes.byref(o_bad), ctypes.byref(out)) == rr.RR_INVALID_ARG
    o_bad = rr.rr_default_options(solver=7)
    assert L.rr_setup(ctypes.byref(X), 1.0, 1, ctypes.byref(o_bad), ctypes.byref(out)) == rr.RR_INVALID_ARG
    X.layout = 7
    assert L.rr_setup(ctypes.byref(X), 1.0, 1, None, ctypes.byref(out)) == rr.RR_INVALID_ARG
    # a dense X needs values and no CSR arrays
    X.layout = rr.RR_DENSE_F32_ROWMAJOR
    assert L.rr_setup(ctypes.byref(X), 1.0, 1, None, ctypes.byref(out)) == rr.RR_INVALID_ARG
