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
    o_bad = rr.rr_default_options(clustering=2)
    assert L.rr_setup(ctypes.byref(X), 1.0, 1, ctypes.byref(o_bad), ctypes.byref(out)) == rr.RR_INVALID_ARG
    o_bad = rr.rr_default_options(clustering=rr.RR_CLUSTER_LEADER, lf_tol2=float("nan"))
    assert L.rr_setup(ctypes.byref(X), 1.0, 1, ctypes.byref(o_bad), ctypes.byref(out)) == rr.RR_INVALID_ARG
    assert "leader-follower" in rr.rr_last_error()
    X.layout = 7
    assert L.rr_setup(ctypes.byref(X), 1.0, 1, None, ctypes.byref(out)) == rr.RR_INVALID_ARG
    # a dense X needs values and no CSR arrays
    X.layout = rr.RR_DENSE_F32_ROWMAJOR
    assert L.rr_setup(ctypes.byref(X), 1.0, 1, None, ctypes.byref(out)) == rr.RR_INVALID_ARG
    # a fork needs a base handle and a place for the result; its lambda is checked
    assert L.rr_fork_lambda(None, 1.0, ctypes.byref(out)) == rr.RR_INVALID_ARG
    assert "rr_fork_lambda" in rr.rr_last_error()
    assert L.rr_solve_many(0, None, None, None, 1e-8, None, None) == rr.RR_INVALID_ARG


def header_prototypes():
    """{name: number of parameters} of every function include/rr.h declares."""
    text = open(os.path.join(ROOT, "include", "rr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for name, params in re.findall(r"\b(rr_[a-z_]+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
        params = params.strip()
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_the_header():
    """Every ctypes signature of the binding takes as many arguments as the
    header's prototype (a mismatch would pass garbage across the C ABI)."""
    from paper_1806_05826_gb300 import rr
    protos = header_prototypes()
    assert len(protos) == len(header_functions())
    for name, (_, argtypes) in rr._SIGS.items():
        assert name in protos, name
        assert len(argtypes) == protos[name], (name, len(argtypes), protos[name])


def test_struct_layouts_match_the_header():
    """The binding's ctypes structures list the header's fields in order."""
    from paper_1806_05826_gb300 import rr
    text = open(os.path.join(ROOT, "include", "rr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    for cname, py in (("rr_matrix", rr.rr_matrix), ("rr_options", rr.rr_options),
                      ("rr_info", rr.rr_info)):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname + r"\s*;", text).group(1)
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            names = decl.split(None, 1)[1] if not decl.startswith("const ") else decl.split(None, 2)[2]
            for n in names.split(","):
                fields.append(re.sub(r"[\s*]|\[.*\]", "", n))
        assert [f[0] for f in py._fields_] == fields, cname


def test_struct_offsets_match_the_c_compiler(tmp_path):
    """Field offsets and sizes of the binding's structures equal those gcc
    gives the header's structures (the layout the library was built with)."""
    import shutil
    import subprocess
    from paper_1806_05826_gb300 import rr
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = (("rr_matrix", rr.rr_matrix), ("rr_options", rr.rr_options), ("rr_info", rr.rr_info))
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rr.h"', "int main(void) {"]
    for cname, py in structs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'  printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    want = {}
    for line in got:
        if line:
            cname, field, value = line.split()
            want[(cname, field)] = int(value)
    for cname, py in structs:
        assert ctypes.sizeof(py) == want[(cname, "size")], cname
        for f in py._fields_:
            assert getattr(py, f[0]).offset == want[(cname, f[0])], (cname, f[0])
