"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/panda.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "panda.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(panda_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1607_08220_gb300 import build_ext, panda
    path = build_ext.build()
    assert os.path.exists(path)
    return panda.load(path), path


def test_header_declares_the_boundary():
    fns = declared_functions()
    for name in ("panda_build", "panda_knn", "panda_free", "panda_build_async", "panda_knn_async",
                 "panda_build_host", "panda_knn_host", "panda_status_string", "panda_last_error"):
        assert name in fns


def test_every_declared_symbol_is_exported(lib):
    L, path = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (panda_[a-z_]+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    for f in declared_functions():
        assert getattr(L, f) is not None


def test_binding_covers_header(lib):
    from paper_1607_08220_gb300 import panda
    assert set(panda.SIGNATURES) == set(declared_functions())


def test_status_strings_and_argument_checks(lib):
    L, _ = lib
    assert L.panda_status_string(0) == b"ok"
    assert L.panda_status_string(8) == b"depth limit exceeded"
    h = ctypes.c_void_p()
    # rejected before any device work: NULL points, bad sizes, unsupported d
    assert L.panda_build(None, 10, 3, 32, ctypes.byref(h)) == 1
    assert L.panda_build(ctypes.c_void_p(16), 0, 3, 32, ctypes.byref(h)) == 1
    assert L.panda_build(ctypes.c_void_p(16), 10, 17, 32, ctypes.byref(h)) == 3
    assert L.panda_build(ctypes.c_void_p(16), 10, 3, 0, ctypes.byref(h)) == 1
    assert L.panda_build(ctypes.c_void_p(16), 10, 3, 257, ctypes.byref(h)) == 3
    assert b"invalid" in L.panda_last_error() or b"unsupported" in L.panda_last_error()
    assert L.panda_knn(None, None, 0, 5, None, None) == 1
    L.panda_free(None)


def test_struct_layouts_match_the_binding(tmp_path):
    """Every struct the binding passes by pointer has the C layout: size and
    field offsets from a C program compiled against include/panda.h."""
    from paper_1607_08220_gb300 import panda
    structs = {"panda_query_params": panda.QueryParams, "panda_tree_info": panda.TreeInfo,
               "panda_set_desc": panda.SetDesc, "panda_tune_result": panda.TuneResult}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "panda.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            cname, field, val = line.split()
            got[(cname, field)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
