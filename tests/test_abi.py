"""The C-ABI library loads and exports every function include/xdcg.h declares
(no GPU needed: no compute call is made)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "xdcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(xdcg_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2111_09294_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2111_09294_gb300 import build
        build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ["xdcg_setup", "xdcg_solve", "xdcg_solve_host", "xdcg_destroy",
                     "xdcg_status_string", "xdcg_spmv", "xdcg_precond"]:
        assert required in names


def test_library_exports_every_declared_function(lib):
    import ctypes
    from paper_2111_09294_gb300 import _lib
    for name in header_functions():
        assert hasattr(lib, name), name
        assert name in _lib.EXPORTS, name
    # status strings are host-only and safe without a GPU
    assert lib.xdcg_status_string(0) == b"ok"
    assert b"SPD" in lib.xdcg_status_string(2)


def test_options_struct_defaults(lib):
    import ctypes
    from paper_2111_09294_gb300 import _lib
    opt = _lib.Options()
    assert lib.xdcg_default_options(ctypes.byref(opt)) == 0
    assert opt.tol == 1e-8 and opt.max_iter == 10000 and opt.precision == _lib.XDCG_FP64


def test_setup_rejects_null_arguments(lib):
    import ctypes
    ctx = ctypes.c_void_p()
    # host-side validation returns before any CUDA call
    bad = ctypes.c_int32(7)
    assert lib.xdcg_setup(None, None, None, None, None, None, ctypes.byref(bad)) == 1
    assert bad.value == -1
    assert lib.xdcg_setup(ctypes.byref(ctx), None, None, None, None, None, None) == 1


def test_binding_structs_match_the_header_layout(tmp_path):
    # every struct the binding passes across the ABI has the header's size and
    # field offsets: a small C program compiled against include/xdcg.h prints
    # them (gcc; no GPU, no CUDA)
    import ctypes
    import shutil
    import subprocess
    from paper_2111_09294_gb300 import _lib
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = {"xdcg_options": _lib.Options, "xdcg_result": _lib.Result,
               "xdcg_info_t": _lib.Info, "xdcg_matrix": _lib.Matrix,
               "xdcg_deflation": _lib.Deflation, "xdcg_blocks": _lib.Blocks}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "xdcg.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'    printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        cname, key, val = line.split()
        got[(cname, key)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)
