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
