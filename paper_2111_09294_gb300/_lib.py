"""ctypes declarations of the xdcg C ABI (include/xdcg.h).

Argument marshalling only: every step of the solve runs in the CUDA
library.  Importing the library fails loudly when it has not been built.
"""
import ctypes
import os

from ctypes import POINTER, c_char_p, c_double, c_int, c_int32, c_int64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libxdcg.so")

XDCG_HOST, XDCG_DEVICE = 0, 1
XDCG_FP64, XDCG_MIXED = 0, 1
XDCG_BLOCK_JACOBI, XDCG_POINT_JACOBI = 0, 1
XDCG_MAX_BLOCK_DOFS = 4096

STATUS = {0: "XDCG_OK", 1: "XDCG_INVALID_ARG", 2: "XDCG_NOT_SPD_BLOCK",
          3: "XDCG_COARSE_NOT_SPD", 4: "XDCG_BREAKDOWN", 5: "XDCG_NO_CONVERGENCE",
          6: "XDCG_CUDA_ERROR", 7: "XDCG_OOM", 8: "XDCG_TOO_LARGE", 9: "XDCG_TIMEOUT"}

# every function the header declares
EXPORTS = ["xdcg_default_options", "xdcg_setup", "xdcg_setup_update", "xdcg_solve", "xdcg_solve_x0", "xdcg_solve_batch",
           "xdcg_solve_systems", "xdcg_solve_host", "xdcg_get_info", "xdcg_get_history", "xdcg_spmv", "xdcg_spmv_noalloc",
           "xdcg_precond", "xdcg_element_sensitivity", "xdcg_stiffness_gradient",
           "xdcg_coarse_matrix", "xdcg_destroy", "xdcg_status_string"]


class Matrix(ctypes.Structure):
    _fields_ = [("n_nodes", c_int32), ("dof_ptr", c_void_p), ("row_ptr", c_void_p),
                ("col", c_void_p), ("val_ptr", c_void_p), ("val", c_void_p), ("mem", c_int32)]


class Deflation(ctypes.Structure):
    _fields_ = [("n_sub", c_int32), ("sub_of_node", c_void_p), ("coords", c_void_p),
                ("hsign", c_void_p), ("centre", c_void_p), ("enriched_modes", c_int32),
                ("mem", c_int32), ("sub_cols", c_void_p), ("values", c_void_p)]


class Blocks(ctypes.Structure):
    _fields_ = [("n_blocks", c_int32), ("dof_ptr", c_void_p), ("mem", c_int32)]


class Options(ctypes.Structure):
    _fields_ = [("tol", c_double), ("max_iter", c_int32), ("precision", c_int32),
                ("inner_tol", c_double), ("max_outer", c_int32), ("time_spmv", c_int32),
                ("jacobi", c_int32), ("record_history", c_int32), ("max_batch", c_int32),
                ("coarse_fp64", c_int32), ("wait_s", c_double), ("autotune", c_int32),
                ("graph", c_int32), ("spmv_shape_fp32", c_int32), ("spmv_shape_fp64", c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("iterations", c_int32), ("outer_cycles", c_int32),
                ("rel_res_recursive", c_double), ("rel_res_true", c_double),
                ("t_solve_ms", c_double), ("bad_index", c_int32), ("n_spmv_timed", c_int32),
                ("t_spmv_ms", c_double), ("n_launches", c_int64),
                ("n_phase_timed", c_int32), ("t_phase_ms", c_double * 5),
                ("n_fp64_iterations", c_int32), ("n_graph_launches", c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["t_phase_ms"] = list(self.t_phase_ms)
        return d


class Info(ctypes.Structure):
    _fields_ = [("n", c_int64), ("n_nodes", c_int32), ("k", c_int32), ("nnz", c_int64),
                ("nnzb3", c_int64), ("spmv_bytes_fp64", c_int64), ("spmv_bytes_fp32", c_int64),
                ("iter_bytes_fp64", c_int64), ("iter_bytes_fp32", c_int64),
                ("t_setup_ms", c_double), ("restrict_bytes_fp32", c_int64),
                ("coarse_bytes_fp32", c_int64), ("prolong_bytes_fp32", c_int64),
                ("nnzb", c_int64), ("spmv_alg_bytes_fp64", c_int64),
                ("spmv_alg_bytes_fp32", c_int64), ("block_entries", c_int64),
                ("t_setup_phase_ms", c_double * 8), ("reused_node_factors", c_int32),
                ("reused_coarse_inverse", c_int32), ("spmv_shape_fp64", c_int32),
                ("spmv_shape_fp32", c_int32), ("spmv_shape_us_fp64", c_double * 8),
                ("spmv_shape_us_fp32", c_double * 8)]

    PHASES = ("validate", "host_layout", "upload", "factors_W_E", "E_inverse", "fp32_level",
              "blocks", "work_vectors")

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["t_setup_phase_ms"] = dict(zip(self.PHASES, list(self.t_setup_phase_ms)))
        d["spmv_shape_us_fp64"] = list(self.spmv_shape_us_fp64)
        d["spmv_shape_us_fp32"] = list(self.spmv_shape_us_fp32)
        return d


_lib = None


def load():
    """Load libxdcg.so (built by paper_2111_09294_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    lib.xdcg_default_options.argtypes = [POINTER(Options)]
    lib.xdcg_setup.argtypes = [POINTER(c_void_p), POINTER(Matrix), POINTER(Deflation),
                               POINTER(Blocks), POINTER(Options), c_void_p, POINTER(c_int32)]
    lib.xdcg_setup_update.argtypes = [POINTER(c_void_p), c_void_p, POINTER(Matrix),
                                      POINTER(Deflation), POINTER(Blocks), POINTER(Options),
                                      c_void_p, POINTER(c_int32)]
    lib.xdcg_solve.argtypes = [c_void_p, c_void_p, c_void_p, c_double, POINTER(Result)]
    lib.xdcg_solve_x0.argtypes = [c_void_p, c_void_p, c_void_p, c_double, POINTER(Result)]
    lib.xdcg_solve_batch.argtypes = [c_void_p, c_void_p, c_void_p, c_int32, c_double, c_void_p]
    lib.xdcg_solve_host.argtypes = [c_void_p, c_void_p, c_void_p, c_double, POINTER(Result)]
    lib.xdcg_solve_systems.argtypes = [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_double,
                                       c_void_p, c_void_p]
    lib.xdcg_get_info.argtypes = [c_void_p, POINTER(Info)]
    lib.xdcg_get_history.argtypes = [c_void_p, c_void_p, c_int32, POINTER(c_int32)]
    lib.xdcg_spmv.argtypes = [c_void_p, c_int32, c_void_p, c_void_p, POINTER(c_double)]
    lib.xdcg_spmv_noalloc.argtypes = [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]
    lib.xdcg_precond.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.xdcg_element_sensitivity.argtypes = [c_void_p, c_int64, c_void_p, c_void_p, c_void_p,
                                             c_void_p, c_int64, c_void_p, c_void_p, c_void_p]
    lib.xdcg_stiffness_gradient.argtypes = [c_void_p, POINTER(Matrix), c_void_p, c_void_p,
                                            c_void_p]
    lib.xdcg_coarse_matrix.argtypes = [c_void_p, c_void_p]
    lib.xdcg_destroy.argtypes = [c_void_p]
    lib.xdcg_status_string.argtypes = [c_int]
    lib.xdcg_status_string.restype = c_char_p
    for name in EXPORTS:
        if name != "xdcg_status_string":
            getattr(lib, name).restype = c_int
    _lib = lib
    return lib


class XdcgError(RuntimeError):
    def __init__(self, status, what, bad_index=-1):
        self.status = status
        self.bad_index = bad_index
        msg = load().xdcg_status_string(status).decode()
        super().__init__(f"{what}: {STATUS.get(status, status)} ({msg})"
                         + (f", index {bad_index}" if bad_index >= 0 else ""))


def check(status, what, bad_index=-1):
    if status != 0:
        raise XdcgError(status, what, bad_index)
