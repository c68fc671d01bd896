"""xdcg_spmv_noalloc: the SpMV entry point for callers that cannot allocate
device memory where they call it (code running while another allocator holds
the device memory budget, or on a latency-critical path where cudaMalloc
could synchronise the device).  Its reduction scratch lives in a fixed device
array inside the library.

Two calls in a row are checked against the oracle's product: K x for the
FP64 operator, and the oracle-built block-scaled K~ x = L^-1 K L^-T x for the
FP32 one, within the tolerances of the SpMV parity tests; the second call
also shows that the shared scratch left by the first is cleared.  Collected
last on purpose: it exercises the shared scratch after every other test has
used the library, and it passes alone in a fresh process as well."""
import ctypes

import numpy as np
import pytest
import scipy.sparse as sp

import xfem_inputs as X
from oracle import adef2 as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _block_inverse_factor(M, shape):
    """Block-diagonal inverse of the oracle's node-block Cholesky factors."""
    r, c, v = [], [], []
    for idx, L in M.groups:
        Linv = np.linalg.inv(L)
        for t in range(idx.shape[0]):
            rr, cc = np.meshgrid(idx[t], idx[t], indexing="ij")
            r.append(rr.ravel()); c.append(cc.ravel()); v.append(Linv[t].ravel())
    return sp.csr_matrix((np.concatenate(v), (np.concatenate(r), np.concatenate(c))), shape=shape)


@pytest.mark.parametrize("name", ["cube8_edge", "cube24_ellipse"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_spmv_matches_oracle_on_consecutive_calls(name, prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_09294_gb300 import Solver, _lib
    lib = _lib.load()
    dev = torch.device("cuda:0")
    P = X.make(name)
    K = O.stiffness_csr(P)
    s = Solver.from_problem(P, precision="mixed")
    dt = torch.float64 if prec == "fp64" else torch.float32
    code = _lib.XDCG_FP64 if prec == "fp64" else _lib.XDCG_MIXED
    rng = np.random.default_rng(3)
    x = torch.tensor(rng.standard_normal(P.n), dtype=dt, device=dev)
    xd = x.double().cpu().numpy()           # the FP32 input's exact values for FP32
    # the oracle's operator and the tolerances of the SpMV parity tests,
    # relative to |A| |x| per row
    if prec == "fp64":
        A = K
        tol = 1e-12
    else:
        Li = _block_inverse_factor(O.BlockJacobi(K, P.dof_ptr), K.shape)
        A = (Li @ K @ Li.T).tocsr()
        tol = 2e-5
    y_ref = A @ xd
    xty_ref = xd @ y_ref
    bound = tol * (abs(A) @ np.abs(xd))
    for call in range(2):
        y = torch.full_like(x, float("nan"))
        out = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        st = lib.xdcg_spmv_noalloc(s.ctx, code, ctypes.c_void_p(x.data_ptr()),
                                   ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(out.data_ptr()))
        assert st == 0, _lib.STATUS.get(st, st)
        torch.cuda.synchronize()
        yn = y.double().cpu().numpy()
        assert np.all(np.isfinite(yn))
        assert np.all(np.abs(yn - y_ref) <= bound), call
        assert abs(out.item() - xty_ref) <= np.sum(np.abs(xd) * bound), call
    s.close()


def test_noalloc_rejects_bad_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_09294_gb300 import Solver, _lib
    lib = _lib.load()
    P = X.make("cube8_edge")
    s = Solver.from_problem(P)                     # FP64 only: no FP32 operator
    x = torch.zeros(P.n, dtype=torch.float32, device="cuda:0")
    y = torch.zeros_like(x)
    st = lib.xdcg_spmv_noalloc(s.ctx, _lib.XDCG_MIXED, ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(y.data_ptr()), None)
    assert st == 1
    st = lib.xdcg_spmv_noalloc(s.ctx, 7, ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(y.data_ptr()), None)
    assert st == 1
    s.close()
