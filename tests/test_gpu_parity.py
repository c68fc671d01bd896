"""GPU parity: the CUDA path against the FP64 oracle on the same seeded inputs.

Tolerances:
* SpMV FP64: |y - y_ref|_i <= 1e-12 (|K| |x|)_i  (reordered FP64 sums);
* SpMV FP32: |y - y_ref|_i <= 2e-5 (|K| |x|)_i   (FP32 values, FP32 sums of
  up to ~140 terms: a few hundred ulps of 6e-8);
* E: |E - E_ref| <= 1e-12 max|E_ref|;
* preconditioner: ||z - z_ref|| <= 1e-8 ||z_ref|| (block solves with
  condition numbers up to ~5e7 and the coarse inverse, rounding only);
* solves: iteration counts within +-2 of the oracle at tol 1e-8, and at
  tol 1e-12 ||u - u_ref|| <= 1e-7 ||u_ref||, true residual <= tol.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import xfem_inputs as X
from oracle import adef2 as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CONFIGS = ["cube8_edge", "cube24_ellipse"]


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


_cache = {}


def problem(name):
    if name not in _cache:
        P = X.make(name)
        K, M, C = O.setup(P)
        _cache[name] = (P, K, M, C)
    return _cache[name]


def solver(P, **kw):
    from paper_2111_09294_gb300 import Solver
    _cuda()
    return Solver.from_problem(P, **kw)


@pytest.mark.parametrize("name", CONFIGS)
def test_spmv_fp64_and_fp32(name):
    dev = _cuda()
    P, K, M, C = problem(name)
    s = solver(P, precision="mixed")
    rng = np.random.default_rng(7)
    x = rng.standard_normal(P.n)
    y_ref = K @ x
    bound = abs(K) @ np.abs(x)
    y, xty = s.spmv(torch.tensor(x, device=dev), "fp64")
    y = y.cpu().numpy()
    assert np.all(np.abs(y - y_ref) <= 1e-12 * bound)
    assert abs(xty - x @ y_ref) <= 1e-12 * (np.abs(x) @ bound)
    # the FP32 operator is the block-scaled K~ = L^-1 K L^-T (L: node-block factors)
    Lb, Li = block_factor_matrices(M, K.shape)
    Kt = (Li @ K @ Li.T).tocsr()
    x32 = x.astype(np.float32)
    y32, _ = s.spmv(torch.tensor(x32, device=dev), "mixed")
    yr32 = Kt @ x32.astype(np.float64)
    assert np.all(np.abs(y32.cpu().numpy() - yr32) <= 2e-5 * (abs(Kt) @ np.abs(x32)))
    s.close()


def block_factor_matrices(M, shape):
    """Block-diagonal Cholesky factor L of the oracle's node blocks and its inverse."""
    r, c, v, vi = [], [], [], []
    for idx, L in M.groups:
        Linv = np.linalg.inv(L)
        for t in range(idx.shape[0]):
            rr, cc = np.meshgrid(idx[t], idx[t], indexing="ij")
            r.append(rr.ravel()); c.append(cc.ravel())
            v.append(L[t].ravel()); vi.append(Linv[t].ravel())
    r, c = np.concatenate(r), np.concatenate(c)
    return (sp.csr_matrix((np.concatenate(v), (r, c)), shape=shape),
            sp.csr_matrix((np.concatenate(vi), (r, c)), shape=shape))


@pytest.mark.parametrize("name", CONFIGS)
def test_coarse_matrix(name):
    P, K, M, C = problem(name)
    s = solver(P)
    E = s.coarse_matrix()
    assert E.shape == C.E.shape
    assert np.max(np.abs(E - C.E)) <= 1e-12 * np.max(np.abs(C.E))
    s.close()


@pytest.mark.parametrize("name", CONFIGS)
def test_preconditioner(name):
    dev = _cuda()
    P, K, M, C = problem(name)
    s = solver(P)
    rng = np.random.default_rng(11)
    for _ in range(2):
        r = rng.standard_normal(P.n)
        z_ref = O.adef2_apply(K, M, C, r)
        z = s.precond(torch.tensor(r, device=dev)).cpu().numpy()
        assert np.linalg.norm(z - z_ref) <= 1e-8 * np.linalg.norm(z_ref)
    s.close()


@pytest.mark.parametrize("name", CONFIGS)
def test_fp64_solve_matches_oracle(name):
    dev = _cuda()
    P, K, M, C = problem(name)
    ref8 = O.adef2_pcg(K, P.f, M, C, tol=1e-8)
    ref12 = O.adef2_pcg(K, P.f, M, C, tol=1e-12)
    s = solver(P)
    f = torch.tensor(P.f, device=dev)
    u, info = s.solve(f, tol=1e-8)
    assert abs(info["iterations"] - ref8.iterations) <= 2
    assert info["rel_res_true"] <= 1.01e-8
    res_cpu = np.linalg.norm(P.f - K @ u.cpu().numpy()) / np.linalg.norm(P.f)
    assert res_cpu <= 1.05e-8
    u12, info12 = s.solve(f, tol=1e-12)
    assert abs(info12["iterations"] - ref12.iterations) <= 2
    err = np.linalg.norm(u12.cpu().numpy() - ref12.u) / np.linalg.norm(ref12.u)
    assert err <= 1e-7
    # the final residual is orthogonal to the deflation space (A-DEF2 invariant)
    rt = P.f - K @ u12.cpu().numpy()
    assert np.linalg.norm(C.Z.T @ rt) <= 1e-10 * sp.linalg.norm(C.Z) * np.linalg.norm(P.f)
    s.close()


@pytest.mark.parametrize("name", CONFIGS)
def test_mixed_solve_matches_oracle(name):
    dev = _cuda()
    P, K, M, C = problem(name)
    ref12 = O.adef2_pcg(K, P.f, M, C, tol=1e-12)
    s = solver(P, precision="mixed")
    f = torch.tensor(P.f, device=dev)
    u, info = s.solve(f, tol=1e-8)
    assert info["rel_res_true"] <= 1e-8
    res_cpu = np.linalg.norm(P.f - K @ u.cpu().numpy()) / np.linalg.norm(P.f)
    assert res_cpu <= 1.05e-8
    u12, info12 = s.solve(f, tol=1e-12)
    assert info12["rel_res_true"] <= 1e-12
    err = np.linalg.norm(u12.cpu().numpy() - ref12.u) / np.linalg.norm(ref12.u)
    assert err <= 1e-7
    s.close()


def test_solves_are_deterministic():
    dev = _cuda()
    P, K, M, C = problem("cube24_ellipse")
    s = solver(P)
    f = torch.tensor(P.f, device=dev)
    u1, i1 = s.solve(f, tol=1e-8)
    u2, i2 = s.solve(f, tol=1e-8)
    assert i1["iterations"] == i2["iterations"]
    assert torch.equal(u1, u2)
    s.close()


def test_host_memory_solve_matches_device_solve():
    dev = _cuda()
    P, K, M, C = problem("cube8_edge")
    s = solver(P)
    f = torch.tensor(P.f, device=dev)
    u, _ = s.solve(f, tol=1e-8)
    uh = np.empty(P.n)
    s.solve_host(np.ascontiguousarray(P.f), uh, tol=1e-8)
    assert np.array_equal(uh, u.cpu().numpy())
    s.close()
