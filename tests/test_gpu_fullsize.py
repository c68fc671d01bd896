"""GPU parity at the benchmark size (48^3 hexes, two warped cracks, 8^3
boxes: n = 373,254, k = 3,240), in the configuration bench.py times.

The oracle computes everything here at this size within about a minute:
full products K x, the coarse matrix E, one application of Algorithm 3 and
the FP64 A-DEF2 solve to 1e-8 and to 1e-12.  Tolerances are those of the
smaller parity tests (test_gpu_parity.py): iterations within +-2 at 1e-8 and
||u - u_ref|| <= 1e-7 ||u_ref|| with both run to 1e-12, for the FP64 and the
mixed path; Algorithm 3's sensitivity to rounding at this size is measured
in the test itself."""
import numpy as np
import pytest
import scipy.sparse as sp

import xfem_inputs as X
from oracle import adef2 as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAME = "cube48_two_cracks"
_state = {}


def setup_module(module):
    if not torch.cuda.is_available():
        return
    P = X.make(NAME)
    K, M, C = O.setup(P)
    _state.update(P=P, K=K, M=M, C=C)


def _need():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return _state["P"], _state["K"], _state["M"], _state["C"]


def _solver(**kw):
    from paper_2111_09294_gb300 import Solver
    return Solver.from_problem(_state["P"], **kw)


def test_spmv_fp64_and_fp32_full_size():
    P, K, M, C = _need()
    s = _solver(precision="mixed")
    dev = torch.device("cuda:0")
    x = np.random.default_rng(5).standard_normal(P.n)
    y, _ = s.spmv(torch.tensor(x, device=dev), "fp64")
    assert np.all(np.abs(y.cpu().numpy() - K @ x) <= 1e-12 * (abs(K) @ np.abs(x)))
    # FP32 operator K~ = L^-1 K L^-T on a sample of 4000 rows
    r, c, v = [], [], []
    for idx, L in M.groups:
        Li = np.linalg.inv(L)
        for t in range(idx.shape[0]):
            rr, cc = np.meshgrid(idx[t], idx[t], indexing="ij")
            r.append(rr.ravel()); c.append(cc.ravel()); v.append(Li[t].ravel())
    Linv = sp.csr_matrix((np.concatenate(v), (np.concatenate(r), np.concatenate(c))), shape=K.shape)
    x32 = x.astype(np.float32)
    y32, _ = s.spmv(torch.tensor(x32, device=dev), "mixed")
    rows = np.random.default_rng(6).choice(P.n, 4000, replace=False)
    Kt_rows = (Linv[rows] @ K @ Linv.T).tocsr()
    ref = Kt_rows @ x32.astype(np.float64)
    assert np.all(np.abs(y32.cpu().numpy()[rows] - ref) <= 2e-5 * (abs(Kt_rows) @ np.abs(x32)))
    s.close()


def test_coarse_matrix_and_preconditioner_full_size():
    P, K, M, C = _need()
    s = _solver()
    E = s.coarse_matrix()
    assert np.max(np.abs(E - C.E)) <= 1e-12 * np.max(np.abs(C.E))
    r = np.random.default_rng(8).standard_normal(P.n)
    z_ref = O.adef2_apply(K, M, C, r)
    z = s.precond(torch.tensor(r, device="cuda:0")).cpu().numpy()
    # Some jump-node blocks here are nearly singular (condition numbers up to
    # ~1e12), so M^-1 r is that sensitive to the rounding of the block
    # factorisation.  The scale of a correct result's error is what the oracle
    # gives when every block entry is perturbed by one unit in the last place
    # before factoring: the GPU result must lie within ten times that.
    sens = np.linalg.norm(_perturbed_apply(K, M, C, r) - z_ref)
    assert np.linalg.norm(z - z_ref) <= 10.0 * sens + 1e-12 * np.linalg.norm(z_ref)
    s.close()


def _perturbed_apply(K, M, C, r):
    """Algorithm 3 with block Jacobi factors of the node blocks perturbed
    entrywise by a relative 2^-52 (seeded), everything else as the oracle."""
    eps = np.finfo(np.float64).eps
    rng = np.random.default_rng(0)
    y = np.empty_like(r)
    for idx, L in M.groups:
        B = L @ np.swapaxes(L, 1, 2)
        B = B * (1.0 + eps * rng.uniform(-1.0, 1.0, B.shape))
        Lp = np.linalg.cholesky(0.5 * (B + np.swapaxes(B, 1, 2)))
        w = np.linalg.solve(Lp, r[idx][:, :, None])
        y[idx] = np.linalg.solve(np.swapaxes(Lp, 1, 2), w)[:, :, 0]
    return y + C.Z @ (C.solve(C.Z.T @ r) - C.solve(C.Z.T @ (K @ y)))


def test_fp64_and_mixed_solves_full_size():
    # at the benchmark's tolerance: the FP64 iteration count within +-2 of
    # the oracle's, both paths' true residuals, and Z^T r = 0 (Section 3.2)
    P, K, M, C = _need()
    ref = O.adef2_pcg(K, P.f, M, C, tol=1e-8)
    f = torch.tensor(P.f, device="cuda:0")
    fn = np.linalg.norm(P.f)
    zn = sp.linalg.norm(C.Z)
    s = _solver()
    u, info = s.solve(f, tol=1e-8)
    un = u.cpu().numpy()
    assert abs(info["iterations"] - ref.iterations) <= 2
    rt = P.f - K @ un
    assert np.linalg.norm(rt) <= 1.05e-8 * fn
    assert np.linalg.norm(C.Z.T @ rt) <= 1e-10 * zn * fn
    s.close()
    sm = _solver(precision="mixed")
    um, infom = sm.solve(f, tol=1e-8)
    rtm = P.f - K @ um.cpu().numpy()
    assert np.linalg.norm(rtm) <= 1.0e-8 * fn * 1.001
    assert infom["rel_res_true"] <= 1e-8
    # the mixed path's inner FP32 iterations against the oracle's FP64 count:
    # a stated figure per result (its own recurrence, replaced residuals), not
    # bound to +-2; print it for the record and keep it within 25 %
    print(f"\n48^3 iterations to 1e-8: oracle {ref.iterations}, GPU FP64 {info['iterations']}, "
          f"mixed {infom['iterations']} inner / {infom['outer_cycles']} FP64 residuals")
    assert infom["iterations"] <= 1.25 * ref.iterations
    sm.close()


def test_solutions_full_size_at_tight_tolerance():
    # u against the oracle's u with both run to 1e-12 (two runs stopped at
    # 1e-8 one iteration apart can differ by more than 1e-7):
    # ||u - u_ref|| <= 1e-7 ||u_ref|| for the FP64 and the mixed path
    P, K, M, C = _need()
    ref = O.adef2_pcg(K, P.f, M, C, tol=1e-12)
    assert ref.converged
    f = torch.tensor(P.f, device="cuda:0")
    fn = np.linalg.norm(P.f)
    un_ref = np.linalg.norm(ref.u)
    for prec in ("fp64", "mixed"):
        s = _solver(precision=prec)
        u, info = s.solve(f, tol=1e-12)
        un = u.cpu().numpy()
        assert np.linalg.norm(P.f - K @ un) <= 1.05e-12 * fn, (prec, info)
        err = np.linalg.norm(un - ref.u) / un_ref
        print(f"\n48^3 at 1e-12, {prec}: ||u - u_ref|| / ||u_ref|| = {err:.2e}, "
              f"iterations {info['iterations']} (oracle {ref.iterations})")
        assert err <= 1e-7, (prec, err)
        s.close()


def test_element_sensitivity_full_size():
    # every element at 48^3 on the GPU (5,058 enriched elements with their
    # own matrices, the rest sharing one); the oracle's formula on a sample
    # of 2,000 standard elements and all enriched ones, same seeded u and lam
    P = _need()[0]
    from paper_2111_09294_gb300 import Elements
    D = X.element_data(P)
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(71)
    u, lam = rng.standard_normal(P.n), rng.standard_normal(P.n)
    s = _solver()
    g = s.element_sensitivity(Elements.from_dict(D, dev), torch.tensor(u, device=dev),
                              torch.tensor(lam, device=dev)).cpu().numpy()
    enr = np.asarray(P.enr_elements)
    std = np.setdiff1d(np.arange(len(g)), enr)
    sample = np.concatenate([enr, rng.choice(std, 2000, replace=False)])
    ref = O.element_sensitivity(D, u, lam, sample)
    Da = dict(D)
    Da["mats"] = np.abs(D["mats"])
    scale = -O.element_sensitivity(Da, np.abs(u), np.abs(lam), sample)
    assert np.all(np.abs(g[sample] - ref) <= 1e-13 * scale)
    assert np.all(np.isfinite(g))
    s.close()
