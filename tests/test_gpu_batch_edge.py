"""Batched solves at their edges: each column leaves on its own outcome (a
non-finite load case, the iteration cap, the replacement cap), a bounded
copy wait that runs out ends the call with XDCG_TIMEOUT (one system, and one
system of a fused call over several), and the contexts stay usable."""
import numpy as np
import pytest

import xfem_inputs as X
from oracle import adef2 as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _solver(P, **kw):
    from paper_2111_09294_gb300 import Solver
    _cuda()
    return Solver.from_problem(P, precision="mixed", **kw)


def test_nonfinite_column_breaks_down_alone():
    # column 1 holds a NaN: it leaves at the start (bad_index 1); the other
    # columns are solved as the oracle solves them
    dev = _cuda()
    P = X.make("cube8_edge")
    K, M, C = O.setup(P)
    F = X.load_cases(P, 3, seed=21)
    F[1, 7] = np.nan
    s = _solver(P, max_batch=4)
    U, infos = s.solve_batch(torch.tensor(F, device=dev), tol=1e-10, raise_on_error=False)
    assert infos[1]["bad_index"] == 1 and infos[1]["status"] == "XDCG_BREAKDOWN"
    Un = U.cpu().numpy()
    for j in (0, 2):
        assert infos[j]["bad_index"] == -1 and infos[j]["rel_res_true"] <= 1e-10
        ref = O.adef2_pcg(K, F[j], M, C, tol=1e-10)
        assert np.linalg.norm(Un[j] - ref.u) <= 1e-6 * np.linalg.norm(ref.u)
    s.close()


def test_iteration_cap_ends_every_column():
    dev = _cuda()
    P = X.make("cube8_edge")
    F = X.load_cases(P, 2, seed=22)
    s = _solver(P, max_batch=2, max_iter=5)
    U, infos = s.solve_batch(torch.tensor(F, device=dev), tol=1e-10, raise_on_error=False)
    for i in infos:
        assert i["status"] == "XDCG_NO_CONVERGENCE"
        assert i["iterations"] == 5 and i["outer_cycles"] == 1
        # CG minimises the error in the energy norm, not ||f - K u||: after 5
        # iterations the relative residual may still exceed 1; it is finite
        assert np.isfinite(i["rel_res_true"]) and i["rel_res_true"] > 0.0
    assert np.isfinite(U.cpu().numpy()).all()
    s.close()


def test_replacement_cap_ends_every_column():
    # max_outer 1: each column leaves at its first FP64 residual replacement,
    # about inner_tol below its start, far from tol
    dev = _cuda()
    P = X.make("cube24_ellipse")
    F = X.load_cases(P, 4, seed=23)
    s = _solver(P, max_batch=4, max_outer=1)
    U, infos = s.solve_batch(torch.tensor(F, device=dev), tol=1e-12, raise_on_error=False)
    for i in infos:
        assert i["status"] == "XDCG_NO_CONVERGENCE" and i["outer_cycles"] == 1
        assert 1e-12 < i["rel_res_true"] < 1e-1 and i["iterations"] > 0
    s.close()


def test_bounded_wait_timeout_in_batched_and_fused_calls():
    dev = _cuda()
    from paper_2111_09294_gb300 import sweep as S
    from paper_2111_09294_gb300._lib import XdcgError
    P = X.make("cube24_ellipse")
    F = torch.tensor(X.load_cases(P, 2, seed=24), device=dev)
    bad = _solver(P, max_batch=2, wait_s=0.0)
    _, infos = bad.solve_batch(F, tol=1e-8, raise_on_error=False)
    assert all(i["status"] == "XDCG_TIMEOUT" for i in infos)
    # the same context inside a fused call over two systems
    good = _solver(P, max_batch=2, stream=torch.cuda.Stream())
    with pytest.raises(XdcgError, match="TIMEOUT"):
        S.solve_systems([good, bad], [F, F.clone()], 1e-8, fused=True)
    bad.close()
    torch.cuda.synchronize()
    # the other context still solves, alone and fused with a fresh one
    U, infos = good.solve_batch(F, tol=1e-8)
    assert all(i["rel_res_true"] <= 1e-8 for i in infos)
    fresh = _solver(P, max_batch=2, stream=torch.cuda.Stream())
    res = S.solve_systems([good, fresh], [F, F.clone()], 1e-8, fused=True)
    assert torch.equal(res[0][0], U) and torch.equal(res[1][0], U)
    good.close()
    fresh.close()
