"""GPU edge cases and error statuses, all raised from host-side inputs: zero
and tiny systems, ragged sizes, iteration caps, non-finite loads, an
indefinite node block, an asymmetric matrix and unsupported arguments."""
import numpy as np
import pytest

import xfem_inputs as X
from oracle import adef2 as O
from xfem_inputs.cracks import PlanarEdgeCrack, WarpedPennyCrack

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _solver(P, **kw):
    from paper_2111_09294_gb300 import Solver
    _cuda()
    return Solver.from_problem(P, **kw)


def test_zero_load_gives_zero_solution():
    dev = _cuda()
    P = X.make("cube8_edge")
    s = _solver(P)
    u, info = s.solve(torch.zeros(P.n, dtype=torch.float64, device=dev))
    assert info["iterations"] == 0
    assert torch.count_nonzero(u).item() == 0
    sm = _solver(P, precision="mixed")
    u, info = sm.solve(torch.zeros(P.n, dtype=torch.float64, device=dev))
    assert info["iterations"] == 0 and torch.count_nonzero(u).item() == 0


@pytest.mark.parametrize("m,nb", [(1, 1), (2, 1), (3, 2), (5, 3)])
def test_tiny_and_ragged_meshes(m, nb):
    # sizes that leave partial SpMV slices, boxes with few nodes, no enrichment
    dev = _cuda()
    cracks = [PlanarEdgeCrack(0.43, 0.6, 0.15)] if m >= 3 else []
    P = X.build_problem(m, cracks, nb)
    K, Mj, C = O.setup(P)
    ref = O.adef2_pcg(K, P.f, Mj, C, tol=1e-12)
    for prec in ("fp64", "mixed"):
        s = _solver(P, precision=prec)
        u, info = s.solve(torch.tensor(P.f, device=dev), tol=1e-12)
        err = np.linalg.norm(u.cpu().numpy() - ref.u) / np.linalg.norm(ref.u)
        assert err <= 1e-7, (prec, err)


def test_iteration_cap_reports_no_convergence():
    dev = _cuda()
    P = X.make("cube8_edge")
    from paper_2111_09294_gb300 import XdcgError
    s = _solver(P, max_iter=5)
    u, info = s.solve(torch.tensor(P.f, device=dev), raise_on_error=False)
    assert info["status"] == "XDCG_NO_CONVERGENCE"
    assert info["iterations"] == 5
    assert np.isfinite(u.cpu().numpy()).all()
    with pytest.raises(XdcgError):
        s.solve(torch.tensor(P.f, device=dev))


def test_nonfinite_load_reports_breakdown():
    dev = _cuda()
    P = X.make("cube8_edge")
    s = _solver(P)
    f = torch.tensor(P.f, device=dev)
    f[10] = float("nan")
    _, info = s.solve(f, raise_on_error=False)
    assert info["status"] in ("XDCG_BREAKDOWN", "XDCG_NO_CONVERGENCE")
    assert info["status"] == "XDCG_BREAKDOWN"


def test_indefinite_block_is_rejected_at_setup():
    _cuda()
    from paper_2111_09294_gb300 import XdcgError
    P = X.make("cube8_edge")
    val = P.val.copy()
    I = 5
    p = [q for q in range(P.row_ptr[I], P.row_ptr[I + 1]) if P.col[q] == I][0]
    val[P.val_ptr[p]] = -1.0           # first diagonal entry of node 5
    from paper_2111_09294_gb300 import Solver
    with pytest.raises(XdcgError) as ei:
        Solver(P.dof_ptr, P.row_ptr, P.col, P.val_ptr, val, P.sub_of_node, P.coords, P.hsign,
               P.centres)
    assert ei.value.status == 2 and ei.value.bad_index == I


def test_asymmetric_matrix_is_rejected():
    _cuda()
    from paper_2111_09294_gb300 import Solver, XdcgError
    P = X.make("cube8_edge")
    val = P.val.copy()
    p = P.row_ptr[3]                    # first off-diagonal block of node 3
    val[P.val_ptr[p]] += 1e-3
    with pytest.raises(XdcgError) as ei:
        Solver(P.dof_ptr, P.row_ptr, P.col, P.val_ptr, val, P.sub_of_node, P.coords, P.hsign,
               P.centres)
    assert ei.value.status == 1


def test_rank_deficient_deflation_is_rejected():
    # every node placed at one point: the rotation columns vanish, E is singular
    _cuda()
    from paper_2111_09294_gb300 import Solver, XdcgError
    P = X.make("cube8_edge")
    centres = P.centres.copy()
    coords = np.repeat(centres[P.sub_of_node], 1, axis=0)
    with pytest.raises(XdcgError) as ei:
        Solver(P.dof_ptr, P.row_ptr, P.col, P.val_ptr, P.val, P.sub_of_node, coords, P.hsign,
               centres)
    assert ei.value.status == 3


def test_rigid_only_deflation_matches_oracle():
    dev = _cuda()
    P = X.build_problem(6, [WarpedPennyCrack((0.5, 0.5, 0.5), 0.3, 0.02, 0.1)], 2)
    K, M, C = O.setup(P, enriched_modes=False)
    ref = O.adef2_pcg(K, P.f, M, C, tol=1e-8)
    s = _solver(P, enriched_modes=False)
    assert s.k == C.k
    _, info = s.solve(torch.tensor(P.f, device=dev), tol=1e-8)
    assert abs(info["iterations"] - ref.iterations) <= 2


@pytest.mark.parametrize("prec,nphase", [("fp64", 5), ("mixed", 4)])
def test_kernel_timing_mode_times_every_iteration(prec, nphase):
    # time_spmv = 2: CUDA events around every kernel of the loop; results
    # must be those of the untimed solve
    dev = _cuda()
    P = X.make("cube8_edge")
    f = torch.tensor(P.f, device=dev)
    u0, i0 = _solver(P, precision=prec).solve(f)
    u1, i1 = _solver(P, precision=prec, time_spmv="kernels").solve(f)
    assert torch.equal(u0, u1)
    assert i1["iterations"] == i0["iterations"]
    assert i1["n_phase_timed"] == i1["iterations"] == i1["n_spmv_timed"]
    t = i1["t_phase_ms"]
    assert all(x > 0 for x in t[:nphase]) and all(x == 0 for x in t[nphase:])
    assert abs(t[0] - i1["t_spmv_ms"]) <= 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bounded_copy_wait_that_runs_out_reports_timeout(prec):
    # The SpMV waits for its own bulk copies with a limit (xdcg_options.wait_s);
    # with no time allowed, the waits give up while copies are still in
    # flight.  The kernel flags the failure, lets every issued copy land
    # (that drain keeps its own fixed limit) and returns; the call reports
    # XDCG_TIMEOUT.  The context is then destroyed cleanly, and a fresh one on
    # the same device solves correctly.
    dev = _cuda()
    P = X.make("cube24_ellipse")
    f = torch.tensor(P.f, device=dev)
    s = _solver(P, precision=prec, wait_s=0.0)
    u, info = s.solve(f, tol=1e-8, raise_on_error=False)
    assert info["status"] == "XDCG_TIMEOUT", info
    s.close()
    torch.cuda.synchronize()
    s2 = _solver(P, precision=prec)
    u, info = s2.solve(f, tol=1e-8)
    assert info["rel_res_true"] <= 1e-8 * 1.01
    s2.close()


def test_mixed_solve_with_fp64_coarse_matches_oracle():
    # the mixed path with E^-1 applied in FP64 inside the FP32 iteration: the
    # same answer as the oracle's at 1e-12, as with the FP32 copy
    dev = _cuda()
    P = X.make("cube24_ellipse")
    K, M, C = O.setup(P)
    ref = O.adef2_pcg(K, P.f, M, C, tol=1e-12)
    f = torch.tensor(P.f, device=dev)
    for fp64 in (False, True):
        s = _solver(P, precision="mixed", coarse_fp64=fp64)
        u, info = s.solve(f, tol=1e-12)
        un = u.cpu().numpy()
        assert np.linalg.norm(P.f - K @ un) <= 1.05e-12 * np.linalg.norm(P.f)
        assert np.linalg.norm(un - ref.u) <= 1e-7 * np.linalg.norm(ref.u), fp64
        s.close()
