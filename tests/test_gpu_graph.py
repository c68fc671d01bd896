"""Iterations enqueued as recorded CUDA graphs (xdcg_options.graph).

A batch of iterations is recorded once by stream capture and replayed with
one graph launch per batch (single-RHS solves), or per tick of the batched
and multi-system solves, recorded again whenever the set of live systems
changes.  The graphs hold the same kernels, in the same order and with the
same programmatic ordering, as the launches of the uncaptured loop, so every
result must be the same bits; graph launches must actually have been made;
and the timing modes, whose events sit between the kernels, run without
graphs.  One graph solve per path is also checked against the oracle at
tol 1e-12 (||u - u_ref|| <= 1e-7 ||u_ref||, the solves' parity tolerance)."""
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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_solves_are_the_same_bits(prec):
    dev = _cuda()
    from paper_2111_09294_gb300 import Solver
    P = X.make("cube24_ellipse")
    f = torch.tensor(P.f, device=dev)
    plain = Solver.from_problem(P, precision=prec)
    graph = Solver.from_problem(P, precision=prec, graph=True)
    for tol in (1e-8, 1e-12):
        ua, ia = plain.solve(f, tol=tol)
        ub, ib = graph.solve(f, tol=tol)
        assert torch.equal(ua, ub), (prec, tol)
        assert ia["iterations"] == ib["iterations"] and ia["outer_cycles"] == ib["outer_cycles"]
        assert ia["n_graph_launches"] == 0 and ib["n_graph_launches"] > 0
        assert ia["n_launches"] == ib["n_launches"]
    # a warm start (the FP32 cycles start at other iteration parities)
    x0 = 0.5 * ua
    va, ja = plain.solve(f, tol=1e-10, x0=x0)
    vb, jb = graph.solve(f, tol=1e-10, x0=x0)
    assert torch.equal(va, vb) and ja["iterations"] == jb["iterations"]
    # the same context again: the recorded batches are replayed, not re-recorded
    uc, ic = graph.solve(f, tol=1e-12)
    assert torch.equal(uc, ub) and ic["n_graph_launches"] > 0
    # against the oracle
    K, M, C = O.setup(P)
    ref = O.adef2_pcg(K, P.f, M, C, tol=1e-12)
    err = np.linalg.norm(ub.cpu().numpy() - ref.u) / np.linalg.norm(ref.u)
    assert err <= 1e-7, (prec, err)
    plain.close()
    graph.close()


def test_graph_option_is_ignored_by_the_timing_modes():
    dev = _cuda()
    from paper_2111_09294_gb300 import Solver
    P = X.make("cube8_edge")
    f = torch.tensor(P.f, device=dev)
    a = Solver.from_problem(P, precision="mixed")
    b = Solver.from_problem(P, precision="mixed", graph=True, time_spmv="kernels")
    ua, ia = a.solve(f, tol=1e-10)
    ub, ib = b.solve(f, tol=1e-10)
    assert torch.equal(ua, ub) and ib["n_graph_launches"] == 0 and ib["n_phase_timed"] > 0
    a.close()
    b.close()


def test_graph_batched_and_multi_system_solves_are_the_same_bits():
    dev = _cuda()
    from paper_2111_09294_gb300 import sweep as S
    # three systems of different sizes (the small ones leave first, so the
    # fused tick is recorded again for each new set of live systems)
    Ps = [X.make(n) for n in ("cube8_edge", "trend12", "cube24_ellipse")]
    ms = (3, 2, 4)
    loads = [torch.tensor(X.load_cases(P, m, seed=21 + i), device=dev)
             for i, (P, m) in enumerate(zip(Ps, ms))]
    plain = S.make_solvers(Ps, max_batch=4)
    graph = S.make_solvers(Ps, max_batch=4, graph=True)
    for fused in (False, True):
        ra = S.solve_systems(plain, loads, 1e-11, fused=fused)
        rb = S.solve_systems(graph, loads, 1e-11, fused=fused)
        for (Ua, ia), (Ub, ib) in zip(ra, rb):
            assert torch.equal(Ua, Ub), fused
            assert [i["iterations"] for i in ia] == [i["iterations"] for i in ib]
            assert all(i["n_graph_launches"] == 0 for i in ia)
            assert all(i["n_graph_launches"] > 0 for i in ib)
            assert all(i["rel_res_true"] <= 1e-11 for i in ib)
    # one system's column against the oracle
    P = Ps[2]
    K, M, C = O.setup(P)
    F = loads[2].cpu().numpy()
    ref = O.adef2_pcg(K, F[1], M, C, tol=1e-11)
    err = np.linalg.norm(rb[2][0][1].cpu().numpy() - ref.u) / np.linalg.norm(ref.u)
    assert err <= 1e-6, err
    for s in plain + graph:
        s.close()
