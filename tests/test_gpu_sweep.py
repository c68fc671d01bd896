"""Systems of a propagation sweep solved together: 32^3 hexes with an
inclined penny whose radius grows from 0.15 to 0.35 (three of the sixteen
crack-front positions here, of different sizes), a few load cases each,
every system a batched mixed solve on its own context.  The fused run (one
launch per kernel over all systems), the concurrent run (one host thread and
stream per system) and the one-after-another run must agree bit for bit,
every column must meet its tolerance on the FP64 true residual, and one
system is checked against the oracle."""
import numpy as np
import pytest

import xfem_inputs as X
from oracle import adef2 as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_sweep_fused_concurrent_sequential_agree_and_match_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    from paper_2111_09294_gb300 import sweep as S
    Ps = X.make_many([X.SWEEP[0], X.SWEEP[7], X.SWEEP[15]], workers=3)
    assert len({P.n for P in Ps}) == 3        # enriched dof counts differ along the sweep
    # different column counts per system; system 1 has a zero load case
    ms = (4, 2, 3)
    loads = [torch.tensor(X.load_cases(P, m, seed=11 + i), device=dev)
             for i, (P, m) in enumerate(zip(Ps, ms))]
    loads[1][1].zero_()
    solvers = S.make_solvers(Ps, max_batch=4)
    fused = S.solve_systems(solvers, loads, 1e-12, fused=True)
    conc = S.solve_systems(solvers, loads, 1e-12)
    seq = S.solve_systems(solvers, loads, 1e-12, concurrent=False)
    for (Uf, jf), (Uc, ic), (Us, iq) in zip(fused, conc, seq):
        assert torch.equal(Uf, Uc) and torch.equal(Uc, Us)
        its = [i["iterations"] for i in jf]
        assert its == [i["iterations"] for i in ic] == [i["iterations"] for i in iq]
        assert [i["outer_cycles"] for i in jf] == [i["outer_cycles"] for i in iq]
        assert all(i["rel_res_true"] <= 1e-12 for i in jf)
        assert all(i["status"] == "XDCG_OK" for i in jf)
    assert torch.all(fused[1][0][1] == 0) and fused[1][1][1]["iterations"] == 0
    P = Ps[2]
    K, M, C = O.setup(P)
    F = loads[2].cpu().numpy()
    for j in (0, 2):
        ref = O.adef2_pcg(K, F[j], M, C, tol=1e-12)
        err = np.linalg.norm(fused[2][0][j].cpu().numpy() - ref.u) / np.linalg.norm(ref.u)
        assert err <= 1e-7, (j, err)
    # a context passed twice shares one set of scalars: refused
    from paper_2111_09294_gb300._lib import XdcgError
    with pytest.raises(XdcgError, match="INVALID_ARG"):
        S.solve_systems([solvers[0], solvers[0]], [loads[0], loads[0].clone()], 1e-8,
                        fused=True)
    for s in solvers:
        s.close()


def test_update_for_next_front_matches_fresh_setup():
    # the context for the next crack front built from the previous one
    # (xdcg_setup_update): the node factors the front left unchanged are
    # carried over, the rest factored; results bit for bit those of a fresh
    # set-up.  The same system again carries over every factor and E^-1.
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_09294_gb300 import Solver
    P0, P1 = X.make_many(X.SWEEP[:2])
    f1 = torch.tensor(P1.f, device="cuda:0")
    for prec in ("fp64", "mixed"):
        s0 = Solver.from_problem(P0, precision=prec)
        fresh = Solver.from_problem(P1, precision=prec)
        upd = Solver.from_problem(P1, precision=prec, prev=s0)
        assert 0 < upd.info["reused_node_factors"] < P1.n_nodes
        assert np.array_equal(upd.coarse_matrix(), fresh.coarse_matrix())
        ua, ia = fresh.solve(f1, tol=1e-8)
        ub, ib = upd.solve(f1, tol=1e-8)
        assert torch.equal(ua, ub) and ia["iterations"] == ib["iterations"], prec
        same = Solver.from_problem(P0, precision=prec, prev=s0)
        assert same.info["reused_node_factors"] == P0.n_nodes
        assert same.info["reused_coarse_inverse"] == 1
        f0 = torch.tensor(P0.f, device="cuda:0")
        assert torch.equal(same.solve(f0, tol=1e-8)[0], s0.solve(f0, tol=1e-8)[0])
        for s in (s0, fresh, upd, same):
            s.close()


def test_warm_start_from_previous_front():
    # the previous front's solution carried into the next system's numbering
    # (standard dofs, and enriched dofs of nodes that keep their enrichment)
    # as u_-1 of Algorithm 2: the same answer as a cold start, in no more
    # iterations
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_09294_gb300 import Solver
    from paper_2111_09294_gb300.sweep import transfer_guess, transfer_index
    P0, P1 = X.make_many(X.SWEEP[:2])
    dev = torch.device("cuda:0")
    s0 = Solver.from_problem(P0)
    u0, _ = s0.solve(torch.tensor(P0.f, device=dev), tol=1e-10)
    s1 = Solver.from_problem(P1, prev=s0)
    f1 = torch.tensor(P1.f, device=dev)
    cold, ic = s1.solve(f1, tol=1e-10)
    guess = transfer_guess(u0, transfer_index(P0.dof_ptr, P0.kind, P1.dof_ptr, P1.kind), P1.n)
    warm, iw = s1.solve(f1, tol=1e-10, x0=guess)
    assert iw["rel_res_true"] <= 1.05e-10
    assert float(torch.linalg.norm(warm - cold) / torch.linalg.norm(cold)) <= 1e-7
    assert iw["iterations"] <= ic["iterations"], (iw["iterations"], ic["iterations"])
    print(f"\nnext front, tol 1e-10: cold {ic['iterations']} iterations, warm {iw['iterations']}")
    s0.close()
    s1.close()
