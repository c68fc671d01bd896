"""Systems of a propagation sweep solved together: 32^3 hexes with an
inclined penny whose radius grows from 0.15 to 0.35 (three of the sixteen
crack-front positions here, of different sizes), four load cases each, every
system a batched mixed solve on its own context and stream, the systems'
calls issued concurrently.  Concurrent and one-after-another runs must agree
bit for bit, every column must meet its tolerance on the FP64 true residual,
and one system is checked against the oracle."""
import numpy as np
import pytest

import xfem_inputs as X
from oracle import adef2 as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_sweep_concurrent_matches_sequential_and_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    from paper_2111_09294_gb300 import sweep as S
    Ps = X.make_many([X.SWEEP[0], X.SWEEP[7], X.SWEEP[15]], workers=3)
    assert len({P.n for P in Ps}) == 3        # enriched dof counts differ along the sweep
    loads = [torch.tensor(X.load_cases(P, 4, seed=11 + i), device=dev) for i, P in enumerate(Ps)]
    solvers = S.make_solvers(Ps, max_batch=4)
    conc = S.solve_systems(solvers, loads, 1e-12)
    seq = S.solve_systems(solvers, loads, 1e-12, concurrent=False)
    for (Uc, ic), (Us, iq) in zip(conc, seq):
        assert torch.equal(Uc, Us)
        assert [i["iterations"] for i in ic] == [i["iterations"] for i in iq]
        assert all(i["rel_res_true"] <= 1e-12 for i in ic)
    P = Ps[2]
    K, M, C = O.setup(P)
    F = loads[2].cpu().numpy()
    for j in (0, 3):
        ref = O.adef2_pcg(K, F[j], M, C, tol=1e-12)
        err = np.linalg.norm(conc[2][0][j].cpu().numpy() - ref.u) / np.linalg.norm(ref.u)
        assert err <= 1e-7, (j, err)
    for s in solvers:
        s.close()
