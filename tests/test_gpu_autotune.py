"""The SpMV autotuner (xdcg_options.autotune): set-up times every compiled
pipeline shape of the product on the context's own matrix and keeps the
fastest.  The tuned context must still meet the solve parity bars against
the oracle (iterations within +-2 at 1e-8, u within 1e-7 at 1e-12), and the
product itself the SpMV parity bars."""
import numpy as np
import pytest

import xfem_inputs as X
from oracle import adef2 as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_autotuned_context_matches_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_09294_gb300 import Solver
    dev = torch.device("cuda:0")
    P = X.make("cube24_ellipse")
    K, M, C = O.setup(P)
    ref8 = O.adef2_pcg(K, P.f, M, C, tol=1e-8)
    ref12 = O.adef2_pcg(K, P.f, M, C, tol=1e-12)
    f = torch.tensor(P.f, device=dev)
    x = np.random.default_rng(13).standard_normal(P.n)
    for prec in ("fp64", "mixed"):
        s = Solver.from_problem(P, precision=prec, autotune=True)
        i = s.info
        t64 = [t for t in i["spmv_shape_us_fp64"] if t >= 0]
        assert len(t64) >= 2 and 0 <= i["spmv_shape_fp64"] < len(i["spmv_shape_us_fp64"])
        assert i["spmv_shape_us_fp64"][i["spmv_shape_fp64"]] == min(t64)
        if prec == "mixed":
            t32 = [t for t in i["spmv_shape_us_fp32"] if t >= 0]
            assert len(t32) >= 2 and i["spmv_shape_us_fp32"][i["spmv_shape_fp32"]] == min(t32)
        y, _ = s.spmv(torch.tensor(x, device=dev), "fp64")
        assert np.all(np.abs(y.cpu().numpy() - K @ x) <= 1e-12 * (abs(K) @ np.abs(x)))
        u, info = s.solve(f, tol=1e-8)
        if prec == "fp64":
            assert abs(info["iterations"] - ref8.iterations) <= 2
        assert info["rel_res_true"] <= 1.05e-8
        u, info = s.solve(f, tol=1e-12)
        assert np.linalg.norm(u.cpu().numpy() - ref12.u) <= 1e-7 * np.linalg.norm(ref12.u), prec
        s.close()
