"""Every pipeline shape of the FP32 SpMV, pinned one at a time
(xdcg_options.spmv_shape_fp32), gives the same product.

Each row's 3x3 block terms are added in the same order by every shape (the
shapes differ in how the matrix stream is staged: steps per bulk-copy stage,
stages per warp, blocks per SM, and for shapes 5-7 the lean kernel's copy
schedule), so y must be the same bits as shape 0's, whose product the SpMV
parity tests check against the oracle.  The fused dot x^T y is summed per
warp over the warp's rows and then over the grid: the same bits where the
shape's grid equals shape 0's, else within FP32 reordering (1e-5 relative
to sum |x_i y_i|).  A mixed solve with each lean shape also meets its
tolerance and matches the oracle."""
import numpy as np
import pytest

import xfem_inputs as X
from oracle import adef2 as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_SHAPES_FP32 = 8
LEAN = (5, 6, 7)


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("name", ["cube8_edge", "cube24_ellipse", "cube48_two_cracks"])
def test_every_fp32_shape_gives_the_same_product(name):
    dev = _cuda()
    from paper_2111_09294_gb300 import Solver
    P = X.make(name)
    rng = np.random.default_rng(7)
    x = torch.tensor(rng.standard_normal(P.n), dtype=torch.float32, device=dev)
    ref = Solver.from_problem(P, precision="mixed", spmv_shape=(0, -1))
    y0, d0 = ref.spmv(x, precision="mixed")
    scale = float(torch.sum(torch.abs(x.double() * y0.double())))
    ref.close()
    for sh in range(1, N_SHAPES_FP32):
        s = Solver.from_problem(P, precision="mixed", spmv_shape=(sh, -1))
        assert s.info["spmv_shape_fp32"] == sh
        y, d = s.spmv(x, precision="mixed")
        assert torch.equal(y, y0), (name, sh)
        assert abs(d - d0) <= 1e-5 * scale, (name, sh, d, d0)
        if sh == 5:
            # the lean kernel at shape 0's pipeline and grid: the dot too
            assert d == d0, (name, d, d0)
        s.close()


@pytest.mark.parametrize("sh", LEAN)
def test_mixed_solve_with_each_lean_shape_matches_oracle(sh):
    dev = _cuda()
    from paper_2111_09294_gb300 import Solver
    P = X.make("cube24_ellipse")
    f = torch.tensor(P.f, device=dev)
    K, M, C = O.setup(P)
    ref = O.adef2_pcg(K, P.f, M, C, tol=1e-12)
    s = Solver.from_problem(P, precision="mixed", spmv_shape=(sh, -1))
    u, info = s.solve(f, tol=1e-12)
    assert info["rel_res_true"] <= 1e-12
    err = np.linalg.norm(u.cpu().numpy() - ref.u) / np.linalg.norm(ref.u)
    assert err <= 1e-7, (sh, err)
    # shape 5 runs shape 0's pipeline and grid: the whole solve is the same bits
    if sh == 5:
        s0 = Solver.from_problem(P, precision="mixed", spmv_shape=(0, -1))
        u0, i0 = s0.solve(f, tol=1e-12)
        assert torch.equal(u, u0) and i0["iterations"] == info["iterations"]
        s0.close()
    s.close()


def test_out_of_range_shapes_are_rejected():
    _cuda()
    from paper_2111_09294_gb300 import Solver
    from paper_2111_09294_gb300._lib import XdcgError
    P = X.make("cube8_edge")
    for bad in ((N_SHAPES_FP32, -1), (-2, -1), (-1, 4)):
        with pytest.raises(XdcgError, match="INVALID_ARG"):
            Solver.from_problem(P, precision="mixed", spmv_shape=bad)
