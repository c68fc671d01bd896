"""GPU parity of the valued form of the deflation space (Section 3.3): Z
given to the boundary as per-node value blocks instead of geometry.

Two seeded cases, each against the oracle with the same Z:
* the oracle's own basis, passed by value: the same coarse matrix E (to
  1e-12) and the same solutions as the geometric form;
* that basis times a seeded invertible 6x6 / 12x12 matrix per box: a
  different Z with the same span, so A-DEF2 gives the same iterates in exact
  arithmetic (the coarse correction depends only on the span of Z), and the
  oracle run with the transformed Z gives the reference.
Tolerances as in the other solve parity tests."""
import numpy as np
import pytest
import scipy.sparse as sp

import xfem_inputs as X
from oracle import adef2 as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def to_values(P, Z, col0):
    """The boundary's valued layout of a deflation basis Z (n x k) whose
    box s owns columns col0[s] .. col0[s + 1]: per-box column counts and
    node blocks, row-major, nodes in order."""
    Zd = Z.toarray() if sp.issparse(Z) else np.asarray(Z)
    cols = np.diff(col0).astype(np.int32)
    dof = np.asarray(P.dof_ptr)
    sub = np.asarray(P.sub_of_node)
    vals = []
    for I in range(P.n_nodes):
        s = sub[I]
        vals.append(Zd[dof[I]:dof[I + 1], col0[s]:col0[s + 1]].ravel())
    return cols, np.concatenate(vals)


def mixed_basis(P, Z, col0, seed):
    """Z Q with Q block diagonal, one seeded well-conditioned block per box."""
    rng = np.random.default_rng(seed)
    blocks = []
    for s in range(P.n_sub):
        m = int(col0[s + 1] - col0[s])
        A = rng.standard_normal((m, m))
        blocks.append(np.eye(m) + 0.3 * A / np.linalg.norm(A, 2))
    return (Z @ sp.block_diag(blocks)).tocsc()


@pytest.mark.parametrize("name", ["cube8_edge", "cube24_ellipse"])
def test_valued_z_reproduces_geometric_form(name):
    from paper_2111_09294_gb300 import Solver
    dev = _cuda()
    P = X.make(name)
    K = O.stiffness_csr(P)
    Z, col0 = O.deflation_basis(P)
    C = O.Coarse(K, Z)
    M = O.BlockJacobi(K, P.dof_ptr)
    cols, vals = to_values(P, Z, col0)
    ref8 = O.adef2_pcg(K, P.f, M, C, tol=1e-8)
    ref12 = O.adef2_pcg(K, P.f, M, C, tol=1e-12)
    f = torch.tensor(P.f, device=dev)
    for prec in ("fp64", "mixed"):
        s = Solver.from_problem(P, precision=prec, z_cols=cols, z_values=vals)
        assert s.k == Z.shape[1]
        E = s.coarse_matrix()
        assert np.max(np.abs(E - C.E)) <= 1e-12 * np.max(np.abs(C.E))
        u, info = s.solve(f, tol=1e-8)
        if prec == "fp64":
            assert abs(info["iterations"] - ref8.iterations) <= 2
        assert info["rel_res_true"] <= 1.05e-8
        u, info = s.solve(f, tol=1e-12)
        assert np.linalg.norm(u.cpu().numpy() - ref12.u) <= 1e-7 * np.linalg.norm(ref12.u), prec
        s.close()


@pytest.mark.parametrize("name", ["cube8_edge", "cube24_ellipse"])
def test_valued_z_with_changed_basis_matches_oracle(name):
    from paper_2111_09294_gb300 import Solver
    dev = _cuda()
    P = X.make(name)
    K = O.stiffness_csr(P)
    Z0, col0 = O.deflation_basis(P)
    Z = mixed_basis(P, Z0, col0, seed=23)
    C = O.Coarse(K, Z)
    M = O.BlockJacobi(K, P.dof_ptr)
    cols, vals = to_values(P, Z, col0)
    ref8 = O.adef2_pcg(K, P.f, M, C, tol=1e-8)
    ref12 = O.adef2_pcg(K, P.f, M, C, tol=1e-12)
    f = torch.tensor(P.f, device=dev)
    s = Solver.from_problem(P, z_cols=cols, z_values=vals)
    E = s.coarse_matrix()
    assert np.max(np.abs(E - C.E)) <= 1e-12 * np.max(np.abs(C.E))
    r = np.random.default_rng(29).standard_normal(P.n)
    z_ref = O.adef2_apply(K, M, C, r)
    z = s.precond(torch.tensor(r, device=dev)).cpu().numpy()
    assert np.linalg.norm(z - z_ref) <= 1e-8 * np.linalg.norm(z_ref)
    u, info = s.solve(f, tol=1e-8)
    assert abs(info["iterations"] - ref8.iterations) <= 2
    u, info = s.solve(f, tol=1e-12)
    assert np.linalg.norm(u.cpu().numpy() - ref12.u) <= 1e-7 * np.linalg.norm(ref12.u)
    s.close()


def test_valued_z_rejects_bad_column_counts():
    from paper_2111_09294_gb300 import Solver, XdcgError
    _cuda()
    P = X.make("cube8_edge")
    Z, col0 = O.deflation_basis(P)
    cols, vals = to_values(P, Z, col0)
    bad = cols.copy()
    bad[0] = 7
    with pytest.raises(XdcgError) as ei:
        Solver.from_problem(P, z_cols=bad, z_values=vals)
    assert ei.value.status == 1
    nan = vals.copy()
    nan[5] = np.nan
    with pytest.raises(XdcgError) as ei:
        Solver.from_problem(P, z_cols=cols, z_values=nan)
    assert ei.value.status == 1
