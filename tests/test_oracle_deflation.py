"""Pins of the oracle's deflation basis Z (Section 3.3) against what the
mechanics and the geometry fix, with no GPU.

Every test calls the oracle's own deflation_basis / collinear /
stiffness_csr.  Each column of Z is checked in two independent ways:

* physically: a column must be a rigid motion t + w x (x - c) of its box
  (Eq. dcg_deflation_space), written here with cross products rather than
  the oracle's 3 x 6 block, or H(x) times one on the standard dofs and the
  plain one on the jump dofs (Eqs. dcg_deflation_space_enr_std,
  dcg_deflation_space_enr_enr), with H taken from the crack's own level set;
* mechanically: on an unconstrained body in one box, every rigid column lies
  in the null space of K, and on a body cut through by a crack so do the
  enriched columns (the two pieces move rigidly and independently).

A wrong rotation entry, a dropped H factor, an enriched column on the wrong
dofs, a missing box offset or a wrong enriched-box decision fails at least
one of them."""
import numpy as np
import pytest

import xfem_inputs as X
from oracle import adef2 as O
from xfem_inputs.cracks import PlanarEdgeCrack

AXES = np.eye(3)


def rigid_motion(mode, x):
    """Displacement at x (p, 3) of rigid mode `mode`: a unit translation
    along axis `mode` (0..2) or a unit rotation about axis `mode` - 3 (3..5)
    through the origin of x."""
    if mode < 3:
        return np.repeat(AXES[mode][None, :], x.shape[0], 0)
    return np.cross(AXES[mode - 3][None, :], x)


def enriched_boxes_by_rank(P):
    """Boxes whose jump-enriched nodes span a plane (affine rank >= 2): the
    boxes that carry enriched modes, decided by an SVD rank test."""
    out = np.zeros(P.n_sub, dtype=bool)
    kind = np.asarray(P.kind)
    sub = np.asarray(P.sub_of_node)
    for s in range(P.n_sub):
        pts = P.coords[(sub == s) & (kind == X.KIND_HEAVISIDE)]
        if pts.shape[0] >= 3:
            sv = np.linalg.svd(pts - pts.mean(0), compute_uv=False)
            out[s] = sv[1] > 1e-6 * sv[0]
    return out


def expected_basis(P, hside, enriched=True):
    """Dense Z built column by column from rigid motions (cross products),
    H(x_I) = hside(x_I) in {+1, -1}, box order and 6 or 12 columns a box."""
    enr = enriched_boxes_by_rank(P) if enriched else np.zeros(P.n_sub, bool)
    m = np.where(enr, 12, 6)
    col0 = np.concatenate([[0], np.cumsum(m)])
    dof = np.asarray(P.dof_ptr)
    kind = np.asarray(P.kind)
    sub = np.asarray(P.sub_of_node)
    Z = np.zeros((P.n, col0[-1]))
    for s in range(P.n_sub):
        nodes = np.nonzero(sub == s)[0]
        xr = P.coords[nodes] - np.asarray(P.centres)[s]
        H = hside(P.coords[nodes])
        for mode in range(6):
            u = rigid_motion(mode, xr)
            for a in range(3):
                Z[dof[nodes] + a, col0[s] + mode] = u[:, a]
                if enr[s]:
                    Z[dof[nodes] + a, col0[s] + 6 + mode] = H * u[:, a]
                    jn = kind[nodes] == X.KIND_HEAVISIDE
                    Z[dof[nodes[jn]] + 3 + a, col0[s] + 6 + mode] = u[jn, a]
    return Z, col0


def plane_side(z0):
    return lambda x: np.where(x[:, 2] - z0 >= 0.0, 1.0, -1.0)


@pytest.mark.parametrize("case", ["cube8_edge", "offplane"])
def test_every_column_matches_rigid_motions_entry_by_entry(case):
    if case == "cube8_edge":
        P, z0 = X.make("cube8_edge"), 0.5
    else:
        # crack plane between node layers, 3^3 boxes, both kinds of enrichment
        P, z0 = X.build_problem(9, [PlanarEdgeCrack(0.53, 0.6, 0.12)], 3), 0.53
    assert P.n_heaviside_dofs > 0 and P.n_tip_dofs > 0
    Z, col0 = O.deflation_basis(P)
    Zx, col0x = expected_basis(P, plane_side(z0))
    assert np.array_equal(col0, col0x)
    assert (np.diff(col0) == 12).sum() >= 1 and (np.diff(col0) == 6).sum() >= 1
    # exact: both sides form each entry from the same coordinates with at
    # most one product
    assert np.array_equal(Z.toarray(), Zx)
    # the rigid-only basis is the same without the enriched columns
    Zr, c0r = O.deflation_basis(P, enriched=False)
    Zrx, _ = expected_basis(P, plane_side(z0), enriched=False)
    assert np.array_equal(Zr.toarray(), Zrx) and np.array_equal(c0r, 6 * np.arange(P.n_sub + 1))


def test_cube8_coarse_dimension_matches_hand_derivation():
    # golden: 8 boxes x 6 rigid modes + 2 boxes with jump nodes x 6
    g = {}
    with open(__file__.replace("test_oracle_deflation.py", "golden/cube8_edge_counts.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                g[k] = int(v)
    P = X.make("cube8_edge")
    Z, col0 = O.deflation_basis(P)
    assert Z.shape == (g["n"], g["coarse_k"]) and col0[-1] == g["coarse_k"]


def test_rigid_columns_lie_in_null_space_of_free_cracked_body():
    # one box over an unconstrained cracked cube (jump and tip dofs present):
    # the six rigid columns move the whole body rigidly
    P = X.build_problem(6, [PlanarEdgeCrack(0.5, 0.45, 0.2)], 1, bc="none")
    assert P.n_heaviside_dofs > 0 and P.n_tip_dofs > 0
    K = O.stiffness_csr(P)
    Z, col0 = O.deflation_basis(P, enriched=False)
    assert Z.shape[1] == 6
    Zd = Z.toarray()
    assert np.linalg.norm((K @ Zd)) <= 1e-12 * np.linalg.norm(K.toarray()) * np.linalg.norm(Zd)
    assert np.linalg.matrix_rank(Zd) == 6


def test_enriched_columns_lie_in_null_space_of_body_cut_through():
    # a crack through the whole cube (off the node layers): two free pieces,
    # 12 zero-energy modes; the oracle's 12 columns of the single box span
    # exactly that null space
    P = X.build_problem(4, [PlanarEdgeCrack(0.47, 5.0, 0.0)], 1, bc="none")
    assert P.n_tip_dofs == 0 and P.n_heaviside_dofs > 0
    K = O.stiffness_csr(P).toarray()
    Z, col0 = O.deflation_basis(P)
    assert Z.shape[1] == 12
    Zd = Z.toarray()
    assert np.linalg.norm(K @ Zd) <= 1e-12 * np.linalg.norm(K) * np.linalg.norm(Zd)
    assert np.linalg.matrix_rank(Zd) == 12
    w, V = np.linalg.eigh(K)
    null = V[:, w < 1e-10 * w[-1]]
    assert null.shape[1] == 12
    # Z spans the null space: projecting Z onto it loses nothing
    assert np.linalg.norm(Zd - null @ (null.T @ Zd)) <= 1e-9 * np.linalg.norm(Zd)


def test_enriched_columns_fail_without_the_heaviside_factor():
    # the null-space pin above is sharp: the same columns with H dropped on
    # the standard dofs are far from the null space
    P = X.build_problem(4, [PlanarEdgeCrack(0.47, 5.0, 0.0)], 1, bc="none")
    K = O.stiffness_csr(P).toarray()
    Zd = O.deflation_basis(P)[0].toarray()
    bad = Zd.copy()
    dof = np.asarray(P.dof_ptr)
    for a in range(3):
        bad[dof[:-1] + a, 6:] = Zd[dof[:-1] + a, :6]
    assert np.linalg.norm(K @ bad[:, 6:]) > 1e-3 * np.linalg.norm(K) * np.linalg.norm(bad[:, 6:])


def test_collinear_decides_lines_and_planes():
    rng = np.random.default_rng(4)
    d = rng.standard_normal(3)
    line = np.array([0.1, 0.2, 0.3]) + np.outer(rng.uniform(-1, 1, 7), d)
    assert O.collinear(line)
    assert O.collinear(line[:2])                   # fewer than 3 points
    assert O.collinear(np.zeros((0, 3)))
    assert O.collinear(np.array([[0.0, 0.0, 0.5], [0.125, 0.0, 0.5], [0.25, 0.0, 0.5]]))
    tri = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    assert not O.collinear(tri)
    bent = line.copy()
    bent[3] += 1e-3 * np.cross(d, [1.0, 0.0, 0.0])
    assert not O.collinear(bent)
    assert not O.collinear(rng.standard_normal((5, 3)))


@pytest.mark.parametrize("case", ["cube8_edge", "small"])
def test_stiffness_csr_reproduces_block_storage_exactly(case):
    P = X.make("cube8_edge") if case == "cube8_edge" else \
        X.build_problem(3, [PlanarEdgeCrack(0.5, 0.45, 0.2)], 1)
    A = O.stiffness_csr(P).toarray()
    assert np.array_equal(A, X.to_dense(P))
