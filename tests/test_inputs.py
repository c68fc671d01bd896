"""Pins of the synthetic XFEM inputs against facts the mechanics fixes
(no GPU).  Each test would fail for a plausible slip in the generator: a
wrong shape-function derivative, Hooke matrix, traction weight, enrichment
set, Heaviside shift, sub-tetrahedral split or branch-function gradient."""
import os

import numpy as np
import pytest

import xfem_inputs as X
from xfem_inputs.assemble import _standard_element_matrix, lame
from xfem_inputs.cracks import PlanarEdgeCrack
from xfem_inputs.enrichment import branch_functions, polar
from xfem_inputs.quadrature import HEX_TETS, map_tet, split_tet, tet_rule

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                out[k] = int(v)
    return out


def test_cube8_edge_counts_match_hand_derivation():
    g = read_golden("cube8_edge_counts.txt")
    P = X.make("cube8_edge")
    assert P.n_nodes == g["free_nodes"]
    assert 3 * P.n_nodes == g["standard_dofs"]
    assert P.n_heaviside_dofs == g["heaviside_dofs"]
    assert P.n_tip_dofs == g["tip_dofs"]
    assert P.n == g["n"]
    # the coarse dimension of the hand derivation, from the oracle's own basis
    from oracle import adef2 as O
    Z, col0 = O.deflation_basis(P)
    assert Z.shape[1] == col0[-1] == g["coarse_k"]


def test_tet_rule_exact_for_degree_5():
    # monomials x^a y^b z^c on the reference tet integrate to a! b! c! / (a+b+c+3)!
    from math import factorial
    xi, w = tet_rule(3)
    for a, b, c in [(0, 0, 0), (2, 1, 0), (1, 1, 1), (4, 0, 1), (0, 3, 2), (2, 2, 1)]:
        exact = factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 3)
        got = np.sum(w * xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c)
        assert abs(got - exact) < 1e-15


def test_hex_tets_and_splits_tile_volume():
    rng = np.random.default_rng(0)
    cube = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                     [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], float)
    total = sum(np.sum(map_tet(cube[t], 2)[1]) for t in HEX_TETS)
    assert abs(total - 1.0) < 1e-14
    for _ in range(50):
        g = rng.normal(size=3)
        s0 = rng.normal() * 0.3
        for t in HEX_TETS:
            v = cube[t]
            s = s0 + v @ g
            s[rng.random(4) < 0.15] = 0.0           # exercise vertices on the cut
            pieces = split_tet(v, s)
            vol = abs(np.linalg.det(v[1:] - v[0])) / 6
            assert abs(sum(abs(np.linalg.det(p[1:] - p[0])) / 6 for p, _ in pieces) - vol) < 1e-13
            for p, side in pieces:                  # each piece lies on one side
                vals = (p - v[0]) @ np.linalg.solve(v[1:] - v[0], s[1:] - s[0]) + s[0]
                assert np.all(side * vals >= -1e-12)


def test_standard_element_has_six_rigid_modes():
    lam, mu = lame(1.0, 0.3)
    Ke = _standard_element_matrix(0.25, lam, mu)
    ev = np.linalg.eigvalsh(Ke)
    assert np.all(np.abs(ev[:6]) < 1e-12 * ev[-1])
    assert ev[6] > 1e-3 * ev[-1]


def test_uniaxial_patch_test_exact():
    # roller supports, unit tension on z = 1: u = (-nu x, -nu y, z) / E exactly
    E, nu = 2.0, 0.3
    P = X.build_problem(3, [], 1, E=E, nu=nu, bc="roller")
    K = X.to_dense(P)
    u = np.linalg.solve(K, P.f)
    x = P.coords
    expect = np.stack([-nu * x[:, 0] / E, -nu * x[:, 1] / E, x[:, 2] / E], 1).ravel()
    assert np.max(np.abs(u - expect)) < 1e-12


def _rigid(x):
    X_, Y, Z = x
    return np.array([[1, 0, 0, 0, Z, -Y], [0, 1, 0, -Z, 0, X_], [0, 0, 1, Y, -X_, 0]], float)


def test_rigid_modes_in_nullspace_of_unconstrained_cracked_K():
    P = X.build_problem(6, [PlanarEdgeCrack(0.5, 0.45, 0.2)], 2, bc="none")
    assert P.n_tip_dofs > 0 and P.n_heaviside_dofs > 0
    K = X.to_dense(P)
    Zr = np.zeros((P.n, 6))
    for I in range(P.n_nodes):
        Zr[P.dof_ptr[I]:P.dof_ptr[I] + 3] = _rigid(P.coords[I])
    assert np.linalg.norm(K @ Zr) <= 1e-12 * np.linalg.norm(K) * np.linalg.norm(Zr)


def test_through_crack_has_twelve_zero_energy_modes():
    # a crack cutting the whole cube (psi < 0 everywhere, off the node layers)
    # leaves two free pieces: 6 + 6 rigid modes; the extra 6 are exactly the
    # field H(x) (rigid motion), nodal values H(x_I) R(x_I) on standard dofs
    # and R(x_I) on jump dofs.
    P = X.build_problem(4, [PlanarEdgeCrack(0.47, 5.0, 0.0)], 1, bc="none")
    assert P.n_tip_dofs == 0 and P.n_heaviside_dofs == 3 * 2 * 25
    K = X.to_dense(P)
    ev = np.linalg.eigvalsh(K)
    assert np.sum(ev < 1e-10 * ev[-1]) == 12
    assert ev[12] > 1e-6 * ev[-1]
    Ze = np.zeros((P.n, 6))
    for I in range(P.n_nodes):
        d0 = P.dof_ptr[I]
        R = _rigid(P.coords[I])
        H = 1.0 if P.coords[I][2] - 0.47 >= 0 else -1.0
        Ze[d0:d0 + 3] = H * R
        if P.kind[I] == X.KIND_HEAVISIDE:
            Ze[d0 + 3:d0 + 6] = R
    assert np.linalg.norm(K @ Ze) <= 1e-12 * np.linalg.norm(K) * np.linalg.norm(Ze)


def test_branch_function_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    gphi = np.array([0.1, 0.2, 1.0])
    gpsi = np.array([1.0, -0.1, 0.0])
    x = rng.uniform(-0.3, 0.3, size=(40, 3))

    def fields(x):
        phi, psi = x @ gphi, x @ gpsi
        r, th = polar(phi, psi)
        gr = (phi[:, None] * gphi + psi[:, None] * gpsi) / r[:, None]
        gth = (psi[:, None] * gphi - phi[:, None] * gpsi) / (r * r)[:, None]
        return r, th, gr, gth

    for th_i in [0.3, -2.0, np.pi, np.pi / 3, 1.7]:
        r, th, gr, gth = fields(x)
        F, dF = branch_functions(r, th, gr, gth, 0.05, th_i)
        eps = 1e-6
        for d in range(3):
            e = np.zeros(3)
            e[d] = eps
            rp, tp, grp, gtp = fields(x + e)
            rm, tm, grm, gtm = fields(x - e)
            ok = np.abs(tp - tm) < 1.0                 # stay off the crack-face branch cut
            Fp, _ = branch_functions(rp, tp, grp, gtp, 0.05, th_i)
            Fm, _ = branch_functions(rm, tm, grm, gtm, 0.05, th_i)
            fd = (Fp - Fm) / (2 * eps)
            assert np.max(np.abs(fd[:, ok] - dF[:, ok, d])) < 1e-6


def test_branch_functions_vanish_at_their_node():
    for th_i in [0.2, -1.0, np.pi, np.pi / 3, -np.pi / 3, 2.5]:
        r_i = 0.07
        F, _ = branch_functions(np.array([r_i]), np.array([th_i]), np.zeros((1, 3)),
                                np.zeros((1, 3)), r_i, th_i)
        assert np.max(np.abs(F)) < 1e-15


def test_stiffness_is_symmetric_and_definite():
    P = X.make("cube8_edge")
    K = X.to_dense(P)
    assert np.max(np.abs(K - K.T)) <= 1e-14 * np.max(np.abs(K))
    np.linalg.cholesky(K)


def test_load_cases_are_linear_in_the_traction():
    # the unit-tension case reproduces the workload's own load, and the loads
    # add up as the tractions do (consistent nodal forces are linear in t)
    P = X.make("cube8_edge")
    F = X.load_cases(P, 4, seed=3)
    t = X.tractions(4, seed=3)
    assert F.shape == (4, P.n)
    w = X.face_weights(P)
    assert np.isclose(w.sum(), 1.0)            # the loaded face has unit area
    for c in range(4):
        total = F[c].reshape(-1)
        dof = np.asarray(P.dof_ptr)
        for d in range(3):
            assert np.isclose(total[dof[:-1] + d].sum(), t[c, d])
    assert np.all((0.5 <= np.abs(t)) & (np.abs(t) <= 1.5)) and np.all(t[:, 2] > 0)


def test_element_data_reassembles_K():
    # K = sum_e E_e Khat_e scattered to each element's dofs (eliminated dofs
    # dropped), with per-element moduli: a wrong local dof order, a missing
    # enriched block or a matrix taken at the wrong modulus breaks it
    from xfem_inputs.configs import CONFIGS
    cfg = CONFIGS["cube8_edge"]
    young = np.random.default_rng(9).lognormal(0.0, 0.3, cfg["m"] ** 3)
    P = X.build_problem(cfg["m"], cfg["cracks"](), cfg["n_box"], young=young)
    D = X.element_data(P)
    K = X.to_dense(P)
    Ks = np.zeros_like(K)
    for e in range(len(D["mat_off"])):
        d = D["dofs"][D["dof_ptr"][e]:D["dof_ptr"][e + 1]]
        de = d.size
        Kh = D["mats"][D["mat_off"][e]:D["mat_off"][e] + de * de].reshape(de, de)
        live = d >= 0
        Ks[np.ix_(d[live], d[live])] += D["young"][e] * Kh[np.ix_(live, live)]
    assert np.max(np.abs(Ks - K)) <= 1e-14 * np.max(np.abs(K))
    assert np.all(D["young"] == young)


def test_subdomain_renumbering_moves_entries_only():
    # by_subdomain relabels nodes box by box: K, f and the element dof maps
    # are the same up to that permutation, and each box's dofs are one range
    P = X.make("cube8_edge")
    P2, bp = X.by_subdomain(P)
    d = P2.dof_map_from
    assert np.array_equal(np.sort(d), np.arange(P.n))
    assert np.array_equal(X.to_dense(P2)[np.ix_(d, d)], X.to_dense(P))
    assert np.array_equal(P2.f[d], P.f)
    sub2 = np.asarray(P2.sub_of_node)
    assert np.all(np.diff(sub2) >= 0)
    dof2 = np.asarray(P2.dof_ptr)
    for s in range(P.n_sub):
        nodes = np.nonzero(sub2 == s)[0]
        assert bp[s] == dof2[nodes[0]] and bp[s + 1] == dof2[nodes[-1] + 1]
    D1, D2 = X.element_data(P), X.element_data(P2)
    assert np.array_equal(np.where(D1["dofs"] >= 0, d[np.maximum(D1["dofs"], 0)], -1), D2["dofs"])
