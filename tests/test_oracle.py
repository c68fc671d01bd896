"""Pins of the FP64 oracle (no GPU) against what the mathematics fixes:
dense Cholesky solves, the A-DEF2 invariant Z^T r_k = 0, monotone energy
error, reductions to textbook CG, finite termination with exact eigenvector
deflation, one-iteration convergence with the exact preconditioner, and the
equivalence of A-DEF2 (started by Algorithm 2) with Nicolaides' deflated CG
(Section 3.2).  A dropped term, a sign flip in lambda - mu, a transposed
triangular solve or a wrong coarse column would break at least one of them."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import xfem_inputs as X
from oracle import adef2 as O
from xfem_inputs.cracks import PlanarEdgeCrack, WarpedPennyCrack


@pytest.fixture(scope="module")
def cube8():
    P = X.make("cube8_edge")
    K, M, C = O.setup(P)
    return P, K, M, C


def small_problems():
    return [X.build_problem(3, [PlanarEdgeCrack(0.5, 0.45, 0.2)], 1),
            X.build_problem(4, [PlanarEdgeCrack(0.43, 0.6, 0.15)], 2),
            X.build_problem(4, [WarpedPennyCrack((0.5, 0.5, 0.55), 0.3, 0.02, 0.1)], 2)]


@pytest.mark.parametrize("idx", [0, 1, 2])
def test_converges_to_dense_cholesky_solution(idx):
    P = small_problems()[idx]
    K, M, C = O.setup(P)
    res = O.adef2_pcg(K, P.f, M, C, tol=1e-14)
    Kd = K.toarray()
    u = sla.cho_solve(sla.cho_factor(Kd), P.f)
    std = np.zeros(P.n, bool)
    for I in range(P.n_nodes):
        std[P.dof_ptr[I]:P.dof_ptr[I] + 3] = True
    assert res.converged
    assert np.linalg.norm(res.u - u) <= 1e-9 * np.linalg.norm(u)
    assert np.linalg.norm((res.u - u)[std]) <= 1e-11 * np.linalg.norm(u[std])


def test_deflated_residuals_are_orthogonal_to_Z(cube8):
    P, K, M, C = cube8
    res = O.adef2_pcg(K, P.f, M, C, tol=1e-10, record=True)
    zn = sp.linalg.norm(C.Z)
    assert max(res.ztr) <= 1e-10 * zn * np.linalg.norm(P.f)


def test_energy_error_decreases_monotonically(cube8):
    P, K, M, C = cube8
    Kd = K.toarray()
    u_star = sla.cho_solve(sla.cho_factor(Kd), P.f)
    res = O.adef2_pcg(K, P.f, M, C, tol=1e-9, max_iterates=200)
    errs = [np.sqrt((u_star - u) @ (Kd @ (u_star - u))) for u in res.iterates]
    assert len(errs) > 20
    assert all(b <= a * (1 + 1e-9) for a, b in zip(errs, errs[1:]))


def _textbook_cg(A, b, tol, maxit):
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = r @ r
    xs = []
    for _ in range(maxit):
        Ap = A @ p
        a = rr / (p @ Ap)
        x = x + a * p
        r = r - a * Ap
        xs.append(x.copy())
        if np.linalg.norm(r) <= tol * np.linalg.norm(b):
            break
        rr2 = r @ r
        p = r + rr2 / rr * p
        rr = rr2
    return xs


def test_no_deflation_identity_preconditioner_is_textbook_cg():
    P = X.build_problem(5, [], 1)                # uncracked: plain CG converges
    K = O.stiffness_csr(P)
    C0 = O.Coarse(K, sp.csc_matrix((P.n, 0)))
    res = O.adef2_pcg(K, P.f, O.Identity(), C0, tol=1e-10, max_iterates=5000)
    ref = _textbook_cg(K, P.f, 1e-10, 5000)
    assert res.converged
    assert res.iterations == len(ref)
    for a, b in zip(res.iterates[1:], ref):
        assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(b)


def test_exact_preconditioner_converges_in_one_iteration(cube8):
    P, K, _, C = cube8
    M1 = O.BlockJacobi(K, [0, P.n])              # one block holding all of K
    res = O.adef2_pcg(K, P.f, M1, C, tol=1e-8)
    assert res.iterations <= 1


def test_eigenvector_deflation_terminates_finitely():
    P = small_problems()[1]
    K, _, _ = O.setup(P)
    w, V = np.linalg.eigh(K.toarray())
    keep = 3                                    # leave the 3 largest eigenvalues
    Z = sp.csc_matrix(V[:, :-keep])
    C = O.Coarse(K, Z)
    res = O.adef2_pcg(K, P.f, O.Identity(), C, tol=1e-10)
    assert res.iterations <= keep


def test_adef2_matches_nicolaides_deflated_cg(cube8):
    P, K, M, C = cube8
    a = O.adef2_pcg(K, P.f, M, C, tol=1e-8, max_iterates=12)
    _, _, b = O.nicolaides_dcg(K, P.f, M, C, tol=1e-8, max_iterates=12)
    for ua, ub in zip(a.iterates, b):
        assert np.linalg.norm(ua - ub) <= 1e-9 * np.linalg.norm(ub)


def test_global_and_centred_rigid_coordinates_give_same_iterates():
    P = X.build_problem(8, [PlanarEdgeCrack(0.5, 0.45, 0.15)], 2)
    Pg = X.build_problem(8, [PlanarEdgeCrack(0.5, 0.45, 0.15)], 2, centred_modes=False)
    a = O.solve(P, tol=1e-8)
    b = O.solve(Pg, tol=1e-8)
    assert abs(a.iterations - b.iterations) <= 1
    assert np.linalg.norm(a.u - b.u) <= 1e-7 * np.linalg.norm(b.u)


def test_paper_trends_on_cube8(cube8):
    P, K, M, C = cube8
    bj_enr = O.adef2_pcg(K, P.f, M, C).iterations
    K0, M0, C0 = O.setup(P, enriched_modes=False)
    bj_std = O.adef2_pcg(K0, P.f, M0, C0).iterations
    Mj = O.BlockJacobi(K, np.arange(P.n + 1))  # point Jacobi: blocks of one dof
    j_enr = O.adef2_pcg(K, P.f, Mj, C).iterations
    assert bj_enr <= bj_std                     # enriched deflation never hurts
    assert bj_enr < j_enr                       # block Jacobi beats point Jacobi


def test_indefinite_block_is_rejected():
    P = X.make("cube8_edge")
    K = O.stiffness_csr(P).tolil()
    d = int(P.dof_ptr[5])
    K[d, d] = -1.0
    with pytest.raises(O.NotSPD) as ei:
        O.BlockJacobi(K.tocsr(), P.dof_ptr)
    assert ei.value.args[0] == 5


def test_algorithm2_with_nonzero_start(cube8):
    # Algorithm 2 with any u_-1 makes Z^T r_0 vanish (the start lies in the
    # deflated affine space), and the run from it reaches the same solution
    P, K, M, C = cube8
    rng = np.random.default_rng(21)
    u_m1 = rng.standard_normal(P.n) * np.linalg.norm(P.f) / np.sqrt(P.n)
    u0 = O.adef2_initial(K, C, P.f, u_m1)
    r0 = P.f - K @ u0
    zn = sp.linalg.norm(C.Z)
    assert np.linalg.norm(C.Z.T @ r0) <= 1e-10 * zn * np.linalg.norm(P.f)
    cold = O.adef2_pcg(K, P.f, M, C, tol=1e-12)
    warm = O.adef2_pcg(K, P.f, M, C, tol=1e-12, u_m1=u_m1)
    assert np.linalg.norm(warm.u - cold.u) <= 1e-8 * np.linalg.norm(cold.u)
    # a start that already meets the tolerance is returned after Algorithm 2
    # with no iteration
    again = O.adef2_pcg(K, P.f, M, C, tol=1e-8, u_m1=cold.u)
    assert again.iterations == 0
    assert np.linalg.norm(again.u - cold.u) <= 1e-12 * np.linalg.norm(cold.u)


def test_element_sensitivity_matches_central_differences():
    # J = w.u, u = K(E)^-1 f.  The oracle's -lam_e^T Khat_e u_e against
    # differences of J over systems rebuilt with E_e +- delta, for the element
    # of largest sensitivity among standard, jump- and tip-enriched elements;
    # and sum_e E_e dJ/dE_e = -lam^T K u = -w^T u (K is linear in E).
    from xfem_inputs.configs import CONFIGS
    cfg = CONFIGS["cube8_edge"]
    P = X.make("cube8_edge")
    D = X.element_data(P)
    K = X.to_dense(P)
    w = np.random.default_rng(51).standard_normal(P.n)
    u = np.linalg.solve(K, P.f)
    lam = np.linalg.solve(K, w)
    g = O.element_sensitivity(D, u, lam)
    J = w @ u
    assert abs(D["young"] @ g + J) <= 1e-10 * (np.abs(D["young"]) @ np.abs(g))
    en = np.asarray(P.elem_nodes_free)
    kind = np.where(en >= 0, np.asarray(P.kind)[np.maximum(en, 0)], X.KIND_STD)
    groups = {"std": ~(kind > 0).any(1), "jump": (kind == X.KIND_HEAVISIDE).any(1),
              "tip": (kind == X.KIND_TIP).any(1)}
    for name, sel in groups.items():
        cand = np.nonzero(sel)[0]
        e = int(cand[np.argmax(np.abs(g[cand]))])
        delta = 1e-4 * D["young"][e]
        Ks = []
        for s in (1.0, -1.0):
            y = D["young"].copy()
            y[e] += s * delta
            Ks.append(X.to_dense(X.build_problem(cfg["m"], cfg["cracks"](), cfg["n_box"],
                                                 young=y)))
        # J(E + delta) - J(E - delta) = -w^T K+^-1 (K+ - K-) K-^-1 f exactly; the
        # product form keeps K's conditioning (~1e9) out of the difference
        u_m = np.linalg.solve(Ks[1], P.f)
        fd = -(w @ np.linalg.solve(Ks[0], (Ks[0] - Ks[1]) @ u_m)) / (2 * delta)
        assert abs(fd - g[e]) <= 1e-5 * abs(g[e]), (name, e, fd, g[e])


def test_compliance_gradient_matches_differences_on_20_elements():
    # the differentiable-solve objective (compliance J = f^T u, so lam = u)
    # with log-normal element moduli, at the oracle's size: 20 seeded
    # elements against exact product-form differences of J over
    # K +- delta dK/dE_e (the element data themselves are pinned by their
    # reassembly of K in test_inputs)
    from xfem_inputs.configs import CONFIGS
    cfg = CONFIGS["cube8_edge"]
    young = np.random.default_rng(1).lognormal(0.0, 0.3, cfg["m"] ** 3)
    P = X.build_problem(cfg["m"], cfg["cracks"](), cfg["n_box"], young=young)
    D = X.element_data(P)
    K = X.to_dense(P)
    u = np.linalg.solve(K, P.f)
    g = O.element_sensitivity(D, u, u)
    assert np.all(g <= 1e-12 * np.max(np.abs(g)))     # -u_e^T Khat_e u_e, Khat_e PSD
    assert abs(young @ g + P.f @ u) <= 1e-10 * (np.abs(young) @ np.abs(g))
    for e in np.random.default_rng(2).choice(len(young), 20, replace=False):
        d = D["dofs"][D["dof_ptr"][e]:D["dof_ptr"][e + 1]]
        de = d.size
        Kh = D["mats"][D["mat_off"][e]:D["mat_off"][e] + de * de].reshape(de, de)
        live = d >= 0
        dK = np.zeros_like(K)
        dK[np.ix_(d[live], d[live])] = Kh[np.ix_(live, live)]
        delta = 1e-4 * young[e]
        u_m = np.linalg.solve(K - delta * dK, P.f)
        fd = -(P.f @ np.linalg.solve(K + delta * dK, (2 * delta * dK) @ u_m)) / (2 * delta)
        assert abs(fd - g[e]) <= 1e-5 * abs(g[e]) + 1e-12 * np.max(np.abs(g)), (e, fd, g[e])


def test_subdomain_blocks_reduce_to_node_blocks_and_cut_iterations():
    # one group per node gives the node-block M^-1 exactly; one group per box
    # (the paper's block choice) needs fewer iterations than node blocks with
    # the same deflation space (Section 4.1: larger blocks, fewer iterations)
    P = X.make("cube24_ellipse")
    K, M, C = O.setup(P)
    dof = np.asarray(P.dof_ptr, dtype=np.int64)
    nodes = O.SubdomainJacobi(K, [np.arange(dof[I], dof[I + 1]) for I in range(P.n_nodes)])
    r = np.random.default_rng(91).standard_normal(P.n)
    a, b = nodes.apply(r), M.apply(r)
    # two factorisation routes of the same blocks: rounding times the blocks'
    # condition numbers (up to ~7e8 here)
    assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(b)
    boxes = O.SubdomainJacobi(K, O.subdomain_dofs(P))
    assert sorted(np.concatenate(boxes.groups).tolist()) == list(range(P.n))
    node_run = O.adef2_pcg(K, P.f, M, C, tol=1e-8)
    box_run = O.adef2_pcg(K, P.f, boxes, C, tol=1e-8)
    assert np.linalg.norm(P.f - K @ box_run.u) <= 1.01e-8 * np.linalg.norm(P.f)
    assert box_run.iterations < node_run.iterations, (box_run.iterations, node_run.iterations)
