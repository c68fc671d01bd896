"""GPU checks of the differentiable solve beyond a single step.

* dJ/dK = -lam u^T sampled on K's pattern (xdcg_stiffness_gradient): every
  stored entry equals the product the oracle side forms (both are one FP64
  product, so bit for bit), and its contraction with K matches the element
  kernel's sum_e E_e dJ/dE_e (K = sum_e E_e Khat_e).
* dJ/dE_e against central differences through the GPU solver itself at
  24^3 with log-normal moduli: for 20 seeded elements, contexts are rebuilt
  with E_e +- delta and J(E + delta) - J(E - delta) is formed in product form,
  -u_+^T (K_+ - K_-) u_- (so K's conditioning does not enter the difference).
* the total compliance over four crack-front positions with u recomputed in
  the backward instead of stored, against the oracle's dense solves."""
import numpy as np
import pytest

import xfem_inputs as X
from oracle import adef2 as O
from xfem_inputs.cracks import PlanarEdgeCrack

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def element_value_positions(P, D, e):
    """Positions in P.val of element e's local dof pairs (live dofs only):
    (local rows, local cols, value indices)."""
    d = D["dofs"][D["dof_ptr"][e]:D["dof_ptr"][e + 1]].astype(np.int64)
    live = np.nonzero(d >= 0)[0]
    dof = np.asarray(P.dof_ptr, dtype=np.int64)
    rowp, col = np.asarray(P.row_ptr), np.asarray(P.col)
    node = np.searchsorted(dof, d[live], side="right") - 1
    rows, cols, idx = [], [], []
    for a, I in zip(live, node):
        for b, J in zip(live, node):
            p = rowp[I] + int(np.searchsorted(col[rowp[I]:rowp[I + 1]], J))
            bJ = dof[J + 1] - dof[J]
            rows.append(a)
            cols.append(b)
            idx.append(P.val_ptr[p] + (d[a] - dof[I]) * bJ + (d[b] - dof[J]))
    return np.array(rows), np.array(cols), np.array(idx)


def test_stiffness_gradient_is_the_sampled_outer_product():
    from paper_2111_09294_gb300 import Elements, Pattern, Solver
    dev = _cuda()
    P = X.make("cube8_edge")
    rng = np.random.default_rng(41)
    u, lam = rng.standard_normal(P.n), rng.standard_normal(P.n)
    s = Solver.from_problem(P)
    G = s.stiffness_gradient(Pattern.from_problem(P, dev), torch.tensor(lam, device=dev),
                             torch.tensor(u, device=dev)).cpu().numpy()
    dof = np.asarray(P.dof_ptr, dtype=np.int64)
    ref = np.empty(P.val.size)
    for I in range(P.n_nodes):
        for p in range(P.row_ptr[I], P.row_ptr[I + 1]):
            J = P.col[p]
            blk = -np.outer(lam[dof[I]:dof[I + 1]], u[dof[J]:dof[J + 1]])
            ref[P.val_ptr[p]:P.val_ptr[p + 1]] = blk.ravel()
    assert np.array_equal(G, ref)
    # <dJ/dK, K> = -lam^T K u, and the element kernel's contraction with the
    # moduli gives the same number
    D = X.element_data(P)
    g = s.element_sensitivity(Elements.from_dict(D, dev), torch.tensor(u, device=dev),
                              torch.tensor(lam, device=dev)).cpu().numpy()
    K = O.stiffness_csr(P)
    a, b, c = G @ P.val, -(lam @ (K @ u)), D["young"] @ g
    scale = np.abs(G) @ np.abs(P.val)
    assert abs(a - b) <= 1e-12 * scale and abs(c - b) <= 1e-12 * scale
    s.close()


def test_modulus_gradient_matches_gpu_central_differences():
    from paper_2111_09294_gb300 import Elements, Solver
    dev = _cuda()
    cfg = X.CONFIGS["cube24_ellipse"]
    young = np.random.default_rng(3).lognormal(0.0, 0.3, cfg["m"] ** 3)
    P = X.build_problem(cfg["m"], cfg["cracks"](), cfg["n_box"], young=young)
    D = X.element_data(P)
    f = torch.tensor(P.f, device=dev)
    s = Solver.from_problem(P)
    u, _ = s.solve(f, tol=1e-12)
    g = s.element_sensitivity(Elements.from_dict(D, dev), u, u).cpu().numpy()   # J = f^T u
    s.close()
    rng = np.random.default_rng(7)
    enr = np.asarray(P.enr_elements)
    std = np.setdiff1d(np.arange(len(young)), enr)
    picks = np.concatenate([rng.choice(enr, 10, replace=False), rng.choice(std, 10, replace=False)])
    gmax = np.max(np.abs(g))
    val0 = P.val.copy()
    for e in picks:
        de = int(D["dof_ptr"][e + 1] - D["dof_ptr"][e])
        Kh = D["mats"][D["mat_off"][e]:D["mat_off"][e] + de * de].reshape(de, de)
        rows, cols, idx = element_value_positions(P, D, e)
        delta = 1e-3 * young[e]
        us = []
        for sign in (1.0, -1.0):
            P.val = val0.copy()
            np.add.at(P.val, idx, sign * delta * Kh[rows, cols])
            sp = Solver.from_problem(P)
            ui, info = sp.solve(f, tol=1e-12)
            assert info["rel_res_true"] <= 1.05e-12
            us.append(ui.cpu().numpy())
            sp.close()
        # J(E+d) - J(E-d) = f^T (u_+ - u_-) = -u_+^T (K_+ - K_-) u_-, K_+ - K_- = 2 d Khat_e
        d = D["dofs"][D["dof_ptr"][e]:D["dof_ptr"][e + 1]]
        live = d >= 0
        up = np.where(live, us[0][np.maximum(d, 0)], 0.0)
        um = np.where(live, us[1][np.maximum(d, 0)], 0.0)
        fd = -(up @ (Kh @ um))
        assert abs(fd - g[e]) <= 1e-5 * abs(g[e]) + 1e-9 * gmax, (e, fd, g[e])
    P.val = val0


def test_compliance_over_four_steps_recomputes_u():
    from paper_2111_09294_gb300 import Elements, Solver
    from paper_2111_09294_gb300.autograd import compliance_steps
    dev = _cuda()
    young = np.random.default_rng(5).lognormal(0.0, 0.3, 8 ** 3)
    Ps = [X.build_problem(8, [PlanarEdgeCrack(0.5, xf, 0.15)], 2, young=young)
          for xf in (0.40, 0.45, 0.52, 0.58)]
    Ds = [X.element_data(P) for P in Ps]
    for prec, tol, rtol in (("fp64", 1e-12, 1e-7), ("mixed", 1e-10, 1e-5)):
        solvers = [Solver.from_problem(P, precision=prec) for P in Ps]
        elems = [Elements.from_dict(D, dev) for D in Ds]
        fs = [torch.tensor(P.f, device=dev, requires_grad=True) for P in Ps]
        yg = torch.tensor(young, device=dev, requires_grad=True)
        saved = []

        def pack(t):
            saved.append(t)
            return t

        with torch.autograd.graph.saved_tensors_hooks(pack, lambda t: t):
            J = compliance_steps(solvers, fs, tol, young=yg, elements=elems)
        # nothing but the loads is kept for the backward (u is recomputed)
        assert len(saved) == len(fs)
        assert all(any(t.data_ptr() == f.data_ptr() for f in fs) for t in saved)
        J.backward()
        J_ref, g_ref = 0.0, np.zeros(len(young))
        for P, D, f in zip(Ps, Ds, fs):
            u = np.linalg.solve(X.to_dense(P), P.f)
            J_ref += P.f @ u
            g_ref += O.element_sensitivity(D, u, u)
            assert np.linalg.norm(f.grad.cpu().numpy() - 2 * u) <= rtol * np.linalg.norm(2 * u)
        assert abs(float(J) - J_ref) <= rtol * abs(J_ref)
        assert np.max(np.abs(yg.grad.cpu().numpy() - g_ref)) <= rtol * np.max(np.abs(g_ref)), prec
        for s in solvers:
            s.close()
