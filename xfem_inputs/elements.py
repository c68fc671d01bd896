"""Per-element data for the sensitivity of a solve to each element's Young's
modulus: K = sum_e E_e Khat_e with Khat_e the element stiffness for E = 1
(nu fixed), so dK/dE_e = Khat_e scattered to the element's dofs.

element_data(P) returns the layout the library's element-sensitivity call
takes:

* dof_ptr [n_el + 1] (int64): element e's local dofs are dofs[dof_ptr[e]:dof_ptr[e+1]];
* dofs (int32): the global dof of each local dof, -1 where the dof is
  eliminated (clamped node, fixed dof);
* mat_off [n_el] (int64): element e's d_e x d_e row-major Khat_e starts at
  mats[mat_off[e]] (d_e = dof_ptr[e+1] - dof_ptr[e]); elements without
  enriched nodes share one 24 x 24 matrix;
* mats (float64).

Local dofs are node-major over the element's 8 corners, each node's dofs in
its own block order [3 standard | enriched], as the element matrices are
built.
"""
import numpy as np


def element_data(P):
    en = np.asarray(P.elem_nodes_free)               # (n_el, 8), -1 for clamped nodes
    n_el = en.shape[0]
    dof = np.asarray(P.dof_ptr, dtype=np.int64)
    bsz = np.diff(dof)
    size = np.where(en >= 0, bsz[np.maximum(en, 0)], 3)  # clamped nodes: 3 eliminated dofs
    d_e = size.sum(1)
    dof_ptr = np.zeros(n_el + 1, dtype=np.int64)
    dof_ptr[1:] = np.cumsum(d_e)
    dofs = np.full(int(dof_ptr[-1]), -1, dtype=np.int64)
    # element-local position of each node's first dof
    node_off = dof_ptr[:-1, None] + np.concatenate(
        [np.zeros((n_el, 1), dtype=np.int64), np.cumsum(size, 1)[:, :-1]], axis=1)
    for a in range(8):
        I = en[:, a]
        live = I >= 0
        for i in range(int(size.max())):
            sel = live & (i < size[:, a])
            dofs[node_off[sel, a] + i] = dof[I[sel]] + i
    fixed = np.asarray(getattr(P, "fixed_dofs", np.zeros(P.n, dtype=bool)))
    if fixed.any():
        live = dofs >= 0
        dofs[live & fixed[np.maximum(dofs, 0)]] = -1
    # matrices: the shared standard one first, then the enriched elements'
    khat_std = np.asarray(P.khat_std, dtype=np.float64)
    mats = np.concatenate([khat_std.ravel(), np.asarray(P.khat_enr, dtype=np.float64)])
    mat_off = np.zeros(n_el, dtype=np.int64)
    enr = np.asarray(P.enr_elements, dtype=np.int64)
    mat_off[enr] = khat_std.size + np.asarray(P.khat_enr_ptr, dtype=np.int64)[:-1]
    # each enriched matrix must match its element's dof count
    sizes = np.diff(np.asarray(P.khat_enr_ptr))
    if np.any(sizes != d_e[enr] ** 2) or np.any(d_e[np.setdiff1d(np.arange(n_el), enr)] != 24):
        raise ValueError("element matrices do not match the elements' dof counts")
    return {"dof_ptr": dof_ptr, "dofs": dofs.astype(np.int32), "mat_off": mat_off, "mats": mats,
            "young": np.asarray(P.young, dtype=np.float64)}
