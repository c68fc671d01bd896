"""Several load cases on one crack configuration (the right-hand sides of a
batched solve).  Every case is a uniform traction on the face z = 1 with
consistent nodal forces; the workloads' own load is the unit tension
t = (0, 0, 1), so its z-entries are the nodes' face weights and any traction t
gives f_t = weight * t on each loaded node's standard dofs."""
import numpy as np


def face_weights(P):
    """Per-node consistent face weight of the loaded face (from the unit-tension load)."""
    dof = np.asarray(P.dof_ptr)
    w = np.asarray(P.f)[dof[:-1] + 2].copy()
    if np.any(np.asarray(P.f)[dof[:-1]] != 0) or np.any(np.asarray(P.f)[dof[:-1] + 1] != 0):
        raise ValueError("the problem's load is not the unit tension along z")
    return w


def tractions(count, seed=0):
    """count seeded tractions: shear components (x, y) and a tension component
    (z), each of magnitude U[0.5, 1.5]; shear signs random, tension positive."""
    rng = np.random.default_rng(seed)
    mag = rng.uniform(0.5, 1.5, size=(count, 3))
    sign = np.where(rng.random((count, 2)) < 0.5, -1.0, 1.0)
    t = mag.copy()
    t[:, :2] *= sign
    return t


def load_cases(P, count, seed=0):
    """(count, n) array of load vectors, one per seeded traction."""
    dof = np.asarray(P.dof_ptr)
    w = face_weights(P)
    F = np.zeros((count, int(dof[-1])))
    for c, t in enumerate(tractions(count, seed)):
        for d in range(3):
            F[c, dof[:-1] + d] = w * t[d]
    return F
