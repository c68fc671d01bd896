"""Seeded synthetic XFEM crack problems: mesh, enrichment sets, element
integration and assembly into the node-blocked stiffness system K u = f.

This module produces the *inputs* of the solver (Section 2: weak form
Eq. weak_form_const_eq, approximation Eq. xfem_displ, block structure
Eq. linear_system).  It holds none of the solver's arithmetic: no CG, no
deflation, no preconditioner.

Mesh: unit cube of m^3 trilinear hexahedra, node (i, j, k) at (i, j, k)/m,
numbered with x fastest.  Nodes on z = 0 are clamped and eliminated together
with any enriched dofs they would carry; the others are the free nodes, kept
in the same order.  Each free node I owns b_I contiguous dofs:
[3 standard | 3 Heaviside] or [3 standard | 12 branch (4 functions x 3)].

Node sets (Section 2.3): a node is tip enriched if an element of its support
touches the front (phi and psi both take values <= 0 and >= 0 on the
element's nodes) or r_I <= r_e; otherwise it is jump enriched if its support
nodes take strictly negative and strictly positive phi while all have psi < 0.
Tip enrichment takes precedence.

Integration: elements without enriched nodes use 2x2x2 Gauss; elements with
enriched nodes are split into six tetrahedra, each split again along the zero
of the linear interpolant of phi, and integrated with the conical product
rule (3 points per direction, 4 when a tip node is present).  Inside such an
element phi and psi are the tetrahedron-wise linear interpolants of the nodal
level sets.
"""
import numpy as np

from .quadrature import HEX_CORNERS, HEX_TETS, hex_gauss, map_tet, split_tet
from .enrichment import branch_functions, heaviside, polar

KIND_STD, KIND_HEAVISIDE, KIND_TIP = 0, 1, 2
BLOCK_OF_KIND = {KIND_STD: 3, KIND_HEAVISIDE: 6, KIND_TIP: 15}


def lame(E, nu):
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def shape_functions(xi, h):
    """Trilinear shape functions on a hexahedron of edge h.

    xi: (P, 3) local coordinates in [0, 1]^3.  Returns N (8, P), dN (8, P, 3) in
    physical units.
    """
    P = xi.shape[0]
    N = np.ones((8, P))
    dN = np.ones((8, P, 3))
    for a in range(8):
        for d in range(3):
            if HEX_CORNERS[a, d] > 0:
                f, df = xi[:, d], 1.0
            else:
                f, df = 1.0 - xi[:, d], -1.0
            N[a] *= f
            for e in range(3):
                dN[a, :, e] *= (df / h) if e == d else f
    return N, dN


def stiffness_from_gradients(grads, w, lam, mu):
    """Element matrix from scalar basis-function gradients.

    grads: (F, P, 3) gradients of F scalar functions g_f; each gives 3 dofs
    (g_f e_c, c = 0..2), ordered f-major.  Returns (3F, 3F):
    K[fc, f'c'] = int lam d_c g_f d_c' g_f' + mu d_c' g_f d_c g_f' + mu delta_cc' grad g_f . grad g_f'.
    """
    F = grads.shape[0]
    G = (grads * np.sqrt(w)[None, :, None]).transpose(0, 2, 1).reshape(3 * F, -1)
    T = (G @ G.T).reshape(F, 3, F, 3)          # T[f, c, f', c'] = int d_c g_f d_c' g_f'
    tr = np.einsum("fdgd->fg", T)
    K = lam * T + mu * T.transpose(0, 3, 2, 1)
    K += mu * tr[:, None, :, None] * np.eye(3)[None, :, None, :]
    return K.reshape(3 * F, 3 * F)


JUMP_MIN_FRACTION = 1e-3


def _side_volumes(coords, elem_nodes, pe, h):
    """Volume of each element on the phi >= 0 and phi < 0 sides of the
    tetrahedron-wise linear interpolant of the nodal phi."""
    n_el = elem_nodes.shape[0]
    vpos = np.where(pe.min(1) >= 0, h ** 3, 0.0)
    vneg = np.where(pe.max(1) <= 0, h ** 3, 0.0)
    vpos[(pe.min(1) >= 0) & (pe.max(1) <= 0)] = h ** 3     # phi == 0 on all nodes
    cut = np.nonzero((pe.min(1) < 0) & (pe.max(1) > 0))[0]
    for e in cut:
        corners = coords[elem_nodes[e, 0]] + h * HEX_CORNERS
        vp = vn = 0.0
        for tet in HEX_TETS:
            for sub, side in split_tet(corners[tet], pe[e][tet]):
                vol = abs(np.linalg.det(sub[1:] - sub[0])) / 6.0
                if side > 0:
                    vp += vol
                else:
                    vn += vol
        vpos[e], vneg[e] = vp, vn
    return vpos, vneg


class Problem:
    """Assembled system plus the geometric data the deflation space is built from."""


def _standard_element_matrix(h, lam, mu):
    pts, w = hex_gauss(2)
    _, dN = shape_functions(pts, h)
    return stiffness_from_gradients(dN, w * h ** 3, lam, mu)


def _enriched_element_matrix(x0, h, lam, mu, kinds, phi8, psi8, rI, thI, order):
    """Element matrix of an element with enriched nodes (dofs node-major,
    [3 std | enriched] per node, in the node's own block order)."""
    corners = x0 + h * HEX_CORNERS
    pts_l, w_l, phi_l, psi_l, gphi_l, gpsi_l, side_l = [], [], [], [], [], [], []
    for tet in HEX_TETS:
        v = corners[tet]
        s = phi8[tet]
        t = psi8[tet]
        Jm = v[1:] - v[0]
        gphi = np.linalg.solve(Jm, s[1:] - s[0])
        gpsi = np.linalg.solve(Jm, t[1:] - t[0])
        for sub, side in split_tet(v, s):
            vol = abs(np.linalg.det(sub[1:] - sub[0])) / 6.0
            if vol < 1e-13 * h ** 3:
                continue
            p, w = map_tet(sub, order)
            dp = p - v[0]
            pts_l.append(p)
            w_l.append(w)
            phi_l.append(s[0] + dp @ gphi)
            psi_l.append(t[0] + dp @ gpsi)
            gphi_l.append(np.broadcast_to(gphi, p.shape))
            gpsi_l.append(np.broadcast_to(gpsi, p.shape))
            side_l.append(np.full(p.shape[0], float(side)))
    pts = np.concatenate(pts_l)
    w = np.concatenate(w_l)
    side = np.concatenate(side_l)
    phi = side * np.abs(np.concatenate(phi_l))     # sign fixed by the integration cell
    psi = np.concatenate(psi_l)
    gphi = np.concatenate(gphi_l)
    gpsi = np.concatenate(gpsi_l)
    N, dN = shape_functions((pts - x0) / h, h)
    H = side                                        # H(x) = sign(phi), +1 on phi >= 0
    grads = []
    need_polar = np.any(kinds == KIND_TIP)
    if need_polar:
        r, th = polar(phi, psi)
        r2 = np.maximum(r * r, 1e-300)
        gr = (phi[:, None] * gphi + psi[:, None] * gpsi) / np.maximum(r, 1e-300)[:, None]
        gth = (psi[:, None] * gphi - phi[:, None] * gpsi) / r2[:, None]
    for a in range(8):
        grads.append(dN[a])
        if kinds[a] == KIND_HEAVISIDE:
            Ha = 1.0 if phi8[a] >= 0.0 else -1.0
            grads.append(dN[a] * (H - Ha)[:, None])
        elif kinds[a] == KIND_TIP:
            F, dF = branch_functions(r, th, gr, gth, rI[a], thI[a])
            for j in range(4):
                grads.append(dN[a] * F[j][:, None] + N[a][:, None] * dF[j])
    return stiffness_from_gradients(np.stack(grads), w, lam, mu)


def build_problem(m, cracks, n_box, E=1.0, nu=0.3, traction=(0.0, 0.0, 1.0),
                  bc="clamp_bottom", young=None, centred_modes=True):
    """Assemble the XFEM system of one synthetic configuration.

    m: hexahedra per axis; cracks: list of Crack; n_box: box subdomains per axis;
    young: optional per-element Young's modulus (m^3,), else E everywhere;
    bc: "clamp_bottom" (z = 0 clamped), "roller" (u_x = 0 on x = 0, u_y = 0 on
    y = 0, u_z = 0 on z = 0) or "none" (unconstrained).
    """
    h = 1.0 / m
    n1 = m + 1
    ii, jj, kk = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
    # node id = i + n1 * (j + n1 * k); build coordinate array in that order
    ijk = np.stack([ii.transpose(2, 1, 0).ravel(), jj.transpose(2, 1, 0).ravel(),
                    kk.transpose(2, 1, 0).ravel()], axis=1)
    coords = ijk.astype(np.float64) / m
    n_all = n1 ** 3

    ei, ej, ek = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    eijk = np.stack([ei.transpose(2, 1, 0).ravel(), ej.transpose(2, 1, 0).ravel(),
                     ek.transpose(2, 1, 0).ravel()], axis=1)
    n_el = m ** 3
    elem_nodes = np.empty((n_el, 8), dtype=np.int64)
    for a in range(8):
        c = eijk + HEX_CORNERS[a].astype(np.int64)
        elem_nodes[:, a] = c[:, 0] + n1 * (c[:, 1] + n1 * c[:, 2])
    if young is None:
        young = np.full(n_el, E)
    young = np.asarray(young, dtype=np.float64)

    # ---- dof elimination per node: clamp_bottom removes whole nodes
    if bc == "clamp_bottom":
        node_free = ijk[:, 2] > 0
    else:
        node_free = np.ones(n_all, dtype=bool)

    # ---- enrichment sets
    kind = np.zeros(n_all, dtype=np.int64)
    owner = np.full(n_all, -1, dtype=np.int64)     # crack enriching the node
    phis, psis = [], []
    for ci, cr in enumerate(cracks):
        phi, psi = cr.phi_psi(coords)
        # level-set values within rounding of zero are snapped to +0.0, so a
        # node lying on the crack surface does not produce a support split by
        # a sliver of rounding-error size
        phi = np.where(np.abs(phi) < 1e-12 * h, 0.0, phi) + 0.0
        psi = np.where(np.abs(psi) < 1e-12 * h, 0.0, psi) + 0.0
        phis.append(phi)
        psis.append(psi)
        pe, qe = phi[elem_nodes], psi[elem_nodes]
        front_el = (pe.min(1) <= 0) & (pe.max(1) >= 0) & (qe.min(1) <= 0) & (qe.max(1) >= 0)
        tip = np.zeros(n_all, dtype=bool)
        tip[elem_nodes[front_el].ravel()] = True
        tip |= np.hypot(phi, psi) <= cr.r_e
        # support extrema over all nodes of the elements around each node
        smin_phi = np.full(n_all, np.inf)
        smax_phi = np.full(n_all, -np.inf)
        smax_psi = np.full(n_all, -np.inf)
        emin_phi, emax_phi, emax_psi = pe.min(1), pe.max(1), qe.max(1)
        for a in range(8):
            np.minimum.at(smin_phi, elem_nodes[:, a], emin_phi)
            np.maximum.at(smax_phi, elem_nodes[:, a], emax_phi)
            np.maximum.at(smax_psi, elem_nodes[:, a], emax_psi)
        jump = (smin_phi < 0) & (smax_phi > 0) & (smax_psi < 0) & ~tip
        # a support cut off by a sliver carries a jump function that is almost
        # zero (a near-dependent dof): keep a jump node only when each side of
        # its support holds at least JUMP_MIN_FRACTION of the support volume
        vpos, vneg = _side_volumes(coords, elem_nodes, pe, h)
        spos = np.zeros(n_all)
        sneg = np.zeros(n_all)
        for a in range(8):
            np.add.at(spos, elem_nodes[:, a], vpos)
            np.add.at(sneg, elem_nodes[:, a], vneg)
        frac = np.minimum(spos, sneg) / np.maximum(spos + sneg, 1e-300)
        jump &= frac >= JUMP_MIN_FRACTION
        new_kind = np.where(tip, KIND_TIP, np.where(jump, KIND_HEAVISIDE, KIND_STD))
        new_kind[~node_free] = KIND_STD             # enriched dofs at Dirichlet nodes are eliminated
        clash = (new_kind > 0) & (kind > 0)
        if np.any(clash):
            raise ValueError("enrichment supports of two cracks overlap")
        sel = new_kind > 0
        kind[sel] = new_kind[sel]
        owner[sel] = ci

    # element crack: the unique crack of its enriched nodes
    ek_kind = kind[elem_nodes]
    ek_owner = owner[elem_nodes]
    enr_el = np.nonzero((ek_kind > 0).any(1))[0]
    for e in enr_el:
        o = set(ek_owner[e][ek_owner[e] >= 0].tolist())
        if len(o) > 1:
            raise ValueError("an element holds nodes enriched by two cracks")

    # ---- free node numbering and dof layout
    free_ids = np.nonzero(node_free)[0]
    fid = np.full(n_all, -1, dtype=np.int64)
    fid[free_ids] = np.arange(free_ids.size)
    N = free_ids.size
    bsz = np.array([BLOCK_OF_KIND[k] for k in range(3)])[kind[free_ids]]
    dof_ptr = np.zeros(N + 1, dtype=np.int64)
    dof_ptr[1:] = np.cumsum(bsz)

    # ---- block pattern: free node pairs sharing an element
    en_f = fid[elem_nodes]                           # (n_el, 8), -1 for clamped
    A = np.repeat(en_f, 8, axis=1)
    B = np.tile(en_f, (1, 8))
    ok = (A >= 0) & (B >= 0)
    keys = np.unique(A[ok] * N + B[ok])
    rows, cols = keys // N, keys % N
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    nnzb = keys.size
    blk_size = bsz[rows] * bsz[cols]
    val_ptr = np.zeros(nnzb + 1, dtype=np.int64)
    val_ptr[1:] = np.cumsum(blk_size)
    val = np.zeros(int(val_ptr[-1]))

    def pair_index(I, J):
        return np.searchsorted(keys, I * N + J)

    # ---- standard elements: shared unit element matrix scaled by E_e
    lam1, mu1 = lame(1.0, nu)
    Ke0 = _standard_element_matrix(h, lam1, mu1)     # (24, 24) for E = 1
    std_el = np.ones(n_el, dtype=bool)
    std_el[enr_el] = False
    se = np.nonzero(std_el)[0]
    for a in range(8):
        Ia = en_f[se, a]
        for b in range(8):
            Jb = en_f[se, b]
            okp = (Ia >= 0) & (Jb >= 0)
            pidx = pair_index(Ia[okp], Jb[okp])
            blk = young[se[okp], None, None] * Ke0[3 * a:3 * a + 3, 3 * b:3 * b + 3][None]
            # scatter the 3x3 std-std part: rows 0..2 of the b_I x b_J block
            base = val_ptr[pidx]
            wJ = bsz[cols[pidx]]
            for r in range(3):
                for c in range(3):
                    np.add.at(val, base + r * wJ + c, blk[:, r, c])

    # ---- enriched elements
    rI_all = np.zeros(n_all)
    thI_all = np.zeros(n_all)
    for ci in range(len(cracks)):
        sel = owner == ci
        r_, t_ = polar(phis[ci][sel], psis[ci][sel])
        rI_all[sel], thI_all[sel] = r_, t_
    n_enr_dofs_el = []
    khat_enr = []                                    # element matrices for E = 1
    for e in enr_el:
        nodes = elem_nodes[e]
        kinds_e = kind[nodes]
        ci = int(ek_owner[e][ek_owner[e] >= 0][0])
        order = 4 if np.any(kinds_e == KIND_TIP) else 3
        x0 = coords[nodes[0]]
        Khat = _enriched_element_matrix(x0, h, lam1, mu1, kinds_e, phis[ci][nodes],
                                        psis[ci][nodes], rI_all[nodes], thI_all[nodes], order)
        khat_enr.append(Khat)
        Ke = young[e] * Khat                         # K_e is linear in E at fixed nu
        loc = np.array([BLOCK_OF_KIND[k] for k in kinds_e])
        off = np.concatenate([[0], np.cumsum(loc)])
        n_enr_dofs_el.append(off[-1])
        for a in range(8):
            I = en_f[e, a]
            if I < 0:
                continue
            for b in range(8):
                J = en_f[e, b]
                if J < 0:
                    continue
                p = pair_index(np.array([I]), np.array([J]))[0]
                blk = Ke[off[a]:off[a + 1], off[b]:off[b + 1]]
                val[val_ptr[p]:val_ptr[p + 1]] += blk.ravel()

    # ---- loads: uniform traction on z = 1 (consistent nodal forces, bilinear face)
    n = int(dof_ptr[-1])
    f = np.zeros(n)
    top = ijk[:, 2] == m
    if np.any(kind[top] > 0) and np.any(np.asarray(traction) != 0):
        raise ValueError("enriched nodes on the loaded face are not supported")
    t = np.asarray(traction, dtype=np.float64)
    face_w = np.zeros(n_all)
    corner_w = h * h / 4.0
    for di in (0, 1):
        for dj in (0, 1):
            face_i = ijk[:, 0] - di
            face_j = ijk[:, 1] - dj
            okf = top & (face_i >= 0) & (face_i < m) & (face_j >= 0) & (face_j < m)
            face_w[okf] += corner_w
    for I_all in np.nonzero(face_w > 0)[0]:
        I = fid[I_all]
        f[dof_ptr[I]:dof_ptr[I] + 3] += face_w[I_all] * t

    # ---- roller / extra constraints: eliminate single std dofs by zeroing rows/cols
    fixed_dofs = np.zeros(n, dtype=bool)
    if bc == "roller":
        for d, axis in ((0, 0), (1, 1), (2, 2)):
            nodes_on = np.nonzero(ijk[:, axis] == 0)[0]
            fixed_dofs[dof_ptr[fid[nodes_on]] + d] = True

    # ---- box subdomains (half-open boxes, last box closed)
    bidx = np.minimum(ijk * n_box // m, n_box - 1)
    sub_all = bidx[:, 0] + n_box * (bidx[:, 1] + n_box * bidx[:, 2])
    n_sub = n_box ** 3
    bc3 = np.stack(np.meshgrid(np.arange(n_box), np.arange(n_box), np.arange(n_box),
                               indexing="ij"), -1).transpose(2, 1, 0, 3).reshape(-1, 3)
    centres = (bc3 + 0.5) / n_box if centred_modes else np.zeros((n_sub, 3))

    # Heaviside sign of each node w.r.t. the crack of its box (the crack of the
    # jump-enriched nodes in that box); +1 in boxes without jump-enriched nodes.
    box_crack = np.full(n_sub, -1, dtype=np.int64)
    jn = np.nonzero((kind == KIND_HEAVISIDE) & node_free)[0]
    for I in jn:
        s = sub_all[I]
        if box_crack[s] >= 0 and box_crack[s] != owner[I]:
            raise ValueError("a box holds jump-enriched nodes of two cracks")
        box_crack[s] = owner[I]
    hsign_all = np.ones(n_all, dtype=np.int8)
    for ci in range(len(cracks)):
        sel = box_crack[sub_all] == ci
        hsign_all[sel] = np.where(phis[ci][sel] >= 0.0, 1, -1).astype(np.int8)

    P = Problem()
    P.m, P.h, P.n_box = m, h, n_box
    P.n_nodes = N
    P.n = n
    P.dof_ptr = dof_ptr.astype(np.int32)
    P.row_ptr = row_ptr.astype(np.int32)
    P.col = cols.astype(np.int32)
    P.val_ptr = val_ptr
    P.val = val
    P.f = f
    P.fixed_dofs = fixed_dofs
    P.coords = coords[free_ids].copy()
    P.kind = kind[free_ids].astype(np.int8)
    P.sub_of_node = sub_all[free_ids].astype(np.int32)
    P.n_sub = n_sub
    P.centres = centres
    P.hsign = hsign_all[free_ids]
    P.node_ids = free_ids
    P.elem_nodes_free = en_f
    P.young = young
    P.nu = nu
    P.n_enriched_elements = len(enr_el)
    # per-element stiffness for unit Young's modulus (dK/dE_e), node-major
    # with each node's dofs in its own block order
    P.khat_std = Ke0
    P.enr_elements = np.asarray(enr_el, dtype=np.int64)
    P.khat_enr_ptr = np.zeros(len(enr_el) + 1, dtype=np.int64)
    P.khat_enr_ptr[1:] = np.cumsum([K.size for K in khat_enr])
    P.khat_enr = (np.concatenate([K.ravel() for K in khat_enr]) if khat_enr
                  else np.zeros(0))
    P.n_heaviside_dofs = int(3 * np.sum(P.kind == KIND_HEAVISIDE))
    P.n_tip_dofs = int(12 * np.sum(P.kind == KIND_TIP))
    if bc == "roller":
        _apply_dof_constraints(P)
    return P


def _apply_dof_constraints(P):
    """Zero-displacement single dofs: remove their rows and columns by zeroing
    them and putting 1 on the diagonal (decoupled identity rows, f = 0)."""
    fixed = P.fixed_dofs
    N = P.n_nodes
    for I in range(N):
        for p in range(P.row_ptr[I], P.row_ptr[I + 1]):
            J = P.col[p]
            bI = P.dof_ptr[I + 1] - P.dof_ptr[I]
            bJ = P.dof_ptr[J + 1] - P.dof_ptr[J]
            blk = P.val[P.val_ptr[p]:P.val_ptr[p + 1]].reshape(bI, bJ)
            ri = fixed[P.dof_ptr[I]:P.dof_ptr[I + 1]]
            cj = fixed[P.dof_ptr[J]:P.dof_ptr[J + 1]]
            blk[ri, :] = 0.0
            blk[:, cj] = 0.0
            if I == J:
                for d in np.nonzero(ri)[0]:
                    blk[d, d] = 1.0
    P.f[fixed] = 0.0


def to_dense(P):
    """Dense K (n x n) of a small problem."""
    K = np.zeros((P.n, P.n))
    for I in range(P.n_nodes):
        for p in range(P.row_ptr[I], P.row_ptr[I + 1]):
            J = P.col[p]
            r0, r1 = P.dof_ptr[I], P.dof_ptr[I + 1]
            c0, c1 = P.dof_ptr[J], P.dof_ptr[J + 1]
            K[r0:r1, c0:c1] = P.val[P.val_ptr[p]:P.val_ptr[p + 1]].reshape(r1 - r0, c1 - c0)
    return K


def by_subdomain(P):
    """The same system with its free nodes renumbered subdomain by
    subdomain (nodes of box 0 first, each box's nodes in their original
    order), so that every box's dofs form one contiguous range.  Returns
    (P2, block_ptr): block_ptr[s] .. block_ptr[s + 1] is box s's dof range,
    the blocks of the subdomain-sized block Jacobi of Section 3.4.  Only
    integer relabelling: every matrix entry, load and coordinate is moved,
    none is computed."""
    import copy
    sub = np.asarray(P.sub_of_node)
    perm = np.argsort(sub, kind="stable")            # new node i = old node perm[i]
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    dof = np.asarray(P.dof_ptr, dtype=np.int64)
    bsz = np.diff(dof)
    nbsz = bsz[perm]
    ndof = np.zeros(P.n_nodes + 1, dtype=np.int64)
    ndof[1:] = np.cumsum(nbsz)
    # dof map old -> new (within-node order kept)
    dmap = np.empty(P.n, dtype=np.int64)
    for I in range(P.n_nodes):
        dmap[dof[I]:dof[I + 1]] = ndof[inv[I]] + np.arange(bsz[I])
    rowp = np.asarray(P.row_ptr, dtype=np.int64)
    col = np.asarray(P.col, dtype=np.int64)
    vptr = np.asarray(P.val_ptr, dtype=np.int64)
    nrowp = np.zeros(P.n_nodes + 1, dtype=np.int64)
    ncol, nvals, nvptr = [], [], [0]
    for i in range(P.n_nodes):
        I = perm[i]
        ps = np.arange(rowp[I], rowp[I + 1])
        ps = ps[np.argsort(inv[col[ps]], kind="stable")]
        for p in ps:
            ncol.append(inv[col[p]])
            nvals.append(P.val[vptr[p]:vptr[p + 1]])
            nvptr.append(nvptr[-1] + vptr[p + 1] - vptr[p])
        nrowp[i + 1] = nrowp[i] + ps.size
    P2 = copy.copy(P)
    P2.dof_ptr = ndof.astype(np.int32)
    P2.row_ptr = nrowp.astype(np.int32)
    P2.col = np.asarray(ncol, dtype=np.int32)
    P2.val_ptr = np.asarray(nvptr, dtype=np.int64)
    P2.val = np.concatenate(nvals)
    f = np.empty(P.n)
    f[dmap] = P.f
    P2.f = f
    fixed = np.zeros(P.n, dtype=bool)
    fixed[dmap] = np.asarray(P.fixed_dofs)
    P2.fixed_dofs = fixed
    P2.coords = P.coords[perm].copy()
    P2.kind = np.asarray(P.kind)[perm].copy()
    P2.sub_of_node = sub[perm].copy()
    P2.hsign = np.asarray(P.hsign)[perm].copy()
    P2.node_ids = np.asarray(P.node_ids)[perm].copy()
    en = np.asarray(P.elem_nodes_free)
    P2.elem_nodes_free = np.where(en >= 0, inv[np.maximum(en, 0)], -1)
    counts = np.bincount(P2.sub_of_node, minlength=P.n_sub)
    node_ptr = np.concatenate([[0], np.cumsum(counts)])
    block_ptr = ndof[node_ptr].astype(np.int32)
    P2.dof_map_from = dmap
    return P2, block_ptr
