"""FP64 CPU oracle of the adapted deflated CG solver (A-DEF2 + block Jacobi).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check of the GPU
library and the CPU-baseline leg of the benchmark may import this module.
It shares no code with the GPU path.

Plain, slow and literal:
* Z      -- subdomain rigid-body modes (Section 3.3.1, Eq. dcg_deflation_space)
            augmented in subdomains holding jump-enriched nodes with the
            enriched modes (Section 3.3.2, Eqs. enriched_deflated_modes,
            dcg_deflation_space_enr_std, dcg_deflation_space_enr_enr).
* M^-1   -- block Jacobi (Section 3.4, Eqs. block_jacobi, block_jacobi_enr):
            dense Cholesky of each diagonal block, two triangular solves;
            blocks per node (the GPU path's choice) or per subdomain (the
            paper's experiments).
* u_0    -- Algorithm 2 (two coarse solves).
* z      -- Algorithm 3 (two coarse solves, W^T K y evaluated as Z^T (K y)).
* loop   -- Algorithm 1, stopped when ||r_i||_2 <= tol ||f||_2, the test made
            after every residual update; the iteration count is the number of
            loop bodies run (products K p).
* dJ/dE  -- sensitivity of J(u), u = K^-1 f, to each element's Young's
            modulus (not in the paper; the adjoint of the solve): K depends on
            E_e through E_e Khat_e, so dJ/dE_e = -lam_e^T Khat_e u_e with
            K lam = dJ/du.  Pinned by central differences of J over rebuilt
            systems and by sum_e E_e dJ/dE_e = -lam^T f.

Readings of the paper that this file fixes:
* the coordinates in the rigid-body block are taken relative to a per-box
  centre supplied with the input (the span is the same as with global
  coordinates, because the translation columns absorb the shift);
* enriched modes exist only in boxes whose jump-enriched nodes are not all
  on one line (so at least three); their entries on branch-function dofs are
  zero;
* a diagonal block whose Cholesky pivot is <= 1e-14 times its largest
  diagonal entry is rejected (no shift is applied).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


class NotSPD(Exception):
    pass


class Breakdown(Exception):
    pass


def stiffness_csr(P):
    """K of Eq. linear_system (Section 2.4) as a scipy CSR matrix, from the
    node-blocked storage of Problem P."""
    dof = np.asarray(P.dof_ptr, dtype=np.int64)
    rowp = np.asarray(P.row_ptr, dtype=np.int64)
    col = np.asarray(P.col, dtype=np.int64)
    vptr = np.asarray(P.val_ptr, dtype=np.int64)
    bsz = np.diff(dof)
    I = np.repeat(np.arange(P.n_nodes), np.diff(rowp))
    bI, bJ = bsz[I], bsz[col]
    rows, cols, vals = [], [], []
    for ri in np.unique(bI):
        for cj in np.unique(bJ):
            sel = np.nonzero((bI == ri) & (bJ == cj))[0]
            if sel.size == 0:
                continue
            a = np.arange(ri)[:, None].repeat(cj, 1).ravel()     # row within block
            b = np.arange(cj)[None, :].repeat(ri, 0).ravel()     # column within block
            rows.append((dof[I[sel]][:, None] + a[None, :]).ravel())
            cols.append((dof[col[sel]][:, None] + b[None, :]).ravel())
            vals.append(P.val[(vptr[sel][:, None] + np.arange(ri * cj)[None, :]).ravel()])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(P.n, P.n))


def rigid_block(x):
    """3 x 6 nodal block of Eq. dcg_deflation_space at position x = (x, y, z)."""
    X, Y, Zc = x
    return np.array([[1.0, 0.0, 0.0, 0.0, Zc, -Y],
                     [0.0, 1.0, 0.0, -Zc, 0.0, X],
                     [0.0, 0.0, 1.0, Y, -X, 0.0]])


def collinear(x):
    """True when the points x (p, 3) lie on one line (always for p < 3).

    The jump dofs of a box carry the enriched modes as the plain rigid block
    (Eq. dcg_deflation_space_enr_enr); over collinear points that block has
    rank < 6, and when every node of the box sits on one side of the crack
    the enriched columns then repeat the rigid ones, so such a box gets no
    enriched modes."""
    if x.shape[0] < 3:
        return True
    a = x[0]
    d2 = np.sum((x - a) ** 2, axis=1)
    b = x[int(np.argmax(d2))]
    ab = b - a
    cr = np.cross(x - a, ab)
    return bool(np.all(np.sum(cr * cr, axis=1) <= 1e-12 * (ab @ ab) ** 2))


def deflation_basis(P, enriched=True):
    """Z (n x k, scipy CSC) of Section 3.3 and the first column of each box.

    Box s owns columns [col0[s], col0[s] + 6) for the rigid modes and, when it
    holds a jump-enriched node (and `enriched`), [col0[s] + 6, col0[s] + 12)
    for the enriched modes.
    """
    kind = np.asarray(P.kind)
    sub = np.asarray(P.sub_of_node)
    has_jump = np.zeros(P.n_sub, dtype=bool)
    if enriched:
        for s in np.unique(sub[kind == 1]):
            has_jump[s] = not collinear(P.coords[(sub == s) & (kind == 1)])
    m_s = np.where(has_jump, 12, 6)
    col0 = np.zeros(P.n_sub + 1, dtype=np.int64)
    col0[1:] = np.cumsum(m_s)
    dof = np.asarray(P.dof_ptr, dtype=np.int64)
    X = np.asarray(P.coords) - np.asarray(P.centres)[sub]
    zero, one = np.zeros(P.n_nodes), np.ones(P.n_nodes)
    # rigid block of Eq. dcg_deflation_space, entry [a][b] for every node
    R = np.array([[one, zero, zero, zero, X[:, 2], -X[:, 1]],
                  [zero, one, zero, -X[:, 2], zero, X[:, 0]],
                  [zero, zero, one, X[:, 1], -X[:, 0], zero]])      # (3, 6, N)
    c0 = col0[sub]
    H = np.asarray(P.hsign, dtype=np.float64)
    enr = has_jump[sub]
    jump = enr & (kind == 1)
    rows, cols, vals = [], [], []
    for a in range(3):
        for b in range(6):
            v = R[a, b]
            rows.append(dof[:-1] + a); cols.append(c0 + b); vals.append(v)
            # Eq. dcg_deflation_space_enr_std on standard dofs of enriched boxes
            rows.append((dof[:-1] + a)[enr]); cols.append((c0 + 6 + b)[enr])
            vals.append((H * v)[enr])
            # Eq. dcg_deflation_space_enr_enr on the jump dofs
            rows.append((dof[:-1] + 3 + a)[jump]); cols.append((c0 + 6 + b)[jump])
            vals.append(v[jump])
    rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    nz = vals != 0.0
    rows, cols, vals = rows[nz], cols[nz], vals[nz]
    Z = sp.csc_matrix((np.array(vals), (np.array(rows), np.array(cols))),
                      shape=(P.n, int(col0[-1])))
    return Z, col0


class BlockJacobi:
    """M^-1 of Eq. block_jacobi / block_jacobi_enr: contiguous dof blocks,
    each factored by dense Cholesky at set-up and applied by two triangular solves."""

    def __init__(self, K, block_ptr):
        self.block_ptr = np.asarray(block_ptr, dtype=np.int64)
        Kc = K.tocsr()
        sizes = np.diff(self.block_ptr)
        self.groups = []
        for b in np.unique(sizes):
            ids = np.nonzero(sizes == b)[0]
            idx = self.block_ptr[ids][:, None] + np.arange(b)[None, :]
            blocks = np.empty((ids.size, b, b))
            for t, i in enumerate(ids):
                d = idx[t]
                blocks[t] = Kc[d[0]:d[-1] + 1, d[0]:d[-1] + 1].toarray()
            L = np.zeros_like(blocks)
            for t in range(ids.size):
                try:
                    L[t] = np.linalg.cholesky(blocks[t])
                except np.linalg.LinAlgError:
                    raise NotSPD(int(ids[t]))
                dmax = np.max(np.diag(blocks[t]))
                if np.min(np.diag(L[t])) ** 2 <= 1e-14 * dmax:
                    raise NotSPD(int(ids[t]))
            self.groups.append((idx, L))

    def apply(self, r):
        y = np.empty_like(r)
        for idx, L in self.groups:
            rb = r[idx][:, :, None]
            w = np.linalg.solve(L, rb)
            y[idx] = np.linalg.solve(np.swapaxes(L, 1, 2), w)[:, :, 0]
        return y


class SubdomainJacobi:
    """M^-1 with one block per subdomain, the block choice of the paper's
    experiments (Section 3.4: all dofs of a subdomain, enriched ones
    included, form one diagonal block of K), each block factored by dense
    Cholesky at set-up.  groups: one array of global dofs per block."""

    def __init__(self, K, groups):
        Kc = K.tocsr()
        self.groups = [np.asarray(g, dtype=np.int64) for g in groups]
        self.cho = []
        for i, g in enumerate(self.groups):
            B = Kc[g][:, g].toarray()
            try:
                self.cho.append(sla.cho_factor(B, lower=True))
            except np.linalg.LinAlgError:
                raise NotSPD(i)

    def apply(self, r):
        y = np.zeros_like(r)
        for g, c in zip(self.groups, self.cho):
            y[g] = sla.cho_solve(c, r[g])
        return y


def subdomain_dofs(P):
    """The dofs of each box subdomain (its nodes' dofs, node by node): the
    blocks of the subdomain-sized block Jacobi of Section 3.4."""
    dof = np.asarray(P.dof_ptr, dtype=np.int64)
    sub = np.asarray(P.sub_of_node)
    out = []
    for s in range(P.n_sub):
        nodes = np.nonzero(sub == s)[0]
        out.append(np.concatenate([np.arange(dof[I], dof[I + 1]) for I in nodes])
                   if nodes.size else np.zeros(0, dtype=np.int64))
    return out


class Identity:
    """M = I: Algorithm 3 without the block-Jacobi part (test cases)."""

    def apply(self, r):
        return r.copy()


class Coarse:
    """E = Z^T K Z, the coarse matrix of the deflation (Section 3.2), factored
    by dense Cholesky; k = 0 gives no deflation."""

    def __init__(self, K, Z):
        self.Z = Z
        self.k = Z.shape[1]
        if self.k:
            E = (Z.T @ (K @ Z)).toarray()
            self.E = 0.5 * (E + E.T)
            try:
                self.cho = sla.cho_factor(self.E, lower=True)
            except np.linalg.LinAlgError:
                raise NotSPD(-1)

    def solve(self, rhs):
        return sla.cho_solve(self.cho, rhs)


def adef2_apply(K, M, C, r):
    """Algorithm 3: z = y + Z (lambda - mu), y = M^-1 r."""
    y = M.apply(r)
    if C.k == 0:
        return y
    mu = C.solve(C.Z.T @ (K @ y))
    lam = C.solve(C.Z.T @ r)
    return y + C.Z @ (lam - mu)


def adef2_initial(K, C, f, u_m1):
    """Algorithm 2: u_0 = u_-1 + Z (mu - lambda)."""
    if C.k == 0:
        return u_m1.copy()
    lam = C.solve(C.Z.T @ (K @ u_m1))
    mu = C.solve(C.Z.T @ f)
    return u_m1 + C.Z @ (mu - lam)


class Result:
    pass


def adef2_pcg(K, f, M, C, tol=1e-8, maxit=10000, u_m1=None, record=False, max_iterates=0):
    """Algorithm 1 preconditioned by Algorithm 3, started from Algorithm 2."""
    n = f.size
    if u_m1 is None:
        u_m1 = np.zeros(n)
    fn = np.linalg.norm(f)
    res = Result()
    res.rel_res, res.true_res, res.ztr, res.iterates = [], [], [], []
    u = adef2_initial(K, C, f, u_m1)
    r = f - K @ u
    if record:
        res.rel_res.append(np.linalg.norm(r) / fn if fn > 0 else 0.0)
        if C.k:
            res.ztr.append(np.linalg.norm(C.Z.T @ r))
    if max_iterates:
        res.iterates.append(u.copy())
    its = 0
    if fn == 0.0 or np.linalg.norm(r) <= tol * fn:
        res.u, res.iterations, res.converged = u, 0, True
        return res
    z = adef2_apply(K, M, C, r)
    p = z.copy()
    rz = r @ z
    converged = False
    for i in range(maxit):
        q = K @ p
        pq = p @ q
        if not (pq > 0.0):
            raise Breakdown(i)
        alpha = rz / pq
        u = u + alpha * p
        r = r - alpha * q
        its = i + 1
        rn = np.linalg.norm(r)
        if record:
            res.rel_res.append(rn / fn)
            res.true_res.append(np.linalg.norm(f - K @ u) / fn)
            if C.k:
                res.ztr.append(np.linalg.norm(C.Z.T @ r))
        if max_iterates and len(res.iterates) < max_iterates:
            res.iterates.append(u.copy())
        if rn <= tol * fn:
            converged = True
            break
        z = adef2_apply(K, M, C, r)
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    res.u, res.iterations, res.converged = u, its, converged
    return res


def nicolaides_dcg(K, f, M, C, tol=1e-8, maxit=10000, max_iterates=0):
    """Deflated PCG in the form of Nicolaides / Saad et al.: start from
    u_0 = Q f, search directions p = z - Z E^-1 Z^T K z with z = M^-1 r.
    Used only to check the equivalence stated for A-DEF2 with the start of
    Algorithm 2 (Section 3.2)."""
    fn = np.linalg.norm(f)
    u = C.Z @ C.solve(C.Z.T @ f)
    r = f - K @ u
    z = M.apply(r)
    p = z - C.Z @ C.solve(C.Z.T @ (K @ z))
    rz = r @ z
    iterates = [u.copy()]
    its = 0
    for i in range(maxit):
        q = K @ p
        alpha = rz / (p @ q)
        u = u + alpha * p
        r = r - alpha * q
        its = i + 1
        if len(iterates) < max_iterates:
            iterates.append(u.copy())
        if np.linalg.norm(r) <= tol * fn:
            break
        z = M.apply(r)
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p - C.Z @ C.solve(C.Z.T @ (K @ z))
    return u, its, iterates


def setup(P, enriched_modes=True):
    """K (CSR), node-block Jacobi, and the coarse operator for Problem P."""
    K = stiffness_csr(P)
    Z, _ = deflation_basis(P, enriched=enriched_modes)
    M = BlockJacobi(K, P.dof_ptr)
    C = Coarse(K, Z)
    return K, M, C


def solve(P, tol=1e-8, maxit=10000, record=False, enriched_modes=True):
    """setup() and adef2_pcg() for Problem P's own load."""
    K, M, C = setup(P, enriched_modes)
    return adef2_pcg(K, P.f, M, C, tol=tol, maxit=maxit, record=record)


def element_sensitivity(D, u, lam, elements=None):
    """dJ/dE_e = -lam_e^T Khat_e u_e for the given elements (all by default).

    D: element data (xfem_inputs.element_data): each element's global dofs
    (-1 where eliminated) and its unit-modulus matrix Khat_e; u: the solution;
    lam: the adjoint solution, K lam = dJ/du.  One element at a time, as
    written."""
    if elements is None:
        elements = range(len(D["mat_off"]))
    out = []
    for e in elements:
        d = D["dofs"][D["dof_ptr"][e]:D["dof_ptr"][e + 1]]
        de = d.size
        Kh = D["mats"][D["mat_off"][e]:D["mat_off"][e] + de * de].reshape(de, de)
        live = d >= 0
        ue = np.where(live, u[np.maximum(d, 0)], 0.0)
        le = np.where(live, lam[np.maximum(d, 0)], 0.0)
        out.append(-(le @ (Kh @ ue)))
    return np.array(out)
