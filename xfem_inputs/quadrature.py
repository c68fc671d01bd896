"""Quadrature rules and the sub-tetrahedral split of cut hexahedra.

Used by the XFEM assembly (Section 2.3, Eq. xfem_displ): elements whose
nodes carry enriched dofs are integrated over six tetrahedra per hexahedron,
each tetrahedron further split along the zero level of the linear interpolant
of the normal level set phi so that the Heaviside and branch functions are
smooth inside every integration cell.

Tetrahedral cells use the conical (collapsed) product rule: Gauss-Jacobi
points in the two collapsed directions (weights (1-a)^2 and (1-b)), plain
Gauss-Legendre in the last one, so an n-point rule integrates every
polynomial of total degree <= 2n-1 exactly.
"""
import numpy as np
from scipy.special import roots_jacobi, roots_legendre

# Corners of the unit hexahedron in the standard trilinear node order.
HEX_CORNERS = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                        [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], dtype=np.float64)

# Six tetrahedra sharing the main diagonal 0-6 (Kuhn triangulation); they tile the cube.
HEX_TETS = np.array([[0, 1, 2, 6], [0, 2, 3, 6], [0, 3, 7, 6],
                     [0, 7, 4, 6], [0, 4, 5, 6], [0, 5, 1, 6]], dtype=np.int64)


def gauss_legendre_01(n):
    """n-point Gauss-Legendre rule on [0, 1]."""
    x, w = roots_legendre(n)
    return 0.5 * (x + 1.0), 0.5 * w


def hex_gauss(n):
    """Tensor Gauss-Legendre rule on the unit cube: points (n^3, 3), weights (n^3,)."""
    x, w = gauss_legendre_01(n)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    WX, WY, WZ = np.meshgrid(w, w, w, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    return pts, (WX * WY * WZ).ravel()


_TET_RULE_CACHE = {}


def tet_rule(n):
    """Conical product rule on the reference tetrahedron {xi >= 0, sum(xi) <= 1}.

    Returns barycentric-style coordinates (n^3, 3) (xi1, xi2, xi3) and weights
    summing to 1/6 (the reference volume).
    """
    if n in _TET_RULE_CACHE:
        return _TET_RULE_CACHE[n]
    xa, wa = roots_jacobi(n, 2.0, 0.0)   # weight (1-x)^2 on [-1, 1]
    xb, wb = roots_jacobi(n, 1.0, 0.0)   # weight (1-x)   on [-1, 1]
    xc, wc = roots_legendre(n)
    a, wa = 0.5 * (xa + 1.0), wa / 8.0
    b, wb = 0.5 * (xb + 1.0), wb / 4.0
    c, wc = 0.5 * (xc + 1.0), wc / 2.0
    A, B, C = np.meshgrid(a, b, c, indexing="ij")
    WA, WB, WC = np.meshgrid(wa, wb, wc, indexing="ij")
    A, B, C = A.ravel(), B.ravel(), C.ravel()
    xi = np.stack([A, (1.0 - A) * B, (1.0 - A) * (1.0 - B) * C], axis=1)
    w = (WA * WB * WC).ravel()
    _TET_RULE_CACHE[n] = (xi, w)
    return xi, w


def tet_volume(v):
    """Unsigned volume of tetrahedron with vertices v (4, 3)."""
    return abs(np.linalg.det(v[1:] - v[0])) / 6.0


def map_tet(v, n):
    """Quadrature points (P, 3) and weights (P,) on the physical tetrahedron v."""
    xi, w = tet_rule(n)
    J = (v[1:] - v[0])                      # rows: edge vectors
    pts = v[0] + xi @ J
    return pts, w * (6.0 * tet_volume(v))


def _prism(a, b, c, a2, b2, c2):
    """Split a prism with triangles (a,b,c), (a2,b2,c2) and lateral edges a-a2, b-b2, c-c2."""
    return [np.array([a, b, c, a2]), np.array([b, c, a2, b2]), np.array([c, a2, b2, c2])]


def split_tet(v, s):
    """Split tetrahedron v (4, 3) along the zero of the linear field with vertex values s.

    Returns a list of (sub-tetrahedron (4, 3), side) with side = +1 where the
    field is >= 0 and -1 where it is < 0.  A tetrahedron without a strict sign
    change is returned whole.
    """
    pos = [i for i in range(4) if s[i] > 0.0]
    neg = [i for i in range(4) if s[i] < 0.0]
    zer = [i for i in range(4) if s[i] == 0.0]
    if not pos or not neg:
        return [(v.copy(), 1 if pos else -1)]

    def cut(i, j):
        t = s[i] / (s[i] - s[j])
        return v[i] + t * (v[j] - v[i])

    out = []
    if len(pos) == 1 and len(neg) == 1:
        p, q = pos[0], neg[0]
        c = cut(p, q)
        z1, z2 = v[zer[0]], v[zer[1]]
        out.append((np.array([v[p], c, z1, z2]), 1))
        out.append((np.array([v[q], c, z1, z2]), -1))
    elif (len(pos) == 1 and len(neg) == 2) or (len(pos) == 2 and len(neg) == 1):
        lone, pair = (pos, neg) if len(pos) == 1 else (neg, pos)
        sl = 1 if len(pos) == 1 else -1
        p = lone[0]
        n1, n2 = pair
        c1, c2 = cut(p, n1), cut(p, n2)
        z = v[zer[0]]
        out.append((np.array([v[p], c1, c2, z]), sl))
        out.append((np.array([z, v[n1], v[n2], c2]), -sl))
        out.append((np.array([z, v[n1], c2, c1]), -sl))
    elif len(pos) == 1 or len(neg) == 1:
        lone, tri = (pos, neg) if len(pos) == 1 else (neg, pos)
        sl = 1 if len(pos) == 1 else -1
        p = lone[0]
        cs = [cut(p, q) for q in tri]
        out.append((np.array([v[p], cs[0], cs[1], cs[2]]), sl))
        for t in _prism(v[tri[0]], v[tri[1]], v[tri[2]], cs[0], cs[1], cs[2]):
            out.append((t, -sl))
    else:  # two positive, two negative
        p1, p2 = pos
        n1, n2 = neg
        c11, c12, c21, c22 = cut(p1, n1), cut(p1, n2), cut(p2, n1), cut(p2, n2)
        for t in _prism(v[p1], c11, c12, v[p2], c21, c22):
            out.append((t, 1))
        for t in _prism(v[n1], c11, c21, v[n2], c12, c22):
            out.append((t, -1))
    return out
