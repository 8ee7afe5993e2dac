"""T10 element: shape functions, 5-point Keast rule, reference geometry, mass.

Paper passages followed:
  * Sec. 4.1 (precomputation): shape-function values s_i(u_q), reference
    gradients, quadrature nodes/weights, J_q = det(dX/dxi), constant element
    mass m_ij = int rho s_i s_j dV with M_e = [m_ij I_3].
  * Sec. 4.3, Stage 1: T10 uses n_en = 10 shape functions and the 5-point
    Keast rule.

Readings where the paper is silent:
  * Node order: corners 0..3, midsides 4:(0,1) 5:(1,2) 6:(0,2) 7:(0,3)
    8:(1,3) 9:(2,3).
  * Keast 5-point rule (degree 3): the centroid with weight -4/5 of the volume
    and the four points with barycentric coordinates (1/2, 1/6, 1/6, 1/6)
    (and permutations) with weight 9/20 of the volume each.
  * The mass matrix is integrated exactly (not with the 5-point rule, which
    makes the T10 consistent mass indefinite).
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial

import numpy as np

EDGES = ((0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3))

# Keast 5-point rule: barycentric coordinates (L0..L3) and weights as
# fractions of the element volume.
KEAST5_L = np.array([
    [0.25, 0.25, 0.25, 0.25],
    [0.5, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0],
    [1.0 / 6.0, 0.5, 1.0 / 6.0, 1.0 / 6.0],
    [1.0 / 6.0, 1.0 / 6.0, 0.5, 1.0 / 6.0],
    [1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 0.5],
])
KEAST5_WFRAC = np.array([-0.8, 0.45, 0.45, 0.45, 0.45])
# Parent tetrahedron {xi >= 0, xi1+xi2+xi3 <= 1} has volume 1/6.
KEAST5_W = KEAST5_WFRAC / 6.0
NQP = 5


def shape_values(L):
    """N_a at barycentric point L (4,): corners L_i(2L_i - 1), midsides 4 L_i L_j."""
    N = np.empty(10)
    for i in range(4):
        N[i] = L[i] * (2.0 * L[i] - 1.0)
    for m, (i, j) in enumerate(EDGES):
        N[4 + m] = 4.0 * L[i] * L[j]
    return N


def shape_dL(L):
    """dN_a/dL_c (10, 4) at barycentric point L, treating L0..L3 as independent."""
    D = np.zeros((10, 4))
    for i in range(4):
        D[i, i] = 4.0 * L[i] - 1.0
    for m, (i, j) in enumerate(EDGES):
        D[4 + m, i] = 4.0 * L[j]
        D[4 + m, j] = 4.0 * L[i]
    return D


# Parent coordinates xi = (L1, L2, L3), L0 = 1 - xi1 - xi2 - xi3.
DL_DXI = np.array([[-1.0, -1.0, -1.0],
                   [1.0, 0.0, 0.0],
                   [0.0, 1.0, 0.0],
                   [0.0, 0.0, 1.0]])


def shape_dxi(L):
    """dN_a/dxi (10, 3) by the chain rule through L(xi)."""
    return shape_dL(L) @ DL_DXI


def reference_geometry(X, conn):
    """Precomputed constants of Sec. 4.1 for every element and quadrature point.

    X: (nn, 3) reference coordinates; conn: (ne, 10).
    Returns gradN (ne, 5, 10, 3) = grad_X N_a at each qp, J0 (ne, 5) =
    det(dX/dxi) and wJ0 (ne, 5) = w_q * J0 with w_q the parent-domain weight.
    The isoparametric map X(xi) = sum_a N_a(xi) X_a is used as written, so
    curved (non-straight) elements are handled too.
    """
    Xe = X[conn]                                    # (ne, 10, 3)
    ne = conn.shape[0]
    gradN = np.empty((ne, NQP, 10, 3))
    J0 = np.empty((ne, NQP))
    for q in range(NQP):
        dNdxi = shape_dxi(KEAST5_L[q])              # (10, 3)
        # J_ij = dX_i/dxi_j = sum_a X_a,i dN_a/dxi_j
        J = np.einsum("eai,aj->eij", Xe, dNdxi)
        J0[:, q] = np.linalg.det(J)
        # grad_X N_a = J^{-T} dN_a/dxi
        Jinv = np.linalg.inv(J)
        gradN[:, q] = np.einsum("eji,aj->eai", Jinv, dNdxi)
    return gradN, J0, J0 * KEAST5_W[None, :]


# ---------------------------------------------------------------------------
# Exact consistent mass (Sec. 4.1, m_ij = int rho s_i s_j dV)
# ---------------------------------------------------------------------------

def _shape_polys():
    """Each N_a as a polynomial in (L0..L3): dict exponent-tuple -> Fraction."""
    polys = []
    for i in range(4):
        e2 = [0, 0, 0, 0]
        e2[i] = 2
        e1 = [0, 0, 0, 0]
        e1[i] = 1
        polys.append({tuple(e2): Fraction(2), tuple(e1): Fraction(-1)})
    for i, j in EDGES:
        e = [0, 0, 0, 0]
        e[i] += 1
        e[j] += 1
        polys.append({tuple(e): Fraction(4)})
    return polys


def _poly_mul(p, r):
    out = {}
    for ea, ca in p.items():
        for eb, cb in r.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            out[e] = out.get(e, Fraction(0)) + ca * cb
    return out


def barycentric_monomial_integral(alpha):
    """int_T L0^a0 L1^a1 L2^a2 L3^a3 dV / V = a0! a1! a2! a3! 3! / (|a| + 3)!."""
    num = 1
    for a in alpha:
        num *= factorial(a)
    return Fraction(num * factorial(3), factorial(sum(alpha) + 3))


def unit_mass_table():
    """10x10 table c_ab with m_ab = rho * V * c_ab (exact rationals)."""
    P = _shape_polys()
    C = [[Fraction(0)] * 10 for _ in range(10)]
    for a in range(10):
        for b in range(10):
            prod = _poly_mul(P[a], P[b])
            C[a][b] = sum((c * barycentric_monomial_integral(e) for e, c in prod.items()),
                          Fraction(0))
    return C


_UNIT_MASS = np.array([[float(c) for c in row] for row in unit_mass_table()])


def element_volumes(X, conn):
    """Volume of the corner tetrahedron of each element."""
    x0, x1, x2, x3 = (X[conn[:, i]] for i in range(4))
    return np.einsum("ei,ei->e", np.cross(x1 - x0, x2 - x0), x3 - x0) / 6.0


def element_mass(X, conn, rho):
    """(ne, 10, 10) scalar consistent mass m_ab of straight-sided T10 elements.

    rho: scalar or (ne,) density.  For straight-sided elements dV = 6V dxi,
    so m_ab = rho V c_ab with the exact table above.
    """
    V = element_volumes(X, conn)
    rho = np.broadcast_to(np.asarray(rho, dtype=np.float64), V.shape)
    return (rho * V)[:, None, None] * _UNIT_MASS[None, :, :]


def is_straight_sided(X, conn, rtol=1e-12):
    Xe = X[conn]
    scale = np.max(np.abs(Xe)) + 1.0
    for m, (i, j) in enumerate(EDGES):
        if np.max(np.abs(Xe[:, 4 + m] - 0.5 * (Xe[:, i] + Xe[:, j]))) > rtol * scale:
            return False
    return True
