"""ANCF3243 beam and ANCF3443 shell elements for the Total-Lagrangian path:
shape functions, Gauss-Legendre rules, reference geometry, consistent mass,
and a mesh class on the same force / Hessian / residual assembly as T10.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper passages:
  * Sec. 2: q collects positions and, for ANCF elements, position gradients;
    the residual, Hessian, ALM and Newton step are those of the T10 path
    taken over coefficient indices (Sec. 4.3: n_dof = 3 n_coef).
  * Sec. 4.3, Stage 1: 12 quadrature points per beam element (3 x 2 x 2
    Gauss-Legendre product rule) and 48 per shell element (4 x 4 x 3);
    F = sum_a e_a (x) grad_X S_a (eq. F_assembly with the coefficient vectors
    e_a in place of nodal positions); 8 shape functions per beam element and
    16 per shell element (four coefficient vectors per physical node).
  * Sec. 4.4: 24 x 24 and 48 x 48 element tangents from eq. tangent_block.
  * Sec. 4.1: m_ij = int rho S_i S_j dV, constant; grad_X S from the
    isoparametric Jacobian of the reference configuration.

Readings (the paper takes the element definitions from its references):
  * Beam (ANCF3243), element length L, width W, height H, natural
    coordinates xi, eta, zeta in [-1, 1], local x = L (1 + xi)/2,
    y = W eta / 2, z = H zeta / 2.  Coefficients per node: r, r_x, r_y,
    r_z.  Along the axis the position is the cubic Hermite interpolant of
    the end positions and axial slopes; the transverse gradients enter as
    y r_y + z r_z, interpolated linearly between the two ends.
  * Shell (ANCF3443), element size L x W, thickness H, local
    x = L (1 + xi)/2, y = W (1 + eta)/2, z = H zeta / 2; corners in the
    order (-1,-1), (1,-1), (1,1), (-1,1), each with r, r_x, r_y, r_z.  The
    mid-surface field lies in the 12-term incomplete bicubic space spanned by
    1, xi, eta, xi^2, xi eta, eta^2, xi^3, xi^2 eta, xi eta^2, eta^3,
    xi^3 eta, xi eta^3 and interpolates r, r_x, r_y at the corners; the
    thickness direction adds z times the bilinear interpolant of r_z.
  * Both spaces are fixed here by their interpolation conditions: the
    shape functions are the columns of the inverse of the conditions
    matrix over the monomial basis (the definition, not a closed form).
  * Mass: integrated exactly for straight, rectangular elements (4 Gauss
    points along each cubic direction, 2 along each linear one), the same
    choice as for T10, where the element rule does not integrate it exactly.
  * Gravity: f_ff,a = g int rho S_a dV.  The T10 shortcut (row sums of M)
    relies on sum_a N_a = 1, which the gradient shape functions break.
  * Clamps act on whole coefficients: c = e - e0 on each fixed coefficient
    (position and gradient vectors of a clamped physical node).
"""
from __future__ import annotations

import functools

import numpy as np

from .assembly import OracleMesh

BEAM = "ancf3243"
SHELL = "ancf3443"


# ---------------------------------------------------------------------------
# Gauss-Legendre rules (Sec. 4.3)
# ---------------------------------------------------------------------------

def gauss_legendre(n):
    """n-point Gauss-Legendre abscissae and weights on [-1, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w


def product_rule(n1, n2, n3):
    """Tensor-product rule: points (n1 n2 n3, 3) with xi slowest, zeta fastest,
    and weights (n1 n2 n3,)."""
    x1, w1 = gauss_legendre(n1)
    x2, w2 = gauss_legendre(n2)
    x3, w3 = gauss_legendre(n3)
    pts = np.array([(a, b, c) for a in x1 for b in x2 for c in x3])
    wts = np.array([wa * wb * wc for wa in w1 for wb in w2 for wc in w3])
    return pts, wts


def element_rule(kind):
    """The paper's element rule: 3 x 2 x 2 for the beam, 4 x 4 x 3 for the shell."""
    return product_rule(3, 2, 2) if kind == BEAM else product_rule(4, 4, 3)


def mass_rule(kind):
    """A rule exact for S_a S_b of a straight, rectangular element."""
    return product_rule(4, 2, 2) if kind == BEAM else product_rule(4, 4, 2)


def nen_of(kind):
    return 8 if kind == BEAM else 16


# ---------------------------------------------------------------------------
# Shape functions from their interpolation conditions
# ---------------------------------------------------------------------------

@functools.lru_cache(maxsize=64)
def _beam_axis_coefficients(L):
    """Coefficients (4, 4) of the cubic Hermite basis in 1, xi, xi^2, xi^3:
    column j is the polynomial whose value / x-slope at xi = -1 / +1 is the
    unit vector e_j, with the conditions ordered (value A, slope A, value B,
    slope B) and d/dx = (2 / L) d/dxi."""
    V = np.zeros((4, 4))
    for row, (xi, deriv) in enumerate([(-1.0, 0), (-1.0, 1), (1.0, 0), (1.0, 1)]):
        for k in range(4):
            V[row, k] = xi ** k if deriv == 0 else (2.0 / L) * k * xi ** (k - 1) if k else 0.0
    return np.linalg.inv(V)


_SHELL_MONOMIALS = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (3, 0), (2, 1), (1, 2), (0, 3),
                    (3, 1), (1, 3)]
SHELL_CORNERS = [(-1.0, -1.0), (1.0, -1.0), (1.0, 1.0), (-1.0, 1.0)]


def _mono(p, k, x):
    """d^k/dx^k of x^p."""
    if p < k:
        return 0.0 * x
    c = 1.0
    for j in range(k):
        c *= p - j
    return c * x ** (p - k)


@functools.lru_cache(maxsize=64)
def _shell_surface_coefficients(L, W):
    """Coefficients (12, 12) over the incomplete bicubic monomials: column j is
    the member of the space whose (value, x-slope, y-slope) at the four
    corners is the unit vector e_j, conditions ordered corner by corner."""
    V = np.zeros((12, 12))
    row = 0
    for (xc, yc) in SHELL_CORNERS:
        for kind in range(3):
            for k, (p, q) in enumerate(_SHELL_MONOMIALS):
                if kind == 0:
                    V[row, k] = _mono(p, 0, xc) * _mono(q, 0, yc)
                elif kind == 1:
                    V[row, k] = (2.0 / L) * _mono(p, 1, xc) * _mono(q, 0, yc)
                else:
                    V[row, k] = (2.0 / W) * _mono(p, 0, xc) * _mono(q, 1, yc)
            row += 1
    return np.linalg.inv(V)


def beam_shape(pt, dims):
    """S (8,) and dS/d(xi, eta, zeta) (8, 3) of the beam at pt = (xi, eta, zeta)."""
    L, W, H = dims
    xi, eta, zeta = pt
    Cax = _beam_axis_coefficients(L)                 # (4 powers, 4 conditions)
    pw = np.array([_mono(k, 0, xi) for k in range(4)])
    dpw = np.array([_mono(k, 1, xi) for k in range(4)])
    hA, hAx, hB, hBx = pw @ Cax
    dA, dAx, dB, dBx = dpw @ Cax
    y, z = 0.5 * W * eta, 0.5 * H * zeta
    lA, lB = 0.5 * (1.0 - xi), 0.5 * (1.0 + xi)      # linear interpolation along the axis
    S = np.array([hA, hAx, lA * y, lA * z, hB, hBx, lB * y, lB * z])
    dS = np.zeros((8, 3), dtype=np.result_type(xi, eta, zeta, float))
    dS[:, 0] = [dA, dAx, -0.5 * y, -0.5 * z, dB, dBx, 0.5 * y, 0.5 * z]
    dS[:, 1] = [0.0, 0.0, lA * 0.5 * W, 0.0, 0.0, 0.0, lB * 0.5 * W, 0.0]
    dS[:, 2] = [0.0, 0.0, 0.0, lA * 0.5 * H, 0.0, 0.0, 0.0, lB * 0.5 * H]
    return S, dS


def shell_shape(pt, dims):
    """S (16,) and dS/d(xi, eta, zeta) (16, 3) of the shell at pt."""
    L, W, H = dims
    xi, eta, zeta = pt
    C = _shell_surface_coefficients(L, W)            # (12 monomials, 12 conditions)
    m = np.array([_mono(p, 0, xi) * _mono(q, 0, eta) for p, q in _SHELL_MONOMIALS])
    mx = np.array([_mono(p, 1, xi) * _mono(q, 0, eta) for p, q in _SHELL_MONOMIALS])
    my = np.array([_mono(p, 0, xi) * _mono(q, 1, eta) for p, q in _SHELL_MONOMIALS])
    s, sx, sy = m @ C, mx @ C, my @ C                # (12,) surface functions, condition order
    z = 0.5 * H * zeta
    S = np.zeros(16, dtype=np.result_type(xi, eta, zeta, float))
    dS = np.zeros((16, 3), dtype=S.dtype)
    for c, (xc, yc) in enumerate(SHELL_CORNERS):
        bl = 0.25 * (1.0 + xc * xi) * (1.0 + yc * eta)           # bilinear corner function
        for j in range(3):                                       # r, r_x, r_y
            S[4 * c + j] = s[3 * c + j]
            dS[4 * c + j] = [sx[3 * c + j], sy[3 * c + j], 0.0]
        S[4 * c + 3] = z * bl
        dS[4 * c + 3] = [z * 0.25 * xc * (1.0 + yc * eta), z * 0.25 * yc * (1.0 + xc * xi), 0.5 * H * bl]
    return S, dS


def shape(kind, pt, dims):
    return beam_shape(pt, dims) if kind == BEAM else shell_shape(pt, dims)


# ---------------------------------------------------------------------------
# Reference geometry and mass (Sec. 4.1)
# ---------------------------------------------------------------------------

def reference_geometry(kind, e0, conn, dims):
    """grad_X S (ne, nqp, nen, 3), det J0 (ne, nqp), w_q det J0 (ne, nqp) at the
    element rule, with J0 = d r0 / d(xi, eta, zeta), r0 = sum_a S_a e0_a."""
    pts, wts = element_rule(kind)
    ne, nen = conn.shape
    gradS = np.zeros((ne, len(pts), nen, 3))
    detJ = np.zeros((ne, len(pts)))
    for e in range(ne):
        E0 = e0[conn[e]]                                   # (nen, 3)
        for q, pt in enumerate(pts):
            _, dS = shape(kind, pt, dims[e])
            J0 = E0.T @ dS                                 # J0[i, j] = sum_a e0_a,i dS_a/dxi_j
            detJ[e, q] = np.linalg.det(J0)
            gradS[e, q] = dS @ np.linalg.inv(J0)           # dS_a/dX_J = sum_j dS_a/dxi_j (J0^-1)_jJ
    return gradS, detJ, detJ * wts[None, :]


def element_mass(kind, e0, conn, dims, rho):
    """(ne, nen, nen) scalar consistent mass m_ab = int rho S_a S_b dV and the
    (ne, nen) gravity weights int rho S_a dV, by the mass rule."""
    pts, wts = mass_rule(kind)
    ne, nen = conn.shape
    Me = np.zeros((ne, nen, nen))
    We = np.zeros((ne, nen))
    for e in range(ne):
        E0 = e0[conn[e]]
        for pt, w in zip(pts, wts):
            S, dS = shape(kind, pt, dims[e])
            dv = w * np.linalg.det(E0.T @ dS)
            Me[e] += rho[e] * dv * np.outer(S, S)
            We[e] += rho[e] * dv * S
    return Me, We


class OracleAncfMesh(OracleMesh):
    """An ANCF mesh: X holds the reference coefficient vectors e0 (ncoef, 3),
    conn the coefficient indices of each element (ne, nen), dims the (L, W, H)
    of each element; fixed_nodes lists clamped coefficients."""

    def __init__(self, kind, e0, conn, dims, materials, mat_of_elem=None, fixed_nodes=(), constraints=None):
        self.kind = kind
        self.dims = np.asarray(dims, dtype=np.float64).reshape(-1, 3)
        super().__init__(e0, conn, materials, mat_of_elem, fixed_nodes, constraints)

    def _reference(self, rho):
        self.gradN, self.J0, self.wJ0 = reference_geometry(self.kind, self.X, self.conn, self.dims)
        self.Me, self.We = element_mass(self.kind, self.X, self.conn, self.dims, rho)

    def gravity_force(self, gravity):
        """f_ff,I = g sum over elements of int rho S_a dV at the coefficient's slot."""
        w = np.zeros(self.nn)
        np.add.at(w, self.conn.ravel(), self.We.ravel())
        return (w[:, None] * np.asarray(gravity)[None, :]).ravel()
