"""Constitutive laws: first Piola-Kirchhoff stress P(F) and tangent A = dP/dF.

Paper passages: Sec. 4.3 Stage 1 (P = P_el(F) + P_vis(F, Fdot); St. Venant-
Kirchhoff or compressible Mooney-Rivlin, optional Kelvin-Voigt damping),
Sec. 4.4 Hessian assembly (the 4th-order material tangent A_{iJkL} and
eq. tangent_block).  The closed forms are in the companion Part I, not in this
paper; the readings used here:

  * SVK: E = (F^T F - I)/2, S = lambda tr(E) I + 2 mu E, P = F S, with
    lambda = E nu/((1+nu)(1-2nu)), mu = E/(2(1+nu)).
    A_{iJkL} = delta_ik S_JL + F_iM F_kN D_MJNL,
    D_MJNL = lambda d_MJ d_NL + mu (d_MN d_JL + d_ML d_JN).
  * Compressible Mooney-Rivlin:
    W = C10 (J^{-2/3} I1 - 3) + C01 (J^{-4/3} I2 - 3) + kappa/2 (J - 1)^2,
    I1 = tr C, I2 = (I1^2 - tr C^2)/2; P = dW/dF; A = dP/dF written out
    term by term (derivation in the comments of mr_tangent).
  * Kelvin-Voigt: Edot = sym(F^T Fdot), S_v = lambda_d tr(Edot) I + 2 eta_d Edot,
    P_v = F S_v; its velocity tangent dP_v/dFdot is returned by kv_tangent.

All functions take stacked arrays (..., 3, 3) and accept complex dtypes.
"""
from __future__ import annotations

import numpy as np

I3 = np.eye(3)


def lame(E, nu):
    return E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), E / (2.0 * (1.0 + nu))


def _tr(A):
    return np.einsum("...ii->...", A)


def _T(A):
    return np.swapaxes(A, -1, -2)


def det3(F):
    """Determinant by cofactor expansion (works for complex arrays)."""
    return (F[..., 0, 0] * (F[..., 1, 1] * F[..., 2, 2] - F[..., 1, 2] * F[..., 2, 1])
            - F[..., 0, 1] * (F[..., 1, 0] * F[..., 2, 2] - F[..., 1, 2] * F[..., 2, 0])
            + F[..., 0, 2] * (F[..., 1, 0] * F[..., 2, 1] - F[..., 1, 1] * F[..., 2, 0]))


def inv_T3(F):
    """F^{-T} via the cofactor matrix: F^{-T} = cof(F) / det F."""
    cof = np.empty_like(F)
    for i in range(3):
        for j in range(3):
            r = [x for x in range(3) if x != i]
            c = [x for x in range(3) if x != j]
            minor = (F[..., r[0], c[0]] * F[..., r[1], c[1]]
                     - F[..., r[0], c[1]] * F[..., r[1], c[0]])
            cof[..., i, j] = ((-1) ** (i + j)) * minor
    return cof / det3(F)[..., None, None]


# ---------------------------------------------------------------------------
# St. Venant-Kirchhoff
# ---------------------------------------------------------------------------

def svk_stress(F, lam, mu):
    """Returns (P, S) for SVK."""
    C = _T(F) @ F
    E = 0.5 * (C - I3)
    S = lam * _tr(E)[..., None, None] * I3 + 2.0 * mu * E
    return F @ S, S


def svk_elasticity(lam, mu):
    """D_MJNL = lambda d_MJ d_NL + mu (d_MN d_JL + d_ML d_JN)."""
    d = I3
    return (lam * np.einsum("MJ,NL->MJNL", d, d)
            + mu * (np.einsum("MN,JL->MJNL", d, d) + np.einsum("ML,JN->MJNL", d, d)))


def svk_tangent(F, S, lam, mu):
    """A_iJkL = delta_ik S_JL + F_iM F_kN D_MJNL."""
    D = svk_elasticity(lam, mu)
    geo = np.einsum("ik,...JL->...iJkL", I3, S)
    mat = np.einsum("...iM,...kN,MJNL->...iJkL", F, F, D)
    return geo + mat


# ---------------------------------------------------------------------------
# Compressible Mooney-Rivlin
# ---------------------------------------------------------------------------

def mr_stress(F, C10, C01, kappa):
    """P = dW/dF with W = C10(J^-2/3 I1 - 3) + C01(J^-4/3 I2 - 3) + kappa/2 (J-1)^2.

    dI1/dF = 2F, dI2/dF = 2(I1 F - F C), dJ/dF = J F^{-T}.
    """
    C = _T(F) @ F
    I1 = _tr(C)
    I2 = 0.5 * (I1 * I1 - _tr(C @ C))
    J = det3(F)
    G = inv_T3(F)
    Q = I1[..., None, None] * F - F @ C
    Jm23 = J ** (-2.0 / 3.0)
    Jm43 = J ** (-4.0 / 3.0)
    P = (C10 * Jm23[..., None, None] * (2.0 * F - (2.0 / 3.0) * I1[..., None, None] * G)
         + C01 * Jm43[..., None, None] * (2.0 * Q - (4.0 / 3.0) * I2[..., None, None] * G)
         + (kappa * (J - 1.0) * J)[..., None, None] * G)
    return P


def mr_tangent(F, C10, C01, kappa):
    """A_iJkL = dP_iJ / dF_kL for the Mooney-Rivlin stress above.

    Building blocks (G = F^{-T}, B = F F^T, Q = I1 F - F C):
      dG_iJ/dF_kL   = -G_iL G_kJ
      d(J^p)/dF_kL  = p J^p G_kL
      dI1/dF_kL     = 2 F_kL,   dI2/dF_kL = 2 Q_kL
      dQ_iJ/dF_kL   = 2 F_kL F_iJ + I1 d_ik d_JL - d_ik C_LJ - F_iL F_kJ - B_ik d_JL
    Term by term:
      C10 J^-2/3 [2 d_ik d_JL - 4/3 (F_iJ G_kL + G_iJ F_kL)
                  + 4/9 I1 G_iJ G_kL + 2/3 I1 G_iL G_kJ]
      C01 J^-4/3 [2 dQ_iJ/dF_kL - 8/3 (Q_iJ G_kL + G_iJ Q_kL)
                  + 16/9 I2 G_iJ G_kL + 4/3 I2 G_iL G_kJ]
      kappa [(2J^2 - J) G_iJ G_kL - (J^2 - J) G_iL G_kJ]
    """
    d = I3
    C = _T(F) @ F
    B = F @ _T(F)
    I1 = _tr(C)
    I2 = 0.5 * (I1 * I1 - _tr(C @ C))
    J = det3(F)
    G = inv_T3(F)
    Q = I1[..., None, None] * F - F @ C
    Jm23 = J ** (-2.0 / 3.0)
    Jm43 = J ** (-4.0 / 3.0)

    def outer(U, W):          # U_iJ W_kL
        return np.einsum("...iJ,...kL->...iJkL", U, W)

    def swap(U, W):           # U_iL W_kJ
        return np.einsum("...iL,...kJ->...iJkL", U, W)

    dd = np.einsum("ik,JL->iJkL", d, d)
    s = lambda x: x[..., None, None, None, None]   # noqa: E731

    dQ = (2.0 * outer(F, F) + s(I1) * dd
          - np.einsum("ik,...LJ->...iJkL", d, C)
          - swap(F, F)
          - np.einsum("...ik,JL->...iJkL", B, d))
    A10 = (2.0 * dd - (4.0 / 3.0) * (outer(F, G) + outer(G, F))
           + (4.0 / 9.0) * s(I1) * outer(G, G) + (2.0 / 3.0) * s(I1) * swap(G, G))
    A01 = (2.0 * dQ - (8.0 / 3.0) * (outer(Q, G) + outer(G, Q))
           + (16.0 / 9.0) * s(I2) * outer(G, G) + (4.0 / 3.0) * s(I2) * swap(G, G))
    Ak = s(2.0 * J * J - J) * outer(G, G) - s(J * J - J) * swap(G, G)
    return C10 * s(Jm23) * A10 + C01 * s(Jm43) * A01 + kappa * Ak


# ---------------------------------------------------------------------------
# Kelvin-Voigt viscous stress
# ---------------------------------------------------------------------------

def kv_stress(F, Fdot, eta, lam_d):
    """P_v = F S_v, S_v = lambda_d tr(Edot) I + 2 eta Edot, Edot = sym(F^T Fdot)."""
    Ed = 0.5 * (_T(F) @ Fdot + _T(Fdot) @ F)
    Sv = lam_d * _tr(Ed)[..., None, None] * I3 + 2.0 * eta * Ed
    return F @ Sv, Sv


def kv_tangent(F, eta, lam_d):
    """dP_v,iJ / dFdot_kL = lambda_d F_iJ F_kL + eta (B_ik d_JL + F_iL F_kJ)."""
    B = F @ _T(F)
    return (lam_d * np.einsum("...iJ,...kL->...iJkL", F, F)
            + eta * (np.einsum("...ik,JL->...iJkL", B, I3)
                     + np.einsum("...iL,...kJ->...iJkL", F, F)))


# ---------------------------------------------------------------------------
# Strain energies (the potentials the stresses above derive from)
# ---------------------------------------------------------------------------

def svk_energy(F, lam, mu):
    """W = lambda/2 (tr E)^2 + mu E:E."""
    E = 0.5 * (_T(F) @ F - I3)
    trE = _tr(E)
    return 0.5 * lam * trE * trE + mu * np.einsum("...ij,...ij->...", E, E)


def mr_energy(F, C10, C01, kappa):
    C = _T(F) @ F
    I1 = _tr(C)
    I2 = 0.5 * (I1 * I1 - _tr(C @ C))
    J = det3(F)
    return (C10 * (J ** (-2.0 / 3.0) * I1 - 3.0) + C01 * (J ** (-4.0 / 3.0) * I2 - 3.0)
            + 0.5 * kappa * (J - 1.0) ** 2)


def elastic_energy(F, mat):
    if mat["kind"] == "svk":
        lam, mu = lame(mat["E"], mat["nu"])
        return svk_energy(F, lam, mu)
    return mr_energy(F, mat["C10"], mat["C01"], mat["kappa"])


# ---------------------------------------------------------------------------
# Dispatch on a material description dict
# ---------------------------------------------------------------------------

def elastic_stress_and_tangent(F, mat, want_tangent=True):
    """Returns (P_el, S_el or None, A_el or None) for mat['kind'] in {'svk','mr'}."""
    if mat["kind"] == "svk":
        lam, mu = lame(mat["E"], mat["nu"])
        P, S = svk_stress(F, lam, mu)
        A = svk_tangent(F, S, lam, mu) if want_tangent else None
        return P, S, A
    if mat["kind"] == "mr":
        P = mr_stress(F, mat["C10"], mat["C01"], mat["kappa"])
        A = mr_tangent(F, mat["C10"], mat["C01"], mat["kappa"]) if want_tangent else None
        return P, None, A
    raise ValueError(mat["kind"])
