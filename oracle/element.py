"""Element internal force and tangent of T10 elements.

Paper passages:
  * eq. F_assembly (Sec. 4.3, Stage 1): F^(e,q) = sum_a x_a (x) grad_X N_a^(e,q);
    the rate Fdot = sum_a v_a (x) grad_X N_a (Sec. 4.1, same gradients).
  * P = P_el(F) + P_vis(F, Fdot) (Sec. 4.3, Stage 1).
  * eq. fint_local: f_a^(e) = sum_q P^(e,q) grad_X N_a^(e,q) J0^(e,q) w_q.
  * eq. tangent_block (Sec. 4.4): [K_ab]_de = sum_q A_dJeL (grad N_a)_J
    (grad N_b)_L J0 w_q, accumulated into the 30x30 K_elem, row r = 3a+d,
    column s = 3b+e.

Reading for Kelvin-Voigt (the paper's Hessian, eq. hessian, has no damping
term and Part I is not available): the Newton matrix uses
  h K_t + D,  K_t = sum_q wJ0 [delta_ik n_a.(S_el + S_v) n_b + n_a.(F D_el F) n_b],
  D = d f_int / d v at fixed q  (through Fdot),
i.e. the material part of d P_v / d F at fixed Fdot (not symmetric) is left
out, in the spirit of the paper's Gauss-Newton remark; the geometric part of
the viscous stress is kept.  For SVK this is exactly A_el with S_el replaced
by S_el + S_v in its geometric term.  For Mooney-Rivlin, whose tangent is not
split into S and F D F, the same geometric term delta_ik n_a.S_v n_b is added.
"""
from __future__ import annotations

import numpy as np

from . import materials as mats


def kinematics(x_e, gradN):
    """F_iJ = sum_a x_a,i dN_a/dX_J.  x_e (ne,10,3), gradN (ne,5,10,3) -> (ne,5,3,3)."""
    return np.einsum("eai,eqaJ->eqiJ", x_e, gradN)


def stresses(F, Fdot, mat, want_tangent):
    """Total P and the pieces of the tangent at every (e, q)."""
    P_el, S_el, A_el = mats.elastic_stress_and_tangent(F, mat, want_tangent)
    eta, lam_d = mat.get("eta_d", 0.0), mat.get("lambda_d", 0.0)
    has_kv = (eta != 0.0) or (lam_d != 0.0)
    if has_kv:
        P_v, S_v = mats.kv_stress(F, Fdot, eta, lam_d)
    else:
        P_v, S_v = np.zeros_like(P_el), None
    out = dict(P=P_el + P_v, P_el=P_el, P_v=P_v)
    if want_tangent:
        A = A_el
        if has_kv:
            A = A + np.einsum("ik,...JL->...iJkL", mats.I3, S_v)
            out["A_vis"] = mats.kv_tangent(F, eta, lam_d)
        else:
            out["A_vis"] = None
        out["A_t"] = A
    return out


def element_force(x_e, v_e, gradN, wJ0, mat):
    """f_e (ne, 10, 3) per eq. fint_local."""
    F = kinematics(x_e, gradN)
    Fdot = kinematics(v_e, gradN)
    P = stresses(F, Fdot, mat, want_tangent=False)["P"]
    return np.einsum("eqiJ,eqaJ,eq->eai", P, gradN, wJ0)


def element_energy(x_e, gradN, wJ0, mat):
    """Pi_e = sum_q wJ0 W(F_q): the hyperelastic potential whose gradient in x
    is the elastic part of eq. fint_local."""
    F = kinematics(x_e, gradN)
    return np.einsum("eq,eq->e", mats.elastic_energy(F, mat), wJ0)


def _tangent_blocks(A, gradN, wJ0):
    """K[e, a, i, b, k] = sum_q A_iJkL n_aJ n_bL wJ0 (eq. tangent_block)."""
    An = np.einsum("eqiJkL,eqaJ->eqaikL", A, gradN)
    return np.einsum("eqaikL,eqbL,eq->eaibk", An, gradN, wJ0, optimize=True)


def element_tangent(x_e, v_e, gradN, wJ0, mat, alpha=1.0, beta=0.0):
    """alpha * K_t,e + beta * D_e as (ne, 3 nen, 3 nen), row 3a+i, column 3b+k
    (nen = 10 for T10; the same contraction serves the ANCF elements)."""
    F = kinematics(x_e, gradN)
    Fdot = kinematics(v_e, gradN)
    st = stresses(F, Fdot, mat, want_tangent=True)
    ne, nen = x_e.shape[0], x_e.shape[1]
    K = alpha * _tangent_blocks(st["A_t"], gradN, wJ0)
    if beta != 0.0 and st["A_vis"] is not None:
        K = K + beta * _tangent_blocks(st["A_vis"], gradN, wJ0)
    return K.reshape(ne, 3 * nen, 3 * nen)


def element_force_and_tangent(x_e, v_e, gradN, wJ0, mat, alpha=1.0, beta=0.0):
    return (element_force(x_e, v_e, gradN, wJ0, mat),
            element_tangent(x_e, v_e, gradN, wJ0, mat, alpha, beta))
