"""One backward-Euler time step with the first-order AdamW inner solver.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper passages: Algorithm 2 (one time step: AdamW solver) inside the ALM
outer loop of Algorithm 1; eq. stepmap (q = q_n + h v), eq. residual / eq.
grad_L (the gradient g), eq. lambda_update.  The inner loop follows the
printed order: moment updates from the previous gradient, bias correction,
velocity update with decoupled weight decay, step map, then the new gradient
and its norm; the moments and the gradient are reset to zero at the start of
every outer iteration, so the first inner update applies only the weight
decay.

Readings (the paper leaves these open):
  * the hyperparameters (step size alpha, beta1, beta2, epsilon, weight decay)
    are not printed: they are inputs here (defaults beta1 = 0.9,
    beta2 = 0.999, epsilon = 1e-8, weight decay 0, constant alpha);
  * the inner test |g| <= eps_in (1 + |v|) or |g| <= eps_rel |g_0| is made
    every `check_every` iterations (the paper's "prescribed check interval";
    g_0 is the first gradient of the outer iteration), with the paper's
    tolerance-table values eps_in = 1e-4, eps_rel = 1e-6 as defaults;
  * after the inner loop the algorithm commits v_n <- v, so later outer
    iterations measure the inertia term from the committed velocity; the
    step returns that committed velocity.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class AdamWParams:
    h: float = 1e-3
    rho_alm: float = 1e12
    eps_out: float = 1e-4
    max_outer: int = 5
    max_inner: int = 1000
    check_every: int = 10
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    weight_decay: float = 0.0
    eps_in: float = 1e-4
    eps_rel: float = 1e-6
    gravity: tuple = (0.0, 0.0, -9.81)


def adamw_update(v, m, s, g, l, prm: AdamWParams):
    """One AdamW update of Algorithm 2 at inner iteration l (1-based):
    moments from the gradient g, bias correction, decoupled weight decay.
    Returns the new (v, m, s)."""
    m = prm.beta1 * m + (1.0 - prm.beta1) * g
    s = prm.beta2 * s + (1.0 - prm.beta2) * g * g
    m_hat = m / (1.0 - prm.beta1 ** l)
    s_hat = s / (1.0 - prm.beta2 ** l)
    v = (1.0 - prm.lr * prm.weight_decay) * v - prm.lr * m_hat / (np.sqrt(s_hat) + prm.eps)
    return v, m, s


def adamw_step(om, q_n, v_n, lam, prm: AdamWParams, f_ext=None, v_start=None):
    """Algorithm 2 for one time step.

    om: OracleMesh; q_n, v_n: (3nn,); lam: (3*nfixed,) multipliers (returned
    updated).  Returns dict(v, q, lam, inner_iters, outer_iters, converged,
    g_norm, c_norm, history)."""
    q_n = np.asarray(q_n, dtype=np.float64).reshape(-1)
    v_n = np.asarray(v_n, dtype=np.float64).reshape(-1).copy()
    lam = np.array(lam, dtype=np.float64).reshape(-1)
    M = om.mass_matrix()
    h = prm.h
    v = v_n.copy() if v_start is None else np.asarray(v_start, dtype=np.float64).reshape(-1).copy()
    history = []
    total_inner = 0
    converged = False
    gn = cn = 0.0
    outer = 0
    for outer in range(1, prm.max_outer + 1):            # ALM outer loop
        g = np.zeros_like(v)
        m = np.zeros_like(v)
        s = np.zeros_like(v)
        g0 = None
        inner_ok = False
        for l in range(1, prm.max_inner + 1):            # AdamW inner loop
            v, m, s = adamw_update(v, m, s, g, l, prm)
            g = om.residual(v, q_n, v_n, h, f_ext, prm.gravity, lam, prm.rho_alm, M=M)
            gn = float(np.linalg.norm(g))
            history.append(gn)
            total_inner += 1
            if g0 is None:
                g0 = gn
            if l % prm.check_every == 0 and (gn <= prm.eps_in * (1.0 + float(np.linalg.norm(v)))
                                             or gn <= prm.eps_rel * g0):
                inner_ok = True
                break
        v_n = v.copy()                                    # commit the velocity
        c = om.constraint(q_n + h * v)
        if len(c):
            lam = lam + prm.rho_alm * c                  # eq. lambda_update
        cn = float(np.linalg.norm(c)) if len(c) else 0.0
        if inner_ok and cn <= prm.eps_out:
            converged = True
            break
    return dict(v=v_n, q=q_n + h * v_n, lam=lam, inner_iters=total_inner, outer_iters=outer,
                converged=converged, g_norm=gn, c_norm=cn, history=history)
