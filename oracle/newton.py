"""One backward-Euler time step by Newton's method inside the ALM loop.

Paper passages: eq. stepmap (q = q_n + h v), eq. residual, eq. hessian,
eq. newton_linear_system (H p = -g), eq. lambda_update, Algorithm 1 (ALM) and
Algorithm 3 (one time step with the Newton solver); eq. armijo for the
optional backtracking line search (c1 = 1e-4, beta = 0.5, j_max = 10).

Readings (the paper leaves these open for the T10 benchmarks):
  * inner stop: ||g|| <= max(atol, rtol * g_ref), where g_ref is the residual
    norm at the plain start v = v_n with the step's initial lambda, whatever
    start is used (so a better warm start does not tighten the target);
  * lambda persists across steps (initialised to zero once, Algorithm 1);
  * the linear system is solved by a sparse direct solver (the step the paper
    delegates to cuDSS); here scipy's SuperLU, or a dense Cholesky on request.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla


@dataclass
class NewtonParams:
    h: float = 1e-3
    rho_alm: float = 1e12
    rtol: float = 1e-8
    atol: float = 0.0
    eps_out: float = 1e-4
    max_inner: int = 20
    max_outer: int = 5
    gravity: tuple = (0.0, 0.0, -9.81)
    line_search: bool = False
    c1: float = 1e-4
    beta: float = 0.5
    j_max: int = 10
    solver: str = "splu"      # "splu" or "dense"


def _solve(Hm, rhs, solver):
    if solver == "dense":
        c = sla.cho_factor(Hm.toarray(), lower=True)
        return sla.cho_solve(c, rhs)
    return spla.spsolve(Hm.tocsc(), rhs)


def newton_step(om, q_n, v_n, lam, prm: NewtonParams, f_ext=None, v_start=None):
    """Algorithm 3 for one time step.

    om: OracleMesh; q_n, v_n: (3nn,); lam: (3*nfixed,) multipliers (returned
    updated, not modified in place); v_start: initial velocity (default v_n).
    Returns dict(v, q, lam, inner_iters, outer_iters, g_ref, g_norm, history).
    """
    q_n = np.asarray(q_n, dtype=np.float64).reshape(-1)
    v_n = np.asarray(v_n, dtype=np.float64).reshape(-1)
    lam = np.array(lam, dtype=np.float64).reshape(-1)
    M = om.mass_matrix()
    h = prm.h

    def g_of(v, lam_):
        return om.residual(v, q_n, v_n, h, f_ext, prm.gravity, lam_, prm.rho_alm, M=M)

    v = (v_n.copy() if v_start is None else np.asarray(v_start, dtype=np.float64).reshape(-1).copy())
    g_ref = float(np.linalg.norm(g_of(v_n, lam)))
    target = max(prm.atol, prm.rtol * g_ref)
    history = []
    total_inner = 0
    outer = 0
    converged = False
    for outer in range(1, prm.max_outer + 1):           # ALM outer loop
        inner_ok = False
        for _l in range(prm.max_inner):                  # Newton inner loop
            g = g_of(v, lam)
            gn = float(np.linalg.norm(g))
            history.append(gn)
            if gn <= target:
                inner_ok = True
                break
            Hm = om.hessian_matrix(q_n, v, h, prm.rho_alm)
            dv = _solve(Hm, -g, prm.solver)              # H dv = -g
            total_inner += 1
            if prm.line_search:                          # eq. armijo
                phi0 = 0.5 * gn * gn
                alpha, accepted = 1.0, False
                for _j in range(prm.j_max):
                    vt = v + alpha * dv
                    gt = g_of(vt, lam)
                    if 0.5 * float(gt @ gt) <= (1.0 - 2.0 * prm.c1 * alpha) * phi0:
                        v, accepted = vt, True
                        break
                    alpha *= prm.beta
                if not accepted:
                    break
            else:
                v = v + dv
        c = om.constraint(q_n + h * v)
        if inner_ok and len(c):
            lam = lam + prm.rho_alm * c                  # eq. lambda_update
        cn = float(np.linalg.norm(c)) if len(c) else 0.0
        if inner_ok and cn <= prm.eps_out:
            converged = True
            break
    # g_norm: the last inner-loop residual (before the final multiplier update)
    return dict(v=v, q=q_n + h * v, lam=lam, inner_iters=total_inner, outer_iters=outer,
                g_ref=g_ref, g_norm=history[-1], target=target, converged=converged,
                history=history)
