"""Pins of the oracle's AdamW time step (Algorithm 2) against what the
algorithm and the mathematics fix: the bias-corrected update under a constant
gradient (closed form), the weight-decay-only first update of every outer
iteration, and that the iteration solves the same nonlinear system as Newton's
method (it approaches the Newton step's velocity)."""
import numpy as np

from oracle import adamw as aw
from oracle import assembly as asm
from oracle import newton as nt
from paper_2604_10357_gb300 import inputs


def test_update_under_constant_gradient_closed_form():
    """With g constant from the first update on, the bias corrections make
    m_hat = g and s_hat = g^2 exactly at every l, so each update moves v by
    -lr g / (|g| + eps) (times the weight decay factor)."""
    prm = aw.AdamWParams(lr=0.01, weight_decay=0.5, eps=1e-8)
    g = np.array([3.0, -0.25, 1e-3, -7.0])
    v = np.array([1.0, -2.0, 0.5, 0.0])
    m = np.zeros(4)
    s = np.zeros(4)
    ref = v.copy()
    for l in range(1, 30):
        v, m, s = aw.adamw_update(v, m, s, g, l, prm)
        ref = (1.0 - prm.lr * prm.weight_decay) * ref - prm.lr * g / (np.abs(g) + prm.eps)
        np.testing.assert_allclose(m / (1 - prm.beta1 ** l), g, rtol=1e-13)
        np.testing.assert_allclose(s / (1 - prm.beta2 ** l), g * g, rtol=1e-12)
        np.testing.assert_allclose(v, ref, rtol=1e-12, atol=1e-15)


def _free_body(perturbed):
    m = inputs.box_t10(3, 2, 2, 0.3, 0.2, 0.2, fixed_face_x0=False)
    om = asm.OracleMesh(m.X, m.conn, [dict(inputs.SVK_1E7)], fixed_nodes=[])
    rng = np.random.default_rng(3)
    q = m.X.ravel() + (1e-4 * rng.normal(size=3 * m.nn) if perturbed else 0.0)
    v = 0.01 * rng.normal(size=3 * m.nn) if perturbed else np.zeros(3 * m.nn)
    return om, q, v


def test_first_update_of_an_outer_iteration_is_weight_decay_only():
    """The gradient and the moments are reset at every outer iteration, so the
    first inner update only scales v by (1 - lr wd)."""
    om, q, v = _free_body(True)
    prm = aw.AdamWParams(h=1e-3, lr=1e-3, weight_decay=0.3, max_inner=1, max_outer=1)
    r = aw.adamw_step(om, q, v, np.zeros(0), prm)
    np.testing.assert_allclose(r["v"], (1.0 - 1e-3 * 0.3) * v, rtol=1e-15, atol=0)
    assert r["inner_iters"] == 1 and not r["converged"]


def test_approaches_the_newton_step():
    """Free fall of an unclamped, unstressed box from rest: AdamW drives the
    gradient of the same augmented cost towards zero, so its velocity
    approaches the Newton step's (v = h g here, the closed form) to a small
    fraction after 2,000 updates."""
    om, q, v = _free_body(False)
    ref = nt.newton_step(om, q, v, np.zeros(0), nt.NewtonParams(h=1e-3, rtol=1e-12, solver="dense"))
    np.testing.assert_allclose(ref["v"].reshape(-1, 3), np.tile([0.0, 0.0, -9.81e-3], (len(v) // 3, 1)),
                               atol=1e-12)
    r = aw.adamw_step(om, q, v, np.zeros(0), aw.AdamWParams(h=1e-3, lr=1e-4, max_inner=2000, max_outer=1,
                                                            eps_in=0.0, eps_rel=0.0))
    assert np.linalg.norm(r["v"] - ref["v"]) <= 1e-3 * np.linalg.norm(ref["v"])
    assert r["history"][-1] < 1e-3 * r["history"][0]
