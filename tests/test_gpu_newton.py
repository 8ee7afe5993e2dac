"""GPU Newton step (Algorithm 3 through tl_newton_step) against the oracle's
Newton step on the same inputs: converged, the oracle's residual at the GPU
velocity meets the tolerance, velocities and multipliers agree."""
import numpy as np
import pytest

from oracle import assembly as asm
from oracle import newton as nt
from paper_2604_10357_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _tl():
    from paper_2604_10357_gb300 import build, tl
    build.build()
    return tl


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(-1), device="cuda")


@pytest.fixture(scope="module")
def small_case():
    w = inputs.workload_small_svk()
    m = w["mesh"]
    om = asm.OracleMesh(m.X, m.conn, [w["material"]], fixed_nodes=m.fixed_nodes)
    prm = nt.NewtonParams(h=w["h"], rtol=1e-8, solver="dense")
    lam0 = np.zeros(3 * len(m.fixed_nodes))
    ref = nt.newton_step(om, w["q_n"].ravel(), w["v"].ravel(), lam0, prm)
    return w, om, prm, ref


@pytest.mark.parametrize("solver", ["direct", "pcg"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_newton_step_matches_oracle(small_case, prec, solver):
    tl = _tl()
    w, om, prm, ref = small_case
    m = w["mesh"]
    g = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP64 if prec == "fp64" else tl.TL_FP32_ELEM)
    g.build_pattern(m.fixed_nodes)
    lam = torch.zeros(3 * len(m.fixed_nodes), dtype=torch.float64, device="cuda")
    p = tl.params(h=prm.h, rho_alm=prm.rho_alm, rtol=prm.rtol, eps_out=prm.eps_out,
                  max_inner=prm.max_inner, max_outer=prm.max_outer,
                  linear_solver=tl.TL_SOLVER_PCG if solver == "pcg" else tl.TL_SOLVER_DIRECT)
    v, q, st = g.newton_step(p, _dev(w["q_n"]), _dev(w["v"]), lam)
    v = v.cpu().numpy()
    assert st["converged"] == 1
    assert abs(st["g_ref"] - ref["g_ref"]) <= 1e-10 * ref["g_ref"]
    assert st["g_norm"] <= 1e-8 * st["g_ref"]
    # validity by the oracle: its residual at the GPU's velocity (with the
    # multipliers of the last inner loop) is below the 1e-8 target
    lam_gpu = lam.cpu().numpy()
    lam_last_inner = lam_gpu - prm.rho_alm * om.constraint(w["q_n"].ravel() + prm.h * v)
    g_at_gpu = om.residual(v, w["q_n"].ravel(), w["v"].ravel(), prm.h, None, prm.gravity, lam_last_inner,
                           prm.rho_alm)
    assert np.linalg.norm(g_at_gpu) <= 1.05 * 1e-8 * ref["g_ref"]
    assert np.linalg.norm(v - ref["v"]) <= 1e-8 * np.linalg.norm(ref["v"])
    assert np.allclose(q.cpu().numpy(), w["q_n"].ravel() + prm.h * v, rtol=0, atol=1e-15)
    assert np.abs(lam_gpu - ref["lam"]).max() <= 1e-6 * np.abs(ref["lam"]).max()


def test_newton_free_fall_closed_form():
    """Unclamped, unstressed body at rest: one step gives v = h g exactly."""
    tl = _tl()
    m = inputs.box_t10(3, 2, 2, 0.3, 0.2, 0.2, fixed_face_x0=False)
    g = tl.Mesh(m.X, m.conn, [dict(inputs.SVK_1E7, eta_d=1e3, lambda_d=1e3)], precision=tl.TL_FP64)
    g.build_pattern(())
    p = tl.params(h=1e-3, rtol=1e-12, atol=1e-12)
    v, q, st = g.newton_step(p, _dev(m.X), _dev(np.zeros_like(m.X)), None)
    expect = np.tile(np.array([0.0, 0.0, -9.81e-3]), m.nn)
    assert np.abs(v.cpu().numpy() - expect).max() < 1e-11 * 9.81e-3


def test_newton_warm_start_reaches_same_state(small_case):
    """Starting from a better guess (the converged velocity perturbed) must
    converge to the same state with at most as many iterations."""
    tl = _tl()
    w, om, prm, ref = small_case
    m = w["mesh"]
    g = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP64)
    g.build_pattern(m.fixed_nodes)
    p = tl.params(h=prm.h, rho_alm=prm.rho_alm, rtol=prm.rtol, eps_out=prm.eps_out)
    lam = torch.zeros(3 * len(m.fixed_nodes), dtype=torch.float64, device="cuda")
    _, _, st0 = g.newton_step(p, _dev(w["q_n"]), _dev(w["v"]), lam)
    lam = torch.zeros_like(lam)
    guess = ref["v"] + 1e-6 * np.random.default_rng(3).normal(size=ref["v"].shape)
    v, _, st1 = g.newton_step(p, _dev(w["q_n"]), _dev(w["v"]), lam, v_init=_dev(guess))
    assert st1["converged"] == 1 and st1["inner_iters"] <= st0["inner_iters"]
    assert st1["g_ref"] == pytest.approx(st0["g_ref"], rel=1e-12)
    assert np.linalg.norm(v.cpu().numpy() - ref["v"]) <= 1e-8 * np.linalg.norm(ref["v"])
