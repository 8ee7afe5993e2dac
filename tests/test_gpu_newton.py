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


@pytest.mark.parametrize("solver", ["direct", "pcg", "pcg_graph"])
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
                  linear_solver=tl.TL_SOLVER_DIRECT if solver == "direct" else tl.TL_SOLVER_PCG,
                  use_graph=1 if solver == "pcg_graph" else 0)
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


@pytest.fixture(scope="module")
def line_search_case():
    """The 240-element SVK box with h = 1e-2: the full Newton step overshoots
    (the residual grows at the fourth iteration), so the Armijo backtracking
    of eq. armijo shortens steps before the step converges."""
    w = inputs.workload_small_svk()
    m = w["mesh"]
    om = asm.OracleMesh(m.X, m.conn, [w["material"]], fixed_nodes=m.fixed_nodes)
    prm = nt.NewtonParams(h=1e-2, rtol=1e-8, solver="dense", line_search=True)
    lam0 = np.zeros(3 * len(m.fixed_nodes))
    ref = nt.newton_step(om, w["q_n"].ravel(), w["v"].ravel(), lam0, prm)
    assert ref["converged"]
    return w, om, prm, ref


@pytest.mark.parametrize("solver", ["direct", "pcg", "pcg_graph"])
def test_newton_line_search_matches_oracle(line_search_case, solver):
    """Line search on: the same converged step as the oracle's Newton step with
    the same backtracking rule (c1 = 1e-4, beta = 0.5, 10 trials), the same
    Newton count, and more trial points than Newton steps (some steps were
    shortened)."""
    tl = _tl()
    w, om, prm, ref = line_search_case
    m = w["mesh"]
    g = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP64)
    g.build_pattern(m.fixed_nodes)
    lam = torch.zeros(3 * len(m.fixed_nodes), dtype=torch.float64, device="cuda")
    p = tl.params(h=prm.h, rho_alm=prm.rho_alm, rtol=prm.rtol, eps_out=prm.eps_out, line_search=1,
                  linear_solver=tl.TL_SOLVER_DIRECT if solver == "direct" else tl.TL_SOLVER_PCG,
                  use_graph=1 if solver == "pcg_graph" else 0)
    v, q, st = g.newton_step(p, _dev(w["q_n"]), _dev(w["v"]), lam)
    v = v.cpu().numpy()
    assert st["converged"] == 1
    assert st["inner_iters"] == ref["inner_iters"]
    assert st["ls_trials"] > st["inner_iters"]
    assert np.linalg.norm(v - ref["v"]) <= 1e-8 * np.linalg.norm(ref["v"])
    assert abs(st["g_ref"] - ref["g_ref"]) <= 1e-10 * ref["g_ref"]


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


def _run_pair(tl, g, w, prm_kw, nsteps=3, v_init_fn=None):
    """The same steps through the host-driven loop and the captured graph."""
    m = w["mesh"]
    out = {}
    for use_graph in (0, 1):
        p = tl.params(linear_solver=tl.TL_SOLVER_PCG, use_graph=use_graph, **prm_kw)
        q = _dev(w["q_n"])
        v = _dev(w["v"])
        lam = torch.zeros(3 * len(m.fixed_nodes), dtype=torch.float64, device="cuda")
        fe = _dev(0.5 * np.random.default_rng(7).normal(size=m.X.shape))
        hist = []
        for k in range(nsteps):
            vi = v_init_fn(v) if v_init_fn else None
            v_new, q_new, st = g.newton_step(p, q, v, lam, v_init=vi, f_ext=fe)
            hist.append(st)
            q, v = q_new.clone(), v_new.clone()
        out[use_graph] = (v.cpu().numpy(), q.cpu().numpy(), lam.cpu().numpy(), hist)
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("adaptive", [0, 1])
def test_newton_graph_equals_host_loop(prec, adaptive):
    """The captured step runs the same kernels with the same arguments in the
    same order, and makes the same tests on the device: the same Newton and
    ALM iteration counts, PCG counts within one check interval per solve, and
    the same converged velocities and multipliers over several steps (with a
    start different from v_n and an external force).  The scatter uses
    atomics, so two runs of either path agree to rounding, not bit for bit."""
    tl = _tl()
    if prec == "fp32":
        # the 15,360-element MR + KV mesh at a mild state (0.25% sine-mode
        # amplitude): at the full 5% state H is indefinite and a plain
        # Newton step inverts elements
        w = inputs.workload_mid_mr_kv()
        X = w["mesh"].X
        w = dict(w, q_n=X + 0.05 * (w["q_n"] - X), v=0.2 * w["v"])
    else:
        w = inputs.workload_small_svk()
    m = w["mesh"]
    g = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP64 if prec == "fp64" else tl.TL_FP32_ELEM)
    g.build_pattern(m.fixed_nodes)
    res = _run_pair(tl, g, w, dict(h=w["h"], rtol=1e-8, lin_adaptive=adaptive),
                    v_init_fn=lambda v: 1.01 * v)
    (v0, q0, l0, h0), (v1, q1, l1, h1) = res[0], res[1]
    for a, b in zip(h0, h1):
        for key in ("inner_iters", "outer_iters", "converged", "status"):
            assert a[key] == b[key], (key, a, b)
        assert abs(a["lin_iters"] - b["lin_iters"]) <= 8 * a["inner_iters"], (a, b)
        assert b["g_ref"] == pytest.approx(a["g_ref"], rel=1e-9)
        assert b["g_init"] == pytest.approx(a["g_init"], rel=1e-6)
        assert b["g_norm"] <= 1e-8 * b["g_ref"] and b["converged"] == 1
    assert np.linalg.norm(v1 - v0) <= 1e-8 * np.linalg.norm(v0)
    assert np.linalg.norm(q1 - q0) <= 1e-12 * np.linalg.norm(q0)
    assert np.abs(l1 - l0).max() <= 1e-6 * np.abs(l0).max()


@pytest.mark.parametrize("use_graph", [0, 1])
def test_pcg_vector_precisions_reach_same_state(use_graph):
    """With a float32 Hessian the PCG vectors may be float32 (dot products in
    float64) or float64: each Newton solve is inexact either way, and both
    converge the float64 residual to 1e-8, so the velocities agree to the
    residual's tolerance and the Newton counts are the same."""
    tl = _tl()
    w = inputs.workload_mid_mr_kv()
    X = w["mesh"].X
    w = dict(w, q_n=X + 0.05 * (w["q_n"] - X), v=0.2 * w["v"])
    m = w["mesh"]
    g = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP32_ELEM)
    g.build_pattern(m.fixed_nodes)
    p = tl.params(h=w["h"], rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG, lin_adaptive=1, use_graph=use_graph)
    out = {}
    for f32 in (0, 1):
        g.tune_set(pcg_f32=f32)
        assert g.tune_get()["pcg_f32"] == f32
        lam = torch.zeros(3 * len(m.fixed_nodes), dtype=torch.float64, device="cuda")
        v, _, st = g.newton_step(p, _dev(w["q_n"]), _dev(w["v"]), lam)
        assert st["converged"] == 1 and st["g_norm"] <= 1e-8 * st["g_ref"]
        out[f32] = (v.cpu().numpy(), st)
    (v0, s0), (v1, s1) = out[0], out[1]
    assert s1["outer_iters"] == s0["outer_iters"]
    assert abs(s1["inner_iters"] - s0["inner_iters"]) <= 1
    assert np.linalg.norm(v1 - v0) <= 1e-7 * np.linalg.norm(v0)


def test_double_float_residual_force_reaches_same_state():
    """Float32 handle: the Newton residual's internal force in float64 and in
    double-float arithmetic give the same converged step (the residual's
    tolerance), with the same Newton counts."""
    tl = _tl()
    w = inputs.workload_small_svk()
    m = w["mesh"]
    g = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP32_ELEM)
    g.build_pattern(m.fixed_nodes)
    p = tl.params(h=w["h"], rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG, use_graph=1)
    out = {}
    for split in (0, 1):
        g.tune_set(force_split=split, residual_split=split)
        lam = torch.zeros(3 * len(m.fixed_nodes), dtype=torch.float64, device="cuda")
        v, _, st = g.newton_step(p, _dev(w["q_n"]), _dev(w["v"]), lam)
        assert st["converged"] == 1 and st["g_norm"] <= 1e-8 * st["g_ref"]
        out[split] = (v.cpu().numpy(), st)
    (v0, s0), (v1, s1) = out[0], out[1]
    assert s1["inner_iters"] == s0["inner_iters"] and s1["outer_iters"] == s0["outer_iters"]
    assert s1["g_ref"] == pytest.approx(s0["g_ref"], rel=1e-11)
    assert np.linalg.norm(v1 - v0) <= 1e-8 * np.linalg.norm(v0)


def test_newton_graph_caps_and_rebuild():
    """Iteration caps end the captured loops with NOT_CONVERGED and the same
    statistics as the host loop; a parameter change rebuilds the graph and a
    repeat reuses it with identical results."""
    tl = _tl()
    w = inputs.workload_small_svk()
    m = w["mesh"]
    g = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP64)
    g.build_pattern(m.fixed_nodes)
    stats = {}
    for use_graph in (0, 1):
        p = tl.params(h=w["h"], rtol=1e-14, max_inner=2, max_outer=2, linear_solver=tl.TL_SOLVER_PCG,
                      lin_max_iter=16, use_graph=use_graph)
        lam = torch.zeros(3 * len(m.fixed_nodes), dtype=torch.float64, device="cuda")
        _, _, st = g.newton_step(p, _dev(w["q_n"]), _dev(w["v"]), lam, raise_on_nonconvergence=False)
        stats[use_graph] = st
    assert stats[1]["status"] == stats[0]["status"] != 0
    for key in ("inner_iters", "outer_iters", "converged", "lin_iters"):
        assert stats[0][key] == stats[1][key], key
    assert stats[1]["inner_iters"] == 4 and stats[1]["outer_iters"] == 2
    assert stats[1]["lin_iters"] <= 4 * 16
    runs = []
    for rtol in (1e-8, 1e-6, 1e-8):
        p = tl.params(h=w["h"], rtol=rtol, linear_solver=tl.TL_SOLVER_PCG, use_graph=1)
        lam = torch.zeros(3 * len(m.fixed_nodes), dtype=torch.float64, device="cuda")
        v, _, st = g.newton_step(p, _dev(w["q_n"]), _dev(w["v"]), lam)
        runs.append((v.cpu().numpy(), st))
    assert np.linalg.norm(runs[2][0] - runs[0][0]) <= 1e-8 * np.linalg.norm(runs[0][0])
    assert runs[2][1]["inner_iters"] == runs[0][1]["inner_iters"]
    assert runs[1][1]["inner_iters"] <= runs[0][1]["inner_iters"]


def test_newton_graph_needs_pcg():
    tl = _tl()
    w = inputs.workload_small_svk()
    m = w["mesh"]
    g = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP64)
    g.build_pattern(m.fixed_nodes)
    p = tl.params(h=w["h"], linear_solver=tl.TL_SOLVER_DIRECT, use_graph=1)
    lam = torch.zeros(3 * len(m.fixed_nodes), dtype=torch.float64, device="cuda")
    with pytest.raises(tl.TLError):
        g.newton_step(p, _dev(w["q_n"]), _dev(w["v"]), lam)
