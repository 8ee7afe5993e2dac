"""ANCF3243 beam and ANCF3443 shell elements through the C ABI against the
oracle: the coefficient-level pattern and slot map (bit-exact), the internal
force, the element tangents, the assembled Hessian values, the residual
(exact mass, gravity weights, clamps), the Newton step (direct and the
captured PCG graph), the closed-form free fall, argument errors, and the
full-size benchmark meshes on sampled elements and coefficients."""
import numpy as np
import pytest

from oracle import ancf
from oracle import assembly as asm
from oracle import newton as nt
from paper_2604_10357_gb300 import inputs

from helpers import TOL_FP32, TOL_FP64, force_error, values_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MR = dict(kind="mr", C10=5e5, C01=1e5, kappa=1e8, rho0=1000.0, eta_d=0.0, lambda_d=0.0)
MATS = {
    "svk": [dict(inputs.SVK_7E8)],
    "svk_kv": [dict(inputs.SVK_7E8, eta_d=1e3, lambda_d=1e3)],
    "mr": [MR],
    "mr_kv": [dict(MR, eta_d=1e3, lambda_d=2e3)],
    "mixed": [dict(inputs.SVK_7E8), dict(MR, eta_d=1e3, lambda_d=1e3)],
}
KINDS = [ancf.BEAM, ancf.SHELL]


def _tl():
    from paper_2604_10357_gb300 import build, tl
    build.build()
    return tl


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(-1), device="cuda")


def _workload(kind):
    """Beam: 21 elements (three CTAs of 8, the last ragged); shell: 5 x 3."""
    return inputs.workload_ancf_beam(21) if kind == ancf.BEAM else inputs.workload_ancf_shell(5, 3)


def _case(kind, mats_key, clamp=True, fp32=False):
    w = _workload(kind)
    m = w["mesh"]
    mats = MATS[mats_key]
    moe = None if len(mats) == 1 else (np.arange(m.ne) % 3 == 1).astype(np.int32)
    fixed = m.fixed_nodes if clamp else np.zeros(0, dtype=np.int32)
    om = ancf.OracleAncfMesh(kind, m.E0, m.conn, m.dims, mats, mat_of_elem=moe, fixed_nodes=fixed)
    tl = _tl()
    g = tl.Mesh.ancf(kind, m.E0, m.conn, m.dims, mats, mat_of_elem=moe,
                     precision=tl.TL_FP32_ELEM if fp32 else tl.TL_FP64)
    g.build_pattern(fixed)
    return w, om, g, tl


def _tangent_error(K_gpu, K_ora):
    nd2 = K_ora.shape[1] * K_ora.shape[2]
    K_gpu = np.asarray(K_gpu, dtype=np.float64).reshape(-1, nd2)
    K_ora = np.asarray(K_ora, dtype=np.float64).reshape(-1, nd2)
    return float(np.max(np.linalg.norm(K_gpu - K_ora, axis=1) / np.linalg.norm(K_ora, axis=1)))


@pytest.mark.parametrize("kind", KINDS)
def test_pattern_and_slot_map_bit_exact(kind):
    w, om, g, tl = _case(kind, "svk")
    row_ptr, col, slot = (a.cpu().numpy() for a in g.get_pattern(with_slot_map=True))
    _, _, r_ref, c_ref = om.pattern()
    assert np.array_equal(row_ptr, r_ref) and np.array_equal(col, c_ref)
    assert np.array_equal(slot.reshape(om.ne, -1), asm.slot_map(om.conn, r_ref, c_ref))
    inf = g.info()
    assert inf["element_kind"] == (tl.TL_ELEM_ANCF3243 if kind == ancf.BEAM else tl.TL_ELEM_ANCF3443)
    assert inf["nen"] == ancf.nen_of(kind) and inf["nnz"] == len(c_ref)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("mats_key", list(MATS))
def test_internal_force(kind, mats_key):
    w, om, g, tl = _case(kind, mats_key)
    f = g.eval_force(_dev(w["q_n"]), _dev(w["v"]), w["h"]).cpu().numpy()
    g.sync()
    ref = om.internal_force(w["q_n"], w["v"], w["h"])
    fe = om.element_forces(w["q_n"] + w["h"] * w["v"], w["v"])
    assert force_error(f, ref, fe) < TOL_FP64


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("mats_key", list(MATS))
def test_element_tangents(kind, mats_key):
    """K_elem = alpha K_t + beta D for (alpha, beta) = (h, 1) and (1, 0)."""
    w, om, g, tl = _case(kind, mats_key)
    h = w["h"]
    x = w["q_n"] + h * w["v"]
    for alpha, beta in ((h, 1.0), (1.0, 0.0)):
        K = g.eval_tangent(_dev(w["q_n"]), _dev(w["v"]), h, alpha, beta).cpu().numpy()
        g.sync()
        assert _tangent_error(K, om.element_tangents(x, w["v"], alpha, beta)) < TOL_FP64


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("mats_key", ["svk", "mr_kv", "mixed"])
def test_hessian_values(kind, mats_key):
    """H = M/h + h K_t + D + h^2 rho C_q^T C_q in the CSR values, and the fused
    force of the same pass."""
    w, om, g, tl = _case(kind, mats_key)
    h, rho = w["h"], 1e8
    f = torch.empty(3 * om.nn, dtype=torch.float64, device="cuda")
    vals = g.assemble_hessian(_dev(w["q_n"]), _dev(w["v"]), h, rho, f_int=f).cpu().numpy()
    g.sync()
    emax, e2 = values_error(vals, om.hessian_values(w["q_n"], w["v"], h, rho))
    assert emax < TOL_FP64 and e2 < TOL_FP64
    fe = om.element_forces(w["q_n"] + h * w["v"], w["v"])
    assert force_error(f.cpu().numpy(), om.internal_force(w["q_n"], w["v"], h), fe) < TOL_FP64


@pytest.mark.parametrize("kind", KINDS)
def test_residual_mass_gravity_clamps(kind):
    """g = M (v - v_n)/h + f_int - f_ext - f_ff + h C^T (lambda + rho c):
    exact mass, the gravity weights int rho S_a dV, clamps on coefficients."""
    w, om, g, tl = _case(kind, "svk_kv")
    m = w["mesh"]
    rng = np.random.default_rng(11)
    v_n = w["v"] + 0.01 * rng.normal(size=w["v"].shape)
    f_ext = rng.normal(size=w["v"].shape)
    lam = rng.normal(size=3 * len(m.fixed_nodes))
    prm = tl.params(h=w["h"], rho_alm=1e6)
    gg, gn = g.eval_residual(prm, _dev(w["q_n"]), _dev(v_n), _dev(w["v"]), _dev(f_ext), _dev(lam))
    g.sync()
    g_ora = om.residual(w["v"], w["q_n"], v_n, w["h"], f_ext, prm.gravity[:], lam, 1e6)
    fe = om.element_forces(w["q_n"] + w["h"] * w["v"], w["v"])
    assert force_error(gg.cpu().numpy(), g_ora, fe) < TOL_FP64
    assert abs(gn.item() - np.linalg.norm(g_ora)) < 1e-10 * np.linalg.norm(g_ora)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("solver", ["direct", "pcg_graph"])
def test_newton_step(kind, solver):
    """One backward-Euler step (Algorithm 3) from the perturbed, bent state:
    the converged velocity, outer iterations and multipliers of the oracle."""
    w, om, g, tl = _case(kind, "svk")
    m = w["mesh"]
    prm = nt.NewtonParams(h=w["h"], rtol=1e-8, solver="dense")
    lam0 = np.zeros(3 * len(m.fixed_nodes))
    ref = nt.newton_step(om, w["q_n"].ravel(), w["v"].ravel(), lam0, prm)
    assert ref["converged"]
    lam = _dev(lam0)
    p = tl.params(h=prm.h, rho_alm=prm.rho_alm, rtol=prm.rtol, eps_out=prm.eps_out,
                  linear_solver=tl.TL_SOLVER_DIRECT if solver == "direct" else tl.TL_SOLVER_PCG,
                  use_graph=1 if solver == "pcg_graph" else 0)
    v, _, st = g.newton_step(p, _dev(w["q_n"]), _dev(w["v"]), lam)
    v = v.cpu().numpy()
    assert st["converged"] == 1 and st["outer_iters"] == ref["outer_iters"]
    assert np.linalg.norm(v - ref["v"]) <= 1e-8 * np.linalg.norm(ref["v"])
    assert np.abs(lam.cpu().numpy() - ref["lam"]).max() <= 1e-6 * np.abs(ref["lam"]).max()


@pytest.mark.parametrize("kind", KINDS)
def test_free_fall_closed_form(kind):
    """Unclamped body at rest in its reference configuration: v = h g on the
    position coefficients and 0 on the gradients after one step."""
    w, om, g, tl = _case(kind, "svk", clamp=False)
    m = w["mesh"]
    p = tl.params(h=1e-3, rtol=1e-12)
    v, _, st = g.newton_step(p, _dev(m.E0), _dev(np.zeros_like(m.E0)), _dev(np.zeros(0)))
    ref = np.zeros_like(m.E0)
    ref[0::4] = 1e-3 * np.asarray(inputs.GRAVITY)
    np.testing.assert_allclose(v.cpu().numpy().reshape(-1, 3), ref, atol=1e-12)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("mats_key", ["svk", "svk_kv", "mr", "mr_kv"])
def test_element_tangents_fp32(kind, mats_key):
    """The float32 element form: K_elem in float32 within 1e-5 of the oracle."""
    w, om, g, tl = _case(kind, mats_key, fp32=True)
    h = w["h"]
    K = g.eval_tangent(_dev(w["q_n"]), _dev(w["v"]), h, h, 1.0)
    g.sync()
    assert K.dtype == torch.float32
    x = w["q_n"] + h * w["v"]
    assert _tangent_error(K.cpu().numpy(), om.element_tangents(x, w["v"], h, 1.0)) < TOL_FP32


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("mats_key", ["svk", "mixed"])
def test_hessian_values_fp32(kind, mats_key):
    """Float32 CSR values within 1e-5; the residual force of the handle stays
    float64-class (1e-11)."""
    w, om, g, tl = _case(kind, mats_key, fp32=True)
    h, rho = w["h"], 1e8
    vals = g.assemble_hessian(_dev(w["q_n"]), _dev(w["v"]), h, rho).cpu().numpy().astype(np.float64)
    g.sync()
    emax, e2 = values_error(vals, om.hessian_values(w["q_n"], w["v"], h, rho))
    assert emax < TOL_FP32 and e2 < TOL_FP32
    prm = tl.params(h=h, rho_alm=1e6)
    lam = np.zeros(3 * len(w["mesh"].fixed_nodes))
    gg, _ = g.eval_residual(prm, _dev(w["q_n"]), _dev(w["v"]), _dev(w["v"]), None, _dev(lam))
    g.sync()
    g_ora = om.residual(w["v"], w["q_n"], w["v"], h, None, prm.gravity[:], lam, 1e6)
    fe = om.element_forces(w["q_n"] + h * w["v"], w["v"])
    assert force_error(gg.cpu().numpy(), g_ora, fe) < TOL_FP64


@pytest.mark.parametrize("kind", KINDS)
def test_newton_step_fp32_graph(kind):
    """Float32 element form, captured graph, inexact-Newton PCG: the step meets
    the oracle's residual target at the converged velocity."""
    w, om, g, tl = _case(kind, "svk", fp32=True)
    m = w["mesh"]
    prm = nt.NewtonParams(h=w["h"], rtol=1e-8, solver="dense")
    lam0 = np.zeros(3 * len(m.fixed_nodes))
    ref = nt.newton_step(om, w["q_n"].ravel(), w["v"].ravel(), lam0, prm)
    lam = _dev(lam0)
    p = tl.params(h=prm.h, rho_alm=prm.rho_alm, rtol=prm.rtol, eps_out=prm.eps_out,
                  linear_solver=tl.TL_SOLVER_PCG, lin_adaptive=1, use_graph=1)
    v, _, st = g.newton_step(p, _dev(w["q_n"]), _dev(w["v"]), lam)
    v = v.cpu().numpy()
    assert st["converged"] == 1
    lam_inner = lam.cpu().numpy() - prm.rho_alm * om.constraint(w["q_n"].ravel() + prm.h * v)
    g_at = om.residual(v, w["q_n"].ravel(), w["v"].ravel(), prm.h, None, prm.gravity, lam_inner, prm.rho_alm)
    assert np.linalg.norm(g_at) <= 1.05 * 1e-8 * ref["g_ref"]
    assert np.linalg.norm(v - ref["v"]) <= 1e-6 * np.linalg.norm(ref["v"])


def test_argument_errors():
    tl = _tl()
    m = inputs.beam_ancf3243(4)
    mat = [dict(inputs.SVK_7E8)]
    with pytest.raises(tl.TLError) as ei:
        tl.Mesh.ancf(7, m.E0, m.conn, m.dims, mat)                   # not an ANCF kind
    assert ei.value.status == 1                                    # TL_ERR_INVALID_ARG
    bad = m.conn.copy()
    bad[2, 5] = m.nn
    with pytest.raises(tl.TLError) as ei:
        tl.Mesh.ancf("ancf3243", m.E0, bad, m.dims, mat)
    assert ei.value.status == 1                                    # TL_ERR_INVALID_ARG
    dims = m.dims.copy()
    dims[1, 2] = 0.0
    with pytest.raises(tl.TLError):
        tl.Mesh.ancf("ancf3243", m.E0, m.conn, dims, mat)
    flipped = m.E0.copy()
    flipped[4 * 2 + 3] *= -1.0                                      # r_z of node 2 reversed: det J0 < 0
    with pytest.raises(tl.TLError) as ei:
        tl.Mesh.ancf("ancf3243", flipped, m.conn, m.dims, mat)
    assert "Jacobian" in str(ei.value)


# ---------------------------------------------------------------------------
# full-size benchmark meshes: sampled elements and coefficient rows
# ---------------------------------------------------------------------------

def _fullsize(kind):
    """The largest resolutions of the paper's ANCF scaling tables: a
    500,000-element beam and a 200 x 200 shell, bent and perturbed."""
    rng = np.random.default_rng(1000 + 8)
    if kind == ancf.BEAM:
        m = inputs.beam_ancf3243(500_000)
        q = inputs.ancf_perturbation(m, inputs.ancf_bend(m, 1e-5), 0.01, rng)
        h = 1e-3
    else:
        m = inputs.shell_ancf3443(200, 200)
        q = inputs.ancf_perturbation(m, inputs.ancf_bend(m, 0.25), 0.01, rng)
        h = 5e-4
    v = rng.normal(0.0, 0.01, size=q.shape)
    v[m.fixed_nodes] = 0.0
    return m, q, v, h


@pytest.mark.parametrize("kind", KINDS)
def test_fullsize_sampled(kind):
    tl = _tl()
    m, q, v, h = _fullsize(kind)
    mat = [dict(inputs.SVK_7E8)]
    g = tl.Mesh.ancf(kind, m.E0, m.conn, m.dims, mat)
    g.build_pattern(m.fixed_nodes)
    rho = 1e8
    vals = g.assemble_hessian(_dev(q), _dev(v), h, rho)
    K = g.eval_tangent(_dev(q), _dev(v), h, h, 1.0)
    row_ptr, col, _ = g.get_pattern()
    g.sync()
    rng = np.random.default_rng(5)
    # sampled element tangents
    els = np.unique(np.concatenate([[0, m.ne - 1], rng.integers(0, m.ne, 16)]))
    nd = 3 * m.conn.shape[1]
    Ks = K.view(m.ne, nd, nd)[torch.as_tensor(els, device="cuda")].cpu().numpy()
    sub = ancf.OracleAncfMesh(kind, m.E0, m.conn[els], m.dims[els], mat)
    x = q + h * v
    # The 100 km beam holds positions up to 5e5 element lengths from the
    # origin: the float64 rounding of q itself perturbs F = sum_a x_a (x) grad S_a
    # by about u |x| / L relative, on either side, so the bar is the larger of
    # 1e-11 and 4 u max|x| / min L (4.4e-10 for the 100 km beam, 1e-11 for the shell).
    tol = max(TOL_FP64, 4.0 * np.finfo(np.float64).eps * np.abs(x).max() / m.dims[:, 0].min())
    assert _tangent_error(Ks, sub.element_tangents(x, v, h, 1.0)) < tol
    # sampled coefficient rows of H: the incident elements' contributions
    rp = row_ptr.cpu().numpy()
    cl = col.cpu().numpy()
    fixed = set(m.fixed_nodes.tolist())
    coefs = [c for c in rng.integers(0, m.nn, 12) if c not in fixed]
    for I in coefs:
        inc = np.nonzero((m.conn == I).any(axis=1))[0]
        so = ancf.OracleAncfMesh(kind, m.E0, m.conn[inc], m.dims[inc], mat)
        Ke = so.element_tangents(x, v, h, 1.0)
        Me = so.Me / h
        row = {}
        for k, e in enumerate(inc):
            a = int(np.nonzero(m.conn[e] == I)[0][0])
            for i in range(3):
                for b, J in enumerate(m.conn[e]):
                    for kk in range(3):
                        val = Ke[k, 3 * a + i, 3 * b + kk] + (Me[k, a, b] if i == kk else 0.0)
                        row[(3 * I + i, 3 * J + kk)] = row.get((3 * I + i, 3 * J + kk), 0.0) + val
        got = {}
        for r in range(3 * I, 3 * I + 3):
            seg = slice(rp[r], rp[r + 1])
            pos = np.arange(rp[r], rp[r + 1])
            for c, p in zip(cl[seg], pos):
                got[(r, int(c))] = p
        assert set(row) == set(got)
        gv = vals[torch.as_tensor([got[k] for k in row], device="cuda")].cpu().numpy()
        ref = np.array(list(row.values()))
        assert np.abs(gv - ref).max() < tol * np.abs(ref).max()


# ---------------------------------------------------------------------------
# the other rows of the framework on ANCF handles
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", KINDS)
def test_adamw_step(kind):
    """Algorithm 2 on an ANCF handle: two outer iterations of 30 fixed updates
    (velocity commit and multiplier update between them) against the oracle's."""
    from oracle import adamw as aw
    w, om, g, tl = _case(kind, "svk")
    m = w["mesh"]
    ap = dict(lr=1e-4, max_inner=30, check_every=1000, eps_in=0.0, eps_rel=0.0)
    lam0 = np.zeros(3 * len(m.fixed_nodes))
    ref = aw.adamw_step(om, w["q_n"].ravel(), w["v"].ravel(), lam0,
                        aw.AdamWParams(h=w["h"], rho_alm=1e12, max_outer=2, **ap))
    lam = _dev(lam0)
    v, _, st = g.adamw_step(tl.params(h=w["h"], rho_alm=1e12, max_outer=2), tl.adamw_params(**ap),
                            _dev(w["q_n"]), _dev(w["v"]), lam, raise_on_nonconvergence=False)
    assert st["inner_iters"] == 60 and st["outer_iters"] == 2
    v = v.cpu().numpy()
    assert np.linalg.norm(v - ref["v"]) <= 1e-9 * np.linalg.norm(ref["v"])
    assert np.abs(lam.cpu().numpy() - ref["lam"]).max() <= 1e-9 * np.abs(ref["lam"]).max()


@pytest.mark.parametrize("kind", KINDS)
def test_general_constraints(kind):
    """General linear rows on ANCF coefficients (Sec. 4.2): the tip position
    tied in z to a mid-span position, and a row over gradient components of
    coefficients that share no element, both holding at the start state;
    pattern with the fill (bit-exact), Hessian values and the Newton step
    against the oracle (the rows still hold after the step)."""
    import scipy.sparse as sp
    w = _workload(kind)
    m = w["mesh"]
    tl = _tl()
    last, mid = 4 * (m.nphys - 1), 4 * (m.nphys // 2)
    far = 4 * 1 + 2                                     # r_y of node 1
    rows = [[(3 * last + 2, 1.0), (3 * mid + 2, -1.0)],
            [(3 * far + 1, 0.5), (3 * (last + 1) + 0, -2.0), (3 * (mid + 3) + 2, 1.5)]]
    ri, ci, vi = zip(*[(r, c, val) for r, row in enumerate(rows) for c, val in row])
    C = sp.csr_matrix((vi, (ri, ci)), shape=(len(rows), 3 * m.nn))
    C.sort_indices()
    bvec = C @ w["q_n"].ravel()                         # the rows hold at the start state
    mat = [dict(inputs.SVK_7E8)]
    om = ancf.OracleAncfMesh(kind, m.E0, m.conn, m.dims, mat, fixed_nodes=m.fixed_nodes, constraints=(C, bvec))
    g = tl.Mesh.ancf(kind, m.E0, m.conn, m.dims, mat)
    g.set_constraints(C.indptr, C.indices, C.data, bvec)
    g.build_pattern(m.fixed_nodes)
    row_ptr, col = (a.cpu().numpy() for a in g.get_pattern()[:2])
    _, _, r_ref, c_ref = om.pattern()
    assert np.array_equal(row_ptr, r_ref) and np.array_equal(col, c_ref)
    h, rho = w["h"], 1e8
    vals = g.assemble_hessian(_dev(w["q_n"]), _dev(w["v"]), h, rho).cpu().numpy()
    g.sync()
    emax, e2 = values_error(vals, om.hessian_values(w["q_n"], w["v"], h, rho))
    assert emax < TOL_FP64 and e2 < TOL_FP64
    prm = nt.NewtonParams(h=h, rtol=1e-8, solver="dense")
    lam0 = np.zeros(3 * len(m.fixed_nodes) + C.shape[0])
    ref = nt.newton_step(om, w["q_n"].ravel(), w["v"].ravel(), lam0, prm)
    assert ref["converged"]
    lam = _dev(lam0)
    p = tl.params(h=prm.h, rho_alm=prm.rho_alm, rtol=prm.rtol, eps_out=prm.eps_out,
                  linear_solver=tl.TL_SOLVER_DIRECT)
    v, _, st = g.newton_step(p, _dev(w["q_n"]), _dev(w["v"]), lam)
    v = v.cpu().numpy()
    assert st["converged"] == 1 and st["outer_iters"] == ref["outer_iters"]
    assert np.linalg.norm(v - ref["v"]) <= 1e-8 * np.linalg.norm(ref["v"])
    assert np.linalg.norm(C @ (w["q_n"].ravel() + h * v) - bvec) <= prm.eps_out
