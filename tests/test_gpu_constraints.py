"""General linear bilateral constraints (Sec. 4.2's user-given C_q rows,
tl_set_constraints) against the oracle: the Newton-matrix pattern with the
constraint fill (bit-exact), the CSR values with h^2 rho C^T C (float64 and
the float32 form), the residual with h C^T (lambda + rho c), and the Newton
step with the multiplier updates of both kinds of rows."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import assembly as asm
from oracle import newton as nt
from paper_2604_10357_gb300 import inputs

from helpers import TOL_FP32, TOL_FP64, force_error, values_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _tl():
    from paper_2604_10357_gb300 import build, tl
    build.build()
    return tl


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(-1), device="cuda")


@pytest.fixture(scope="module")
def case():
    """The 240-element cantilever with three general rows: two tip nodes on
    opposite corners tied in y and z (no element couples them), and one row
    over three DOFs of three nodes; b = C X."""
    w = inputs.workload_small_svk()
    m = w["mesh"]
    X = m.X
    tip = np.nonzero(np.isclose(X[:, 0], X[:, 0].max()))[0]
    a = tip[np.argmin(X[tip, 1] + X[tip, 2])]
    b = tip[np.argmax(X[tip, 1] + X[tip, 2])]
    mid = np.argsort(np.abs(X[:, 0] - 0.5 * X[:, 0].max()))[:3]
    rows = [[(3 * a + 1, 1.0), (3 * b + 1, -1.0)], [(3 * a + 2, 1.0), (3 * b + 2, -1.0)],
            [(3 * mid[0], 0.5), (3 * mid[1] + 1, -2.0), (3 * mid[2] + 2, 1.5)]]
    ri, ci, vi = zip(*[(r, c, val) for r, row in enumerate(rows) for c, val in row])
    C = sp.csr_matrix((vi, (ri, ci)), shape=(len(rows), 3 * m.nn))
    C.sort_indices()
    bvec = C @ X.ravel()
    om = asm.OracleMesh(m.X, m.conn, [w["material"]], fixed_nodes=m.fixed_nodes, constraints=(C, bvec))
    return w, C, bvec, om


def _mesh(tl, w, C, bvec, prec):
    m = w["mesh"]
    g = tl.Mesh(m.X, m.conn, [w["material"]], precision=prec)
    g.set_constraints(C.indptr, C.indices, C.data, bvec)
    g.build_pattern(m.fixed_nodes)
    return g


def test_pattern_with_constraint_fill(case):
    tl = _tl()
    w, C, bvec, om = case
    g = _mesh(tl, w, C, bvec, tl.TL_FP64)
    row_ptr, col = (a.cpu().numpy() for a in g.get_pattern()[:2])
    _, _, r_ref, c_ref = om.pattern()
    assert g.info()["ncon"] == C.shape[0]
    assert np.array_equal(row_ptr, r_ref) and np.array_equal(col, c_ref)
    plain = asm.OracleMesh(w["mesh"].X, w["mesh"].conn, [w["material"]]).pattern()[3]
    assert len(col) > len(plain)                          # the tie is a fill-in


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_hessian_values_with_constraints(case, prec):
    tl = _tl()
    w, C, bvec, om = case
    g = _mesh(tl, w, C, bvec, tl.TL_FP64 if prec == "fp64" else tl.TL_FP32_ELEM)
    h, rho = w["h"], 1e6                                  # h^2 rho = 1: penalties on the scale of M / h
    vals = g.assemble_hessian(_dev(w["q_n"]), _dev(w["v"]), h, rho).cpu().numpy().astype(np.float64)
    g.sync()
    ref = om.hessian_values(w["q_n"], w["v"], h, rho)
    tol = TOL_FP64 if prec == "fp64" else TOL_FP32
    emax, e2 = values_error(vals, ref)
    assert emax < tol and e2 < tol


def test_residual_with_constraints(case):
    tl = _tl()
    w, C, bvec, om = case
    m = w["mesh"]
    g = _mesh(tl, w, C, bvec, tl.TL_FP64)
    rng = np.random.default_rng(41)
    v_n = w["v"] + 0.01 * rng.normal(size=w["v"].shape)
    lam = rng.normal(size=3 * len(m.fixed_nodes) + C.shape[0])
    prm = tl.params(h=w["h"], rho_alm=1e6)
    gg, gn = g.eval_residual(prm, _dev(w["q_n"]), _dev(v_n), _dev(w["v"]), None, _dev(lam))
    g.sync()
    g_ora = om.residual(w["v"], w["q_n"], v_n, w["h"], None, prm.gravity[:], lam, 1e6)
    fe = om.element_forces(w["q_n"] + w["h"] * w["v"], w["v"])
    assert force_error(gg.cpu().numpy(), g_ora, fe) < TOL_FP64
    assert abs(gn.item() - np.linalg.norm(g_ora)) < 1e-10 * np.linalg.norm(g_ora)


@pytest.mark.parametrize("solver", ["direct", "pcg_graph"])
def test_newton_step_with_constraints(case, solver):
    tl = _tl()
    w, C, bvec, om = case
    m = w["mesh"]
    prm = nt.NewtonParams(h=w["h"], rtol=1e-8, solver="dense")
    lam0 = np.zeros(3 * len(m.fixed_nodes) + C.shape[0])
    ref = nt.newton_step(om, w["q_n"].ravel(), w["v"].ravel(), lam0, prm)
    assert ref["converged"]
    g = _mesh(tl, w, C, bvec, tl.TL_FP64)
    lam = _dev(lam0)
    p = tl.params(h=prm.h, rho_alm=prm.rho_alm, rtol=prm.rtol, eps_out=prm.eps_out,
                  linear_solver=tl.TL_SOLVER_DIRECT if solver == "direct" else tl.TL_SOLVER_PCG,
                  use_graph=1 if solver == "pcg_graph" else 0)
    v, _, st = g.newton_step(p, _dev(w["q_n"]), _dev(w["v"]), lam)
    v = v.cpu().numpy()
    assert st["converged"] == 1
    assert st["outer_iters"] == ref["outer_iters"]
    assert np.linalg.norm(v - ref["v"]) <= 1e-8 * np.linalg.norm(ref["v"])
    lg = lam.cpu().numpy()
    assert np.abs(lg - ref["lam"]).max() <= 1e-6 * np.abs(ref["lam"]).max()
    c = C @ (w["q_n"].ravel() + prm.h * v) - bvec           # the tie holds to the ALM tolerance
    assert np.linalg.norm(c) <= prm.eps_out


def test_float32_graph_step_with_constraints(case):
    """The float32 element form with the captured graph and inexact-Newton PCG:
    the converged step satisfies the oracle's residual target and the ties."""
    tl = _tl()
    w, C, bvec, om = case
    m = w["mesh"]
    prm = nt.NewtonParams(h=w["h"], rtol=1e-8, solver="dense")
    lam0 = np.zeros(3 * len(m.fixed_nodes) + C.shape[0])
    ref = nt.newton_step(om, w["q_n"].ravel(), w["v"].ravel(), lam0, prm)
    g = _mesh(tl, w, C, bvec, tl.TL_FP32_ELEM)
    lam = _dev(lam0)
    p = tl.params(h=prm.h, rho_alm=prm.rho_alm, rtol=prm.rtol, eps_out=prm.eps_out,
                  linear_solver=tl.TL_SOLVER_PCG, lin_adaptive=1, use_graph=1)
    v, _, st = g.newton_step(p, _dev(w["q_n"]), _dev(w["v"]), lam)
    v = v.cpu().numpy()
    assert st["converged"] == 1
    lam_inner = lam.cpu().numpy() - prm.rho_alm * om.constraint(w["q_n"].ravel() + prm.h * v)
    g_at = om.residual(v, w["q_n"].ravel(), w["v"].ravel(), prm.h, None, prm.gravity, lam_inner, prm.rho_alm)
    assert np.linalg.norm(g_at) <= 1.05 * 1e-8 * ref["g_ref"]
    assert np.linalg.norm(C @ (w["q_n"].ravel() + prm.h * v) - bvec) <= prm.eps_out


def test_adamw_with_constraints_matches_oracle(case):
    """Algorithm 2 with general rows: two outer iterations of fixed length
    (velocity commit, multiplier update of both kinds of rows)."""
    from oracle import adamw as aw
    tl = _tl()
    w, C, bvec, om = case
    m = w["mesh"]
    ap = dict(lr=1e-4, max_inner=30, check_every=1000, eps_in=0.0, eps_rel=0.0)
    lam0 = np.zeros(3 * len(m.fixed_nodes) + C.shape[0])
    ref = aw.adamw_step(om, w["q_n"].ravel(), w["v"].ravel(), lam0,
                        aw.AdamWParams(h=w["h"], rho_alm=1e12, max_outer=2, **ap))
    g = _mesh(tl, w, C, bvec, tl.TL_FP64)
    lam = _dev(lam0)
    v, _, st = g.adamw_step(tl.params(h=w["h"], rho_alm=1e12, max_outer=2), tl.adamw_params(**ap),
                            _dev(w["q_n"]), _dev(w["v"]), lam, raise_on_nonconvergence=False)
    assert st["inner_iters"] == 60 and st["outer_iters"] == 2
    v = v.cpu().numpy()
    assert np.linalg.norm(v - ref["v"]) <= 1e-9 * np.linalg.norm(ref["v"])
    lg = lam.cpu().numpy()
    assert np.abs(lg - ref["lam"]).max() <= 1e-9 * np.abs(ref["lam"]).max()
    assert st["c_norm"] == pytest.approx(ref["c_norm"], rel=1e-9)
