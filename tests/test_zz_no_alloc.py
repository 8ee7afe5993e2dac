"""GPU tests of tl_eval_residual_noalloc, the residual entry point for
callers that cannot allocate device memory while they step (their memory is
owned by a pool or a fixed budget, or a device-synchronising cudaMalloc is not
acceptable in their loop).  It must give the same g and ||g|| as
tl_eval_residual and as the oracle's residual, on consecutive calls (its
scratch array is shared and keeps the previous call's contents), for float64
and float32-element T10 handles, an ANCF beam handle and a handle with
general constraint rows, and refuse meshes beyond its stated limit.

This file is named so that pytest collects it last."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import ancf as oancf
from oracle import assembly as asm
from paper_2604_10357_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-11


def _tl():
    from paper_2604_10357_gb300 import build, tl
    build.build()
    return tl


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(-1), device="cuda")


def _case(kind):
    """(handle, oracle mesh, workload) for one kind of handle: float64 T10 (small
    SVK box, mid-size Mooney-Rivlin + Kelvin-Voigt box), the float32 element
    form, an ANCF3243 beam, and the small box with general constraint rows."""
    tl = _tl()
    if kind == "ancf_beam":
        w = inputs.workload_ancf_beam()
        m = w["mesh"]
        g = tl.Mesh.ancf("ancf3243", m.E0, m.conn, m.dims, [w["material"]])
        g.build_pattern(m.fixed_nodes)
        om = oancf.OracleAncfMesh("ancf3243", m.E0, m.conn, m.dims, [w["material"]], fixed_nodes=m.fixed_nodes)
        return tl, g, om, w, m.nn
    w = inputs.workload_mid_mr_kv() if kind == "mid_mr_kv" else inputs.workload_small_svk()
    m = w["mesh"]
    prec = tl.TL_FP32_ELEM if kind == "fp32_small" else tl.TL_FP64
    g = tl.Mesh(m.X, m.conn, [w["material"]], precision=prec)
    cons = None
    if kind == "constraints":
        # two tip nodes tied in y and z, and one row over three DOFs of three nodes; b = C X
        X = m.X
        tip = np.nonzero(np.isclose(X[:, 0], X[:, 0].max()))[0]
        a, b = tip[np.argmin(X[tip, 1] + X[tip, 2])], tip[np.argmax(X[tip, 1] + X[tip, 2])]
        mid = np.argsort(np.abs(X[:, 0] - 0.5 * X[:, 0].max()))[:3]
        rows = [[(3 * a + 1, 1.0), (3 * b + 1, -1.0)], [(3 * a + 2, 1.0), (3 * b + 2, -1.0)],
                [(3 * mid[0], 0.5), (3 * mid[1] + 1, -2.0), (3 * mid[2] + 2, 1.5)]]
        ri, ci, vi = zip(*[(r, c, val) for r, row in enumerate(rows) for c, val in row])
        C = sp.csr_matrix((vi, (ri, ci)), shape=(len(rows), 3 * m.nn))
        C.sort_indices()
        cons = (C, C @ X.ravel())
        g.set_constraints(C.indptr, C.indices, C.data, cons[1])
    g.build_pattern(m.fixed_nodes)
    g.tune_set(residual_split=0)          # tl_eval_residual in float64 too: the same arithmetic
    om = asm.OracleMesh(m.X, m.conn, [w["material"]], fixed_nodes=m.fixed_nodes, constraints=cons)
    return tl, g, om, w, m.nn


@pytest.mark.parametrize("kind", ["small_svk", "mid_mr_kv", "fp32_small", "ancf_beam", "constraints"])
def test_noalloc_residual_matches_existing_entry_point_and_oracle(kind):
    """Two calls in a row against tl_eval_residual (same float64 arithmetic,
    so within 1e-11 of it), and against the oracle's residual with the same
    internal force (within 1e-11 of the element-force scale)."""
    tl, g, om, w, nn = _case(kind)
    ncon = om.C_lin.shape[0]
    rng = np.random.default_rng(11)
    v_n = w["v"] + 0.01 * rng.normal(size=w["v"].shape)
    v_n[w["mesh"].fixed_nodes] = 0.0
    q, v, vn = _dev(w["q_n"]), _dev(w["v"]), _dev(v_n)
    f_ext_h = rng.normal(size=3 * nn)
    lam_h = rng.normal(size=3 * len(w["mesh"].fixed_nodes) + ncon)
    f_ext, lam = _dev(f_ext_h), _dev(lam_h)
    prm = tl.params(h=w["h"], rho_alm=1e6)
    f = g.eval_force(q, v, w["h"])
    g_ref, n_ref = g.eval_residual(prm, q, vn, v, f_ext=f_ext, lam=lam, f_int=f)
    g.sync()
    g_ref, n_ref = g_ref.cpu().numpy(), n_ref.item()
    # the oracle's residual with the handle's internal force: M (v - v_n) / h + f - f_ext - gravity
    # + constraint terms, evaluated by the oracle from its own mass, gravity and constraint rows
    f_h = f.cpu().numpy()
    g_ora = om.residual(w["v"].reshape(-1), w["q_n"].reshape(-1), v_n.reshape(-1), w["h"], f_ext_h,
                        prm.gravity[:], lam_h, 1e6) \
        - om.internal_force(w["q_n"].reshape(-1), w["v"].reshape(-1), w["h"]) + f_h
    out = torch.empty(3 * nn, dtype=torch.float64, device="cuda")
    nrm = torch.empty(1, dtype=torch.float64, device="cuda")
    for _call in range(2):
        out.fill_(np.nan)
        nrm.fill_(np.nan)
        g.eval_residual_noalloc(prm, q, vn, v, f, out, nrm, f_ext=f_ext, lam=lam)
        g.sync()
        got = out.cpu().numpy()
        assert np.abs(got - g_ref).max() <= TOL * np.abs(g_ref).max()
        assert abs(nrm.item() - n_ref) <= TOL * n_ref
        assert np.abs(got - g_ora).max() <= TOL * max(np.abs(g_ora).max(), np.abs(f_h).max())
        assert abs(nrm.item() - np.linalg.norm(g_ora)) <= TOL * np.linalg.norm(g_ora)


def test_noalloc_rejects_meshes_beyond_its_limit():
    """4,194,305 nodes (one hexahedron's 6 elements plus unconnected nodes):
    one node past the limit of 16,384 blocks of 256 nodes."""
    tl = _tl()
    box = inputs.box_t10(1, 1, 1, 0.1, 0.1, 0.1, fixed_face_x0=False)
    n_total = 16384 * 256 + 1
    X = np.zeros((n_total, 3))
    X[: box.nn] = box.X
    X[box.nn:, 0] = 10.0 + np.arange(n_total - box.nn) * 1e-3
    g = tl.Mesh(X, box.conn, [dict(inputs.SVK_1E7)], precision=tl.TL_FP64)
    g.build_pattern(())
    zeros = torch.zeros(3 * n_total, dtype=torch.float64, device="cuda")
    out = torch.empty_like(zeros)
    nrm = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(tl.TLError) as ei:
        g.eval_residual_noalloc(tl.params(), zeros, zeros, zeros, zeros, out, nrm)
    assert ei.value.status == 10
    assert "4,194,304" in str(ei.value)
