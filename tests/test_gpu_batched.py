"""Batched bodies: 48 independent bodies of uneven size (1k-60k T10 each,
boxes and cylinders, SVK and Mooney-Rivlin, one face clamped each) in one
handle.  The element pass is one persistent launch over all bodies; parity
with the FP64 oracle at full size on sampled elements (element tangents and
forces) and on sampled CSR rows of the assembled Hessian; and the internal
force of every body is self-equilibrated (it sums to zero over the body); a
captured FP32 Newton step of the whole batch from rest under gravity, checked
body by body against the oracle's residual."""
import numpy as np
import pytest

from oracle import element as oelem
from oracle import t10
from oracle.assembly import OracleMesh, node_adjacency
from paper_2604_10357_gb300 import inputs

from helpers import TOL_FP32, tangent_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _tl():
    from paper_2604_10357_gb300 import build, tl
    build.build()
    return tl


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(-1), device="cuda")


@pytest.fixture(scope="module")
def batched():
    tl = _tl()
    w = inputs.workload_batched()
    m = w["mesh"]
    g = tl.Mesh(m.X, m.conn, w["materials"], w["mat_of_elem"], precision=tl.TL_FP32_ELEM)
    g.build_pattern(m.fixed_nodes)
    rng = np.random.default_rng(31)
    # sampled elements: the first, last and 4 random elements of every body
    idx = []
    starts = np.concatenate([[0], np.cumsum([b.ne for b in w["meshes"]])])
    for b in range(len(w["meshes"])):
        lo, hi = starts[b], starts[b + 1]
        idx += [lo, hi - 1] + list(rng.integers(lo, hi, size=4))
    return tl, w, g, np.unique(np.array(idx, dtype=np.int64))


def _oracle_elements(w, idx, x, v, alpha, beta):
    m = w["mesh"]
    conn = m.conn[idx].astype(np.int64)
    gradN, _, wJ0 = t10.reference_geometry(m.X, conn)
    mats = np.asarray(w["mat_of_elem"])[idx]
    K = np.zeros((len(idx), 30, 30))
    f = np.zeros((len(idx), 10, 3))
    for k in np.unique(mats):
        sel = np.nonzero(mats == k)[0]
        c = conn[sel]
        mat = w["materials"][k]
        K[sel] = oelem.element_tangent(x[c], v[c], gradN[sel], wJ0[sel], mat, alpha, beta)
        f[sel] = oelem.element_force(x[c], v[c], gradN[sel], wJ0[sel], mat)
    return K, f


def test_one_persistent_launch_and_sampled_element_parity(batched):
    tl, w, g, idx = batched
    m = w["mesh"]
    h = w["h"]
    q, v = _dev(w["q_n"]), _dev(w["v"])
    g.timing_read()
    f = g.eval_force(q, v, h)
    g.sync()
    assert g.timing_read()["launches"] == 1          # all 48 bodies, both materials, one launch
    K = g.eval_tangent(q, v, h, h, 1.0)
    Ks = K.view(m.ne, 900)[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    x = w["q_n"] + h * w["v"]
    K_ora, _ = _oracle_elements(w, idx, x, w["v"], h, 1.0)
    assert tangent_error(Ks, K_ora) < TOL_FP32
    del K
    # per-body equilibrium of the assembled internal force
    fb = f.view(-1, 3).cpu().numpy()
    body = np.asarray(m.body_of_node)
    tot = np.zeros((len(w["meshes"]), 3))
    mag = np.zeros(len(w["meshes"]))
    np.add.at(tot, body, fb)
    np.add.at(mag, body, np.abs(fb).sum(1))
    assert np.all(np.linalg.norm(tot, axis=1) <= 1e-6 * mag)


@pytest.mark.parametrize("agg", [0, 1])
def test_sampled_hessian_rows(batched, agg):
    """CSR rows of a few nodes per body: every entry against the oracle's
    element matrices (mass / h + h K_t + D) summed over the elements at the
    node, plus the clamp penalty; with the per-element scatter and with the
    per-tile aggregation of shared node pairs (tiles of both materials, both
    body shapes, and tiles that straddle two bodies)."""
    tl, w, g, _ = batched
    m = w["mesh"]
    h, rho = w["h"], 1e12
    rng = np.random.default_rng(32)
    g.tune_set(elem_agg=agg)
    assert g.tune_get()["elem_agg"] == agg
    vals = g.assemble_hessian(_dev(w["q_n"]), _dev(w["v"]), h, rho)
    g.tune_set(elem_agg=1)
    row_ptr, col = (a.cpu().numpy() for a in g.get_pattern()[:2])
    starts = np.concatenate([[0], np.cumsum([b.nn for b in w["meshes"]])])
    nodes = np.unique(np.concatenate([rng.integers(starts[b], starts[b + 1], size=2)
                                      for b in range(len(w["meshes"]))]
                                     + [m.fixed_nodes[:5]]))
    conn = m.conn.astype(np.int64)
    elems = np.nonzero(np.isin(conn, nodes).any(axis=1))[0]
    x = w["q_n"] + h * w["v"]
    Ke, _ = _oracle_elements(w, elems, x, w["v"], h, 1.0)
    rho0 = np.array([w["materials"][k]["rho0"] for k in np.asarray(w["mat_of_elem"])[elems]])
    Me = t10.element_mass(m.X, conn[elems], rho0) / h
    Kfull = Ke + np.einsum("eab,ik->eaibk", Me, np.eye(3)).reshape(len(elems), 30, 30)
    ref = {}
    for k, e in enumerate(elems):
        dofs = (3 * conn[e][:, None] + np.arange(3)).ravel()
        for r in range(30):
            if conn[e][r // 3] not in nodes:
                continue
            for s in range(30):
                key = (dofs[r], dofs[s])
                ref[key] = ref.get(key, 0.0) + Kfull[k, r, s]
    fixed = set(int(n) for n in m.fixed_nodes)
    for n in (int(n) for n in nodes):
        if int(n) in fixed:
            for d in range(3):
                ref[(3 * n + d, 3 * n + d)] += h * h * rho
    vals = vals.cpu().numpy().astype(np.float64)
    scale = max(abs(val) for (r, s), val in ref.items() if int(r) // 3 not in fixed)
    for (r, s), val in ref.items():
        lo, hi = row_ptr[r], row_ptr[r + 1]
        pos = lo + np.searchsorted(col[lo:hi], s)
        assert col[pos] == s
        penalty = r == s and int(r) // 3 in fixed
        tol = TOL_FP32 * (abs(val) if penalty else scale)
        assert abs(vals[pos] - val) <= tol, (r, s, vals[pos], val)
    # the pattern rows themselves are the oracle's (node adjacency lifted to DOFs)
    node_ptr, node_col = node_adjacency(conn[elems], m.nn)
    for n in nodes:
        expect = set(3 * node_col[node_ptr[n]:node_ptr[n + 1]])
        assert set(col[row_ptr[3 * n]:row_ptr[3 * n + 1]:3]) == expect


def test_batched_newton_step_from_rest(batched):
    """All 48 bodies from rest under gravity (the perturbed state of the
    workload is not a valid start: its Newton matrix is indefinite and Newton
    diverges from it), two captured FP32 steps; after each, the oracle's
    residual of the smallest box and the smallest cylinder at the GPU velocity
    (with the multipliers of the last inner loop) is below the global target."""
    tl, w, g, _ = batched
    m = w["mesh"]
    h, rho = w["h"], 1e12
    p = tl.params(h=h, rho_alm=rho, rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG, lin_adaptive=1, use_graph=1)
    q = _dev(m.X)
    v = torch.zeros_like(q)
    lam = torch.zeros(3 * len(m.fixed_nodes), dtype=torch.float64, device="cuda")
    nn_b = [b.nn for b in w["meshes"]]
    starts = np.concatenate([[0], np.cumsum(nn_b)])
    ne_starts = np.concatenate([[0], np.cumsum([b.ne for b in w["meshes"]])])
    picks = [min(range(0, 48, 2), key=lambda b: w["meshes"][b].ne),
             min(range(1, 48, 2), key=lambda b: w["meshes"][b].ne)]
    fixed_sorted = np.sort(np.asarray(m.fixed_nodes, dtype=np.int64))
    for step in range(2):
        v_new, q_new, st = g.newton_step(p, q, v, lam)
        assert st["converged"] == 1
        target = 1e-8 * st["g_ref"]
        lam_h = lam.cpu().numpy()
        vh, vnh, qnh = v_new.cpu().numpy(), v.cpu().numpy(), q.cpu().numpy()
        for b in picks:
            mb = w["meshes"][b]
            n0, n1 = starts[b], starts[b + 1]
            om = OracleMesh(mb.X, mb.conn, [w["materials"][b]], fixed_nodes=mb.fixed_nodes)
            sel = (fixed_sorted >= n0) & (fixed_sorted < n1)
            jj = np.nonzero(sel)[0]
            lam_b = lam_h.reshape(-1, 3)[jj].reshape(-1)
            vb = vh.reshape(-1, 3)[n0:n1].reshape(-1)
            qb = qnh.reshape(-1, 3)[n0:n1].reshape(-1)
            lam_inner = lam_b - rho * om.constraint(qb + h * vb)
            gb = om.residual(vb, qb, vnh.reshape(-1, 3)[n0:n1].reshape(-1), h, None, (0.0, 0.0, -9.81),
                             lam_inner, rho)
            assert np.linalg.norm(gb) <= 1.05 * target, (b, np.linalg.norm(gb), target)
            assert ne_starts[b + 1] - ne_starts[b] == mb.ne
        q, v = q_new.clone(), v_new.clone()
