"""Parity at full size, in the launch configuration bench.py times (the
autotuner's choice): the 960,000-element box (SVK + Kelvin-Voigt, FP32
element form) and the 103,680-element cantilever (SVK, both precisions).
The oracle evaluates sampled elements and sampled CSR rows one by one; the
internal force of the whole mesh is self-equilibrated."""
import numpy as np
import pytest

from oracle import element as oelem
from oracle import t10
from paper_2604_10357_gb300 import inputs

from helpers import TOL_FP32, TOL_FP64, tangent_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _tl():
    from paper_2604_10357_gb300 import build, tl
    build.build()
    return tl


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(-1), device="cuda")


def _oracle_elements(X, conn, mat, idx, x, v, alpha, beta):
    c = conn[idx].astype(np.int64)
    gradN, _, wJ0 = t10.reference_geometry(X, c)
    return oelem.element_tangent(x[c], v[c], gradN, wJ0, mat, alpha, beta)


def _check_rows(g, mesh, mat, q_n, v, h, rho, nodes, tol, vals):
    """Every entry of the CSR rows of `nodes` against the oracle's element
    matrices (M_e / h + h K_t + D) summed over the elements at each node."""
    row_ptr, col = (a.cpu().numpy() for a in g.get_pattern()[:2])
    conn = mesh.conn.astype(np.int64)
    elems = np.nonzero(np.isin(conn, nodes).any(axis=1))[0]
    x = q_n + h * v
    Ke = _oracle_elements(mesh.X, conn, mat, elems, x, v, h, 1.0)
    Me = t10.element_mass(mesh.X, conn[elems], np.full(len(elems), mat["rho0"])) / h
    Kfull = Ke + np.einsum("eab,ik->eaibk", Me, np.eye(3)).reshape(len(elems), 30, 30)
    node_set = set(int(n) for n in nodes)
    ref = {}
    for k, e in enumerate(elems):
        dofs = (3 * conn[e][:, None] + np.arange(3)).ravel()
        for r in range(30):
            if int(conn[e][r // 3]) not in node_set:
                continue
            for s in range(30):
                key = (int(dofs[r]), int(dofs[s]))
                ref[key] = ref.get(key, 0.0) + Kfull[k, r, s]
    fixed = set(int(n) for n in mesh.fixed_nodes)
    for n in node_set & fixed:
        for d in range(3):
            ref[(3 * n + d, 3 * n + d)] += h * h * rho
    scale = max(abs(val) for (r, s), val in ref.items() if r // 3 not in fixed)
    for (r, s), val in ref.items():
        lo, hi = row_ptr[r], row_ptr[r + 1]
        pos = lo + np.searchsorted(col[lo:hi], s)
        assert pos < hi and col[pos] == s
        penalty = r == s and r // 3 in fixed
        assert abs(vals[pos] - val) <= tol * (abs(val) if penalty else scale), (r, s, vals[pos], val)


@pytest.mark.parametrize("case", ["box960k_fp32", "cantilever_fp32", "cantilever_fp64"])
def test_full_size_sampled_parity(case):
    tl = _tl()
    if case.startswith("box960k"):
        w = inputs.workload_large_svk_kv(scale=1.0)
        q_n, v = w["q_n"], w["v"]
    else:
        w = inputs.workload_warm_start_svk()
        rng = np.random.default_rng(71)
        q_n = inputs.uniform_perturbation(w["mesh"], 0.01, rng)
        v = inputs.gaussian_velocity(w["mesh"], 0.05, rng)
    m, mat, h, rho = w["mesh"], w["material"], w["h"], 1e12
    prec = tl.TL_FP64 if case.endswith("fp64") else tl.TL_FP32_ELEM
    tol = TOL_FP64 if prec == tl.TL_FP64 else TOL_FP32
    g = tl.Mesh(m.X, m.conn, [mat], precision=prec)
    g.build_pattern(m.fixed_nodes)
    qd, vd = _dev(q_n), _dev(v)
    g.autotune(qd, vd, h, reps=1)                       # the launch shapes bench.py times
    f = torch.empty(3 * m.nn, dtype=torch.float64, device="cuda")
    vals = g.assemble_hessian(qd, vd, h, rho, f_int=f).cpu().numpy().astype(np.float64)
    g.sync()
    # the whole mesh's internal force sums to zero (element forces are self-equilibrated)
    fb = f.view(-1, 3).cpu().numpy()
    assert np.linalg.norm(fb.sum(0)) <= (1e-12 if prec == tl.TL_FP64 else 1e-7) * np.abs(fb).sum()
    rng = np.random.default_rng(72)
    # sampled element tangents (first, last and random elements)
    idx = np.unique(np.concatenate([[0, m.ne - 1], rng.integers(0, m.ne, size=62)]))
    K = g.eval_tangent(qd, vd, h, h, 1.0)
    Ks = K.view(m.ne, 900)[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    del K
    x = q_n + h * v
    assert tangent_error(Ks, _oracle_elements(m.X, m.conn, mat, idx, x, v, h, 1.0)) < tol
    # sampled CSR rows: random interior nodes and clamped nodes
    nodes = np.unique(np.concatenate([rng.integers(0, m.nn, size=12), np.asarray(m.fixed_nodes)[:4]]))
    _check_rows(g, m, mat, q_n, v, h, rho, nodes, tol, vals)
