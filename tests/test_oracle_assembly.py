"""Pins of the oracle's sparsity, assembly, residual and Newton step:
brute-force patterns, dense assembly, g = grad Phi (eq. cost), SPD Hessian,
the free-fall closed form and quadratic convergence."""
import numpy as np
import pytest

from oracle import assembly as asm
from oracle import newton as nt
from paper_2604_10357_gb300 import inputs

from helpers import first_frequencies

SVK = dict(kind="svk", E=1e7, nu=0.3, rho0=1000.0)
MR = dict(kind="mr", C10=5e5, C01=1e5, kappa=1e8, rho0=1000.0)
GRAV = (0.0, 0.0, -9.81)


@pytest.fixture(scope="module")
def tiny():
    m = inputs.box_t10(2, 1, 1, 0.2, 0.1, 0.1)
    rng = np.random.default_rng(30)
    q = inputs.uniform_perturbation(m, 0.02, rng)
    v = inputs.gaussian_velocity(m, 0.05, rng)
    return m, q, v


def test_pattern_brute_force(tiny):
    m, _, _ = tiny
    om = asm.OracleMesh(m.X, m.conn, [SVK], fixed_nodes=m.fixed_nodes)
    node_ptr, node_col, row_ptr, col = om.pattern()
    adj = np.zeros((m.nn, m.nn), bool)
    for c in m.conn:
        for a in c:
            for b in c:
                adj[a, b] = True
    dense = np.zeros((3 * m.nn, 3 * m.nn), bool)
    for r in range(3 * m.nn):
        dense[r, col[row_ptr[r]:row_ptr[r + 1]]] = True
        assert np.all(np.diff(col[row_ptr[r]:row_ptr[r + 1]]) > 0)
    assert np.array_equal(dense, np.kron(adj, np.ones((3, 3), bool)))
    assert np.array_equal(dense, dense.T)


def test_small_workload_nnz_by_counting(small_workload):
    """nnz of the 240-element box: 9 x (number of adjacent node pairs), the
    pairs counted with Python sets."""
    m = small_workload["mesh"]
    pairs = set()
    for c in m.conn.tolist():
        for a in c:
            for b in c:
                pairs.add((a, b))
    om = asm.OracleMesh(m.X, m.conn, [SVK])
    assert len(om.pattern()[3]) == 9 * len(pairs) == 102033


def test_slot_map_points_at_element_dofs(tiny):
    m, _, _ = tiny
    om = asm.OracleMesh(m.X, m.conn, [SVK])
    _, _, row_ptr, col = om.pattern()
    sm = asm.slot_map(m.conn, row_ptr, col)
    rows = np.repeat(np.arange(3 * m.nn), np.diff(row_ptr))
    dofs = asm.element_dofs(m.conn)
    for e in range(m.ne):
        for r in range(30):
            for s in range(30):
                p = sm[e, 30 * r + s]
                assert rows[p] == dofs[e, r] and col[p] == dofs[e, s]


@pytest.mark.parametrize("mat", [SVK, dict(MR, eta_d=1e3, lambda_d=1e3)], ids=["svk", "mr_kv"])
def test_hessian_values_equal_dense_assembly(tiny, mat):
    m, q, v = tiny
    om = asm.OracleMesh(m.X, m.conn, [mat], fixed_nodes=m.fixed_nodes)
    h, rho = 1e-3, 1e12
    Hs = om.hessian_matrix(q.ravel(), v.ravel(), h, rho).toarray()
    n = 3 * m.nn
    Hd = np.zeros((n, n))
    x = q + h * v
    Ke = om.element_tangents(x, v, alpha=h, beta=1.0)
    dofs = asm.element_dofs(m.conn)
    for e in range(m.ne):
        Hd[np.ix_(dofs[e], dofs[e])] += Ke[e]
        Hd[np.ix_(dofs[e], dofs[e])] += np.kron(om.Me[e], np.eye(3)) / h
    for r in om.fixed_dofs:
        Hd[r, r] += h * h * rho
    assert np.abs(Hs - Hd).max() <= 1e-13 * np.abs(Hd).max()
    assert np.abs(Hs - Hs.T).max() <= 1e-13 * np.abs(Hd).max()
    if mat["kind"] == "svk":
        np.linalg.cholesky(Hs)      # SPD (Sec. 4.4 remark: SVK elastic regime)
    # at the reference state H = M/h + D + penalty is SPD for any material
    H0 = om.hessian_matrix(m.X.ravel(), v.ravel(), h, rho).toarray()
    np.linalg.cholesky(H0)


def test_residual_is_gradient_of_augmented_cost(tiny):
    """eq. residual is grad_v of eq. cost (hyperelastic case): complex step of
    Phi_rho in every velocity component."""
    m, q, v = tiny
    om = asm.OracleMesh(m.X, m.conn, [SVK], fixed_nodes=m.fixed_nodes)
    rng = np.random.default_rng(31)
    h, rho = 1e-3, 1e6
    v_n = 0.05 * rng.normal(size=v.shape)
    f_ext = rng.normal(size=3 * m.nn)
    lam = rng.normal(size=3 * len(m.fixed_nodes))
    qn = q.copy()
    qn[m.fixed_nodes] += 1e-4 * rng.normal(size=(len(m.fixed_nodes), 3))   # violate c
    g = om.residual(v.ravel(), qn.ravel(), v_n.ravel(), h, f_ext, GRAV, lam, rho)
    gcs = np.zeros_like(g)
    for r in range(3 * m.nn):
        vc = v.ravel().astype(complex)
        vc[r] += 1e-30j
        gcs[r] = om.augmented_cost(vc, qn.ravel(), v_n.ravel(), h, f_ext, GRAV, lam, rho).imag / 1e-30
    assert np.abs(g - gcs).max() < 1e-10 * np.abs(g).max()


def test_gravity_load_row_sums(tiny):
    m, _, _ = tiny
    om = asm.OracleMesh(m.X, m.conn, [SVK])
    f = om.gravity_force(GRAV).reshape(-1, 3)
    V = m.extent[0] * m.extent[1] * m.extent[2]
    assert abs(f[:, 2].sum() - (-9.81 * 1000.0 * V)) < 1e-12 * 9.81 * 1000 * V
    assert np.abs(f[:, :2]).max() == 0.0


def test_free_fall_closed_form():
    """Unclamped, unstressed body at rest under gravity: one backward-Euler
    step gives exactly v = h g at every node (rigid translation)."""
    m = inputs.box_t10(2, 1, 1, 0.2, 0.1, 0.1, fixed_face_x0=False)
    om = asm.OracleMesh(m.X, m.conn, [dict(SVK, eta_d=1e3, lambda_d=1e3)])
    prm = nt.NewtonParams(h=1e-3, solver="dense", rtol=1e-12, atol=1e-12)
    out = nt.newton_step(om, m.X.ravel(), np.zeros(3 * m.nn), np.zeros(0), prm)
    expect = np.tile(np.array(GRAV) * 1e-3, m.nn)
    assert np.abs(out["v"] - expect).max() < 1e-11 * 9.81e-3


def test_newton_quadratic_convergence_and_solver_independence(small_workload):
    """Full Newton steps on the SVK cantilever: the normalised residual
    e_k = |g_k| / |g_0| of the first inner loop satisfies
    log e_{k+1} / log e_k >= 1.8 somewhere before the round-off floor
    (quadratic convergence), and the converged velocity does not depend on
    the linear solver (dense Cholesky vs sparse LU)."""
    w = small_workload
    m = w["mesh"]
    om = asm.OracleMesh(m.X, m.conn, [w["material"]], fixed_nodes=m.fixed_nodes)
    lam0 = np.zeros(3 * len(m.fixed_nodes))
    a = nt.newton_step(om, w["q_n"].ravel(), w["v"].ravel(), lam0,
                       nt.NewtonParams(h=w["h"], rtol=1e-8, solver="dense"))
    first = np.array(a["history"][:a["inner_iters"] + 1])
    first = first[: int(np.argmin(first[:6])) + 1]
    e = first / first[0]
    ratios = [np.log(e[k + 1]) / np.log(e[k]) for k in range(1, len(e) - 1)]
    assert e[-1] < 1e-9
    assert max(ratios) > 1.8, (first, ratios)
    b = nt.newton_step(om, w["q_n"].ravel(), w["v"].ravel(), lam0,
                       nt.NewtonParams(h=w["h"], rtol=1e-8, solver="splu"))
    assert a["converged"] and b["converged"]
    assert a["g_norm"] <= a["target"] and b["g_norm"] <= b["target"]
    assert np.linalg.norm(a["v"] - b["v"]) < 1e-9 * np.linalg.norm(a["v"])


def test_newton_line_search(small_workload):
    """Eq. armijo in the oracle's Newton step.  With h = 1e-3 every full step
    already decreases phi = |g|^2/2 enough, so the line search accepts a = 1
    throughout and the iterates equal those without it.  With h = 1e-2 the
    full step overshoots (|g| grows within the inner loop); with the line
    search every accepted step decreases |g| (the Armijo condition
    phi(a) <= (1 - 2 c1 a) phi(0) < phi(0)), and both runs reach the same
    converged velocity (each to |g| <= 1e-8 |g_ref|, which fixes v to ~1e-7
    here)."""
    w = small_workload
    m = w["mesh"]
    om = asm.OracleMesh(m.X, m.conn, [w["material"]], fixed_nodes=m.fixed_nodes)
    lam0 = np.zeros(3 * len(m.fixed_nodes))
    q, v = w["q_n"].ravel(), w["v"].ravel()
    run = lambda h, ls: nt.newton_step(om, q, v, lam0, nt.NewtonParams(h=h, rtol=1e-8, solver="dense",
                                                                        line_search=ls))
    a, b = run(1e-3, False), run(1e-3, True)
    assert a["history"] == b["history"] and np.array_equal(a["v"], b["v"])
    c, d = run(1e-2, False), run(1e-2, True)
    assert c["converged"] and d["converged"]
    hc, hd = np.array(c["history"]), np.array(d["history"])
    assert np.any(np.diff(hc[:c["inner_iters"] + 1]) > 0)          # the full step overshoots
    assert np.all(np.diff(hd[:d["inner_iters"] + 1]) < 0)          # monotone with the line search
    assert d["inner_iters"] > c["inner_iters"]                     # shortened steps
    assert c["g_norm"] <= c["target"] and d["g_norm"] <= d["target"]
    assert np.linalg.norm(c["v"] - d["v"]) <= 1e-6 * np.linalg.norm(c["v"])


def _tie_constraints(m):
    """General linear constraints on the tiny box: the first and the last
    corner node tied in x and z (2 rows, nodes not sharing an element), and
    one row mixing three DOFs of three nodes; b = C X (satisfied at rest)."""
    import scipy.sparse as sp
    n0, n1 = 0, m.nn - 1
    rows = [[(3 * n0, 1.0), (3 * n1, -1.0)],
            [(3 * n0 + 2, 1.0), (3 * n1 + 2, -1.0)],
            [(3 * 5 + 1, 0.5), (3 * 9 + 1, -2.0), (3 * 12 + 2, 1.5)]]
    ri, ci, vi = [], [], []
    for r, row in enumerate(rows):
        for c, val in row:
            ri.append(r), ci.append(c), vi.append(val)
    C = sp.csr_matrix((vi, (ri, ci)), shape=(len(rows), 3 * m.nn))
    return C, C @ m.X.ravel()


def test_general_constraints_pattern_hessian_and_gradient(tiny):
    """Sec. 4.2 with a general C_q: (i) the pattern is the element adjacency
    plus every node pair coupled by a row of C (brute force); (ii) the
    Hessian values equal a dense assembly of M/h + h K + D + h^2 rho C_q^T C_q
    with C_q = [clamp rows; C]; (iii) the residual stays the gradient of the
    augmented cost (complex step), so the h C_q^T (lambda + rho c) term and
    its Hessian are consistent."""
    m, q, v = tiny
    C, b = _tie_constraints(m)
    om = asm.OracleMesh(m.X, m.conn, [SVK], fixed_nodes=m.fixed_nodes, constraints=(C, b))
    # (i) pattern
    _, _, row_ptr, col = om.pattern()
    adj = np.zeros((m.nn, m.nn), bool)
    for c in m.conn:
        adj[np.ix_(c, c)] = True
    assert not adj[0, m.nn - 1]                          # the tie is a true fill-in
    Cd = C.toarray()
    for r in range(C.shape[0]):
        nodes = np.unique(np.nonzero(Cd[r])[0] // 3)
        adj[np.ix_(nodes, nodes)] = True
    dense = np.zeros((3 * m.nn, 3 * m.nn), bool)
    for r in range(3 * m.nn):
        dense[r, col[row_ptr[r]:row_ptr[r + 1]]] = True
    assert np.array_equal(dense, np.kron(adj, np.ones((3, 3), bool)))
    # (ii) Hessian
    h, rho = 1e-3, 1e6
    Hs = om.hessian_matrix(q.ravel(), v.ravel(), h, rho).toarray()
    om0 = asm.OracleMesh(m.X, m.conn, [SVK], fixed_nodes=m.fixed_nodes)
    H0 = om0.hessian_matrix(q.ravel(), v.ravel(), h, rho).toarray()
    assert np.abs(Hs - H0 - h * h * rho * (Cd.T @ Cd)).max() <= 1e-13 * np.abs(Hs).max()
    # (iii) gradient of the augmented cost
    rng = np.random.default_rng(33)
    v_n = 0.05 * rng.normal(size=v.shape)
    lam = rng.normal(size=3 * len(m.fixed_nodes) + C.shape[0])
    g = om.residual(v.ravel(), q.ravel(), v_n.ravel(), h, None, GRAV, lam, rho)
    assert np.abs(om.constraint(q.ravel() + h * v.ravel())[-C.shape[0]:]).max() > 0   # violated
    gcs = np.zeros_like(g)
    for r in range(3 * m.nn):
        vc = v.ravel().astype(complex)
        vc[r] += 1e-30j
        gcs[r] = om.augmented_cost(vc, q.ravel(), v_n.ravel(), h, None, GRAV, lam, rho).imag / 1e-30
    assert np.abs(g - gcs).max() < 1e-10 * np.abs(g).max()


def test_t10_cantilever_bending_matches_beam_theory():
    """A 2 m cantilever of 0.1 x 0.1 m section (20 x 2 x 2 hexes x 6 = 480 T10,
    E = 7e8, nu = 0) under a 1 N tip load shared by the tip-face nodes: the
    linear static tip deflection equals P L^3 / (3 E I) times the Timoshenko
    shear factor 1 + 6 I / (kappa A L^2) (kappa = 5/6, G = E / 2) within 0.1 %."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    E, Lx, a = 7e8, 2.0, 0.1
    mat = dict(kind="svk", E=E, nu=0.0, rho0=1000.0, eta_d=0.0, lambda_d=0.0)
    m = inputs.box_t10(20, 2, 2, Lx, a, a)
    om = asm.OracleMesh(m.X, m.conn, [mat], fixed_nodes=m.fixed_nodes)
    Ke = om.element_tangents(m.X, 0 * m.X, 1.0, 0.0)
    dofs = asm.element_dofs(om.conn)
    K = sp.coo_matrix((Ke.ravel(), (np.repeat(dofs, 30, axis=1).ravel(), np.tile(dofs, (1, 30)).ravel())),
                      shape=(3 * m.nn, 3 * m.nn)).tocsr()
    fixed = om.fixed_dofs
    free = np.setdiff1d(np.arange(3 * m.nn), fixed)
    tip = np.nonzero(np.isclose(m.X[:, 0], Lx))[0]
    f = np.zeros(3 * m.nn)
    f[3 * tip + 2] = 1.0 / len(tip)
    u = np.zeros(3 * m.nn)
    u[free] = spla.spsolve(K[free][:, free].tocsc(), f[free])
    I, A = a ** 4 / 12, a * a
    theory = Lx ** 3 / (3 * E * I) * (1.0 + 6.0 * I / (5.0 / 6.0 * A * Lx ** 2))
    assert abs(u[3 * tip + 2].mean() / theory - 1.0) < 1e-3


def test_t10_cantilever_first_frequency():
    """The consistent mass with the stiffness: the cantilever's first bending
    frequency is the Euler-Bernoulli 1.8751^2 sqrt(E I / (rho A L^4)) within
    0.3 % (shear and rotary inertia lower it by ~0.15 % here)."""
    E, rho, Lx, a = 7e8, 2700.0, 2.0, 0.1
    mat = dict(kind="svk", E=E, nu=0.0, rho0=rho, eta_d=0.0, lambda_d=0.0)
    m = inputs.box_t10(20, 2, 2, Lx, a, a)
    om = asm.OracleMesh(m.X, m.conn, [mat], fixed_nodes=m.fixed_nodes)
    w_eb = 1.8751040687 ** 2 * np.sqrt(E * a ** 4 / 12 / (rho * a * a * Lx ** 4))
    w = first_frequencies(om, m.nn, 10)
    assert np.all(np.abs(w / w_eb - 1.0) < 3e-3)       # the two transverse directions
