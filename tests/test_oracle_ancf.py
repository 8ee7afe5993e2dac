"""Pins of the oracle's ANCF3243 beam and ANCF3443 shell elements: the
Gauss-Legendre rules, the shape functions (textbook closed forms,
interpolation conditions, derivatives, affine completeness), the reference
geometry, the zero / rigid / homogeneous-deformation force checks, the
energy and complex-step derivatives, the exact mass and gravity weights, the
pattern counts, the paper's printed mesh statistics, the closed-form free
fall of one Newton step, and the Euler-Bernoulli deflection of a slender
cantilever."""
import os

import numpy as np
import pytest

from oracle import ancf
from oracle import element as el
from oracle import newton as nt
from paper_2604_10357_gb300 import inputs

from helpers import first_frequencies

SVK = dict(inputs.SVK_7E8)
MR = dict(kind="mr", C10=5e5, C01=1e5, kappa=1e8, rho0=1000.0, eta_d=0.0, lambda_d=0.0)
SVK_KV = dict(SVK, eta_d=1e3, lambda_d=1e3)
KINDS = [ancf.BEAM, ancf.SHELL]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ancf_mesh_statistics.txt")


def rotation(axis, angle):
    a = np.asarray(axis, float)
    a /= np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K


def small_mesh(kind):
    return inputs.beam_ancf3243(3) if kind == ancf.BEAM else inputs.shell_ancf3443(2, 2)


def affine_coefficients(mesh, A, b):
    """Coefficients of the reference body mapped by X -> A X + b."""
    E = mesh.E0 @ A.T
    E[0::4] += b
    return E


def one_element(kind, rng=None, rotate=False):
    """One element of the kind with its reference coefficients, optionally
    rotated rigidly (a general orientation of the reference frame)."""
    m = inputs.beam_ancf3243(1, L=0.3, W=0.05, H=0.08) if kind == ancf.BEAM else \
        inputs.shell_ancf3443(1, 1, Lx=0.4, Ly=0.3, H=0.05)
    if rotate:
        R = rotation((1.0, 2.0, 3.0), 0.6)
        m.E0 = affine_coefficients(m, R, np.array([0.1, -0.2, 0.3]))
    return m


# ---------------------------------------------------------------------------
# quadrature
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_gauss_legendre_exactness(n):
    """n points integrate xi^k exactly on [-1, 1] for k <= 2n - 1, not for k = 2n."""
    x, w = ancf.gauss_legendre(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-14
    assert abs(np.sum(w * x ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-6


def test_element_rules_sizes():
    """12 points for the beam and 48 for the shell (Sec. 4.3); weights sum to 8."""
    for kind, nq in [(ancf.BEAM, 12), (ancf.SHELL, 48)]:
        p, w = ancf.element_rule(kind)
        assert p.shape == (nq, 3) and abs(w.sum() - 8.0) < 1e-13


# ---------------------------------------------------------------------------
# shape functions
# ---------------------------------------------------------------------------

def test_beam_shape_matches_textbook_hermite():
    """Axial functions = the cubic Hermite polynomials in xi (values and x-slopes
    at the ends), cross-section functions = (1 -+ xi)/2 times y or z."""
    L, W, H = 0.3, 0.05, 0.08
    rng = np.random.default_rng(1)
    for xi, eta, zeta in rng.uniform(-1, 1, size=(20, 3)):
        S, _ = ancf.beam_shape((xi, eta, zeta), (L, W, H))
        ref = [(2 - 3 * xi + xi ** 3) / 4, L * (1 - xi - xi ** 2 + xi ** 3) / 8, W * (1 - xi) * eta / 4,
               H * (1 - xi) * zeta / 4, (2 + 3 * xi - xi ** 3) / 4, L * (-1 - xi + xi ** 2 + xi ** 3) / 8,
               W * (1 + xi) * eta / 4, H * (1 + xi) * zeta / 4]
        np.testing.assert_allclose(S, ref, atol=1e-15)


def test_shell_surface_functions_match_adini_closed_form():
    """The position functions of the incomplete bicubic space equal the
    closed-form rectangle functions (1/8)(1 + xc xi)(1 + yc eta)(2 + xc xi +
    yc eta - xi^2 - eta^2), and the slope functions their Hermite analogues."""
    L, W, H = 0.4, 0.3, 0.05
    rng = np.random.default_rng(2)
    for xi, eta, zeta in rng.uniform(-1, 1, size=(20, 3)):
        S, _ = ancf.shell_shape((xi, eta, zeta), (L, W, H))
        for c, (xc, yc) in enumerate(ancf.SHELL_CORNERS):
            a, b = 1 + xc * xi, 1 + yc * eta
            assert abs(S[4 * c] - a * b * (2 + xc * xi + yc * eta - xi ** 2 - eta ** 2) / 8) < 1e-14
            assert abs(S[4 * c + 1] - L / 16 * xc * a * a * (xc * xi - 1) * b) < 1e-14
            assert abs(S[4 * c + 2] - W / 16 * yc * b * b * (yc * eta - 1) * a) < 1e-14
            assert abs(S[4 * c + 3] - H / 8 * zeta * a * b) < 1e-14


@pytest.mark.parametrize("kind", KINDS)
def test_shape_derivatives_complex_step(kind):
    """dS/d(xi, eta, zeta) equals the complex-step derivative of S."""
    dims = (0.3, 0.2, 0.07)
    rng = np.random.default_rng(3)
    hstep = 1e-30
    for pt in rng.uniform(-1, 1, size=(5, 3)):
        _, dS = ancf.shape(kind, pt, dims)
        for j in range(3):
            p = pt.astype(complex)
            p[j] += 1j * hstep
            Sc, _ = ancf.shape(kind, p, dims)
            np.testing.assert_allclose(dS[:, j], Sc.imag / hstep, rtol=0, atol=1e-13)


@pytest.mark.parametrize("kind", KINDS)
def test_interpolation_conditions_at_nodes(kind):
    """At each node (mid-plane / axis), the position function of that node is
    1 and every other function 0; the x- and y-slope functions have unit slope
    there in their direction (d/dx = (2/L) d/dxi, d/dy = (2/W) d/deta) and zero
    slopes elsewhere; r_z's function has unit z-slope (d/dz = (2/H) d/dzeta)."""
    L, W, H = 0.3, 0.2, 0.07
    if kind == ancf.BEAM:
        nodes = [(-1.0, 0.0), (1.0, 0.0)]
        pts = [(x, 0.0, 0.0) for x, _ in nodes]
    else:
        pts = [(x, y, 0.0) for x, y in ancf.SHELL_CORNERS]
    for n, pt in enumerate(pts):
        S, dS = ancf.shape(kind, pt, (L, W, H))
        grad = dS * np.array([2 / L, 2 / W, 2 / H])
        for k in range(4):
            e = np.zeros(len(S))
            e[4 * n + k] = 1.0
            if k == 0:
                np.testing.assert_allclose(S, e, atol=1e-14)
            else:
                np.testing.assert_allclose(grad[:, k - 1], e, atol=1e-13)


@pytest.mark.parametrize("kind", KINDS)
def test_affine_completeness(kind):
    """Coefficients of an affine map reproduce it exactly everywhere in the
    element: sum_a S_a(xi) e_a = A r0(xi) + b."""
    m = one_element(kind, rotate=True)
    rng = np.random.default_rng(4)
    A = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
    b = rng.standard_normal(3)
    E = affine_coefficients(m, A, b)
    c = m.conn[0]
    for pt in rng.uniform(-1, 1, size=(10, 3)):
        S, _ = ancf.shape(kind, pt, m.dims[0])
        r0 = S @ m.E0[c]
        np.testing.assert_allclose(S @ E[c], A @ r0 + b, atol=1e-13)


@pytest.mark.parametrize("kind", KINDS)
def test_reference_geometry_rectangular(kind):
    """A rigidly placed rectangular element: grad_X S maps the reference field
    to F = I, det J0 = L W H / 8, and sum_q w_q det J0 = L W H."""
    m = one_element(kind, rotate=True)
    gradS, detJ, wJ = ancf.reference_geometry(kind, m.E0, m.conn, m.dims)
    L, W, H = m.dims[0]
    np.testing.assert_allclose(detJ, L * W * H / 8, rtol=1e-13)
    assert abs(wJ.sum() - L * W * H) < 1e-14 * L * W * H
    F = el.kinematics(m.E0[m.conn], gradS)
    np.testing.assert_allclose(F, np.broadcast_to(np.eye(3), F.shape), atol=1e-13)


# ---------------------------------------------------------------------------
# force and tangent
# ---------------------------------------------------------------------------

def _oracle(kind, mesh, mat):
    return ancf.OracleAncfMesh(kind, mesh.E0, mesh.conn, mesh.dims, [mat], fixed_nodes=mesh.fixed_nodes)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("mat", [SVK, MR], ids=["svk", "mr"])
def test_zero_force_reference_and_rigid_motion(kind, mat):
    m = small_mesh(kind)
    om = _oracle(kind, m, mat)
    zero_v = np.zeros_like(m.E0)
    f0 = om.element_forces(m.E0, zero_v)
    assert np.abs(f0).max() < 1e-6
    R = rotation((1.0, 2.0, 3.0), np.deg2rad(37.0))
    E = affine_coefficients(m, R, np.array([0.3, -1.0, 2.0]))
    scale = np.abs(om.element_forces(affine_coefficients(m, np.eye(3) + 1e-3, np.zeros(3)), zero_v)).max()
    assert np.abs(om.element_forces(E, zero_v)).max() < 1e-9 * scale


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("mat", [SVK, MR, SVK_KV], ids=["svk", "mr", "svk_kv"])
def test_homogeneous_deformation_virtual_work(kind, mat):
    """Patch test in weak form: under q = A X + b (and v = B_v X) the stress
    is uniform, so for any affine virtual displacement du = B X + c the
    element forces do the work sum_a de_a . f_a = V (P : B) exactly."""
    m = one_element(kind, rotate=True)
    om = _oracle(kind, m, mat)
    rng = np.random.default_rng(5)
    A = np.eye(3) + 0.05 * rng.standard_normal((3, 3))
    Bv = 0.1 * rng.standard_normal((3, 3))
    E = affine_coefficients(m, A, rng.standard_normal(3))
    V = affine_coefficients(m, Bv, np.zeros(3))
    fe = om.element_forces(E, V)[0]
    gradS = om.gradN[0]
    F = el.kinematics(E[m.conn], om.gradN)[0]
    np.testing.assert_allclose(F, np.broadcast_to(A, F.shape), atol=1e-12)
    P = el.stresses(A[None], (Bv @ np.eye(3))[None], mat, False)["P"][0]
    vol = np.prod(m.dims[0])
    for _ in range(3):
        B = rng.standard_normal((3, 3))
        dE = affine_coefficients(m, B, rng.standard_normal(3))[m.conn[0]]
        work = np.sum(dE * fe)
        assert abs(work - vol * np.sum(P * B)) < 1e-11 * vol * np.abs(P).max() * np.abs(B).max() * 10


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("mat", [SVK, MR], ids=["svk", "mr"])
def test_force_is_energy_gradient(kind, mat):
    """The elastic element force equals the complex-step gradient of the
    element energy sum_q w_q J0 W(F_q)."""
    m = one_element(kind, rotate=True)
    om = _oracle(kind, m, mat)
    rng = np.random.default_rng(6)
    x = m.E0 + 0.02 * rng.standard_normal(m.E0.shape)
    fe = om.element_forces(x, np.zeros_like(x))[0]
    hstep = 1e-30
    g = np.zeros_like(x)
    for a in range(x.shape[0]):
        for i in range(3):
            xc = x.astype(complex)
            xc[a, i] += 1j * hstep
            g[a, i] = el.element_energy(xc[m.conn], om.gradN, om.wJ0, mat)[0].imag / hstep
    np.testing.assert_allclose(fe, g[m.conn[0]], rtol=1e-12, atol=1e-12 * np.abs(g).max())


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("mat", [SVK, MR, SVK_KV], ids=["svk", "mr", "svk_kv"])
def test_tangent_complex_step_and_symmetry(kind, mat):
    """K (alpha = 1, beta = 0) is the complex-step Jacobian of f in x (exactly
    for hyperelastic laws; with Kelvin-Voigt the dropped non-symmetric part is
    what differs, so that case checks D against d f / d v instead) and K is
    symmetric."""
    m = one_element(kind, rotate=True)
    om = _oracle(kind, m, mat)
    rng = np.random.default_rng(7)
    x = m.E0 + 0.02 * rng.standard_normal(m.E0.shape)
    v = 0.1 * rng.standard_normal(m.E0.shape)
    c = m.conn[0]
    nd = 3 * len(c)
    hstep = 1e-30
    kv = mat.get("eta_d", 0.0) != 0.0
    K = om.element_tangents(x, v if kv else 0 * v, alpha=0.0 if kv else 1.0, beta=1.0 if kv else 0.0)[0]
    J = np.zeros((nd, nd))
    for a in range(len(c)):
        for i in range(3):
            if kv:
                vc = v.astype(complex)
                vc[c[a], i] += 1j * hstep
                fc = om.element_forces(x.astype(complex), vc)[0]
            else:
                xc = x.astype(complex)
                xc[c[a], i] += 1j * hstep
                fc = om.element_forces(xc, np.zeros_like(xc))[0]
            J[:, 3 * a + i] = fc.reshape(-1).imag / hstep
    np.testing.assert_allclose(K, J, rtol=0, atol=1e-11 * np.abs(J).max())
    np.testing.assert_allclose(K, K.T, rtol=0, atol=1e-13 * np.abs(K).max())


# ---------------------------------------------------------------------------
# mass and gravity
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", KINDS)
def test_mass_exact_and_spd(kind):
    """The mass rule is exact (it agrees with a 7-point rule in every
    direction); constant fields carry the total mass rho V; the element
    mass is symmetric positive definite."""
    m = one_element(kind, rotate=True)
    rho = 2700.0
    Me, We = ancf.element_mass(kind, m.E0, m.conn, m.dims, np.array([rho]))
    pts, wts = ancf.product_rule(7, 7, 7)
    ref = np.zeros_like(Me[0])
    c = m.conn[0]
    for pt, w in zip(pts, wts):
        S, dS = ancf.shape(kind, pt, m.dims[0])
        ref += rho * w * np.linalg.det(m.E0[c].T @ dS) * np.outer(S, S)
    np.testing.assert_allclose(Me[0], ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    vol = np.prod(m.dims[0])
    pos = np.arange(0, len(c), 4)
    assert abs(Me[0][np.ix_(pos, pos)].sum() - rho * vol) < 1e-12 * rho * vol
    assert abs(We[0][pos].sum() - rho * vol) < 1e-12 * rho * vol
    assert np.linalg.eigvalsh(Me[0]).min() > 0.0


def test_beam_gravity_weights_closed_form():
    """int rho S_a dV for the beam: rho V / 2 at each end position, +-rho W H
    L^2 / 12 at the axial slopes, 0 at the transverse gradients (the
    cross-section is symmetric)."""
    m = one_element(ancf.BEAM)
    L, W, H = m.dims[0]
    rho = 2700.0
    _, We = ancf.element_mass(ancf.BEAM, m.E0, m.conn, m.dims, np.array([rho]))
    ref = rho * np.array([L * W * H / 2, W * H * L * L / 12, 0, 0, L * W * H / 2, -W * H * L * L / 12, 0, 0])
    np.testing.assert_allclose(We[0], ref, atol=1e-15 * rho)


# ---------------------------------------------------------------------------
# mesh level: pattern, the paper's mesh statistics, free fall
# ---------------------------------------------------------------------------

def test_pattern_counts_closed_form():
    """Coefficient adjacency: a chain of ne beam elements couples 64 ne - 16
    (ne - 1) coefficient pairs; an nx x ny shell grid 16 (3 nx + 1)(3 ny + 1)."""
    for ne in (1, 2, 7):
        m = inputs.beam_ancf3243(ne)
        om = _oracle(ancf.BEAM, m, SVK)
        node_ptr, node_col, row_ptr, col = om.pattern()
        assert node_ptr[-1] == 64 * ne - 16 * (ne - 1)
        assert row_ptr[-1] == 9 * node_ptr[-1]
    for nx, ny in ((1, 1), (3, 2)):
        m = inputs.shell_ancf3443(nx, ny)
        om = _oracle(ancf.SHELL, m, SVK)
        assert om.pattern()[0][-1] == 16 * (3 * nx + 1) * (3 * ny + 1)


def _golden_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, res, dofs, nodes, elems, cons = line.split()
                rows.append((k, res, int(dofs), int(nodes), int(elems), int(cons)))
    return rows


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: f"{r[0]}-{r[1]}")
def test_generators_match_paper_mesh_statistics(row):
    """The beam and shell generators reproduce the DOF, node, element and
    constrained-DOF counts the paper prints for each resolution."""
    kind, _, dofs, nodes, elems, cons = row
    if kind == ancf.BEAM:
        m = inputs.beam_ancf3243(elems)
    else:
        n = int(round(np.sqrt(elems)))
        m = inputs.shell_ancf3443(n, n)
    assert (3 * m.nn, m.nphys, m.ne, 3 * len(m.fixed_nodes)) == (dofs, nodes, elems, cons)


@pytest.mark.parametrize("kind", KINDS)
def test_free_fall_closed_form(kind):
    """An unclamped, unstressed body at rest: one Newton step under gravity
    gives v = h g on every position coefficient and 0 on every gradient
    coefficient (the residual vanishes there exactly: the mass applied to a
    uniform translation returns the gravity weights)."""
    m = small_mesh(kind)
    om = ancf.OracleAncfMesh(kind, m.E0, m.conn, m.dims, [SVK])
    q = m.E0.copy()
    v = np.zeros_like(q)
    r = nt.newton_step(om, q, v, np.zeros(0), nt.NewtonParams(h=1e-3, rtol=1e-12, solver="dense"))
    ref = np.zeros_like(q)
    ref[0::4] = 1e-3 * np.asarray(inputs.GRAVITY)
    np.testing.assert_allclose(r["v"].reshape(-1, 3), ref, atol=1e-12)


def _static_tip_deflection(kind, m, mat, fe):
    """Linear static solve K u = f at the reference state (the element
    tangents assembled, clamped coefficients eliminated)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    om = ancf.OracleAncfMesh(kind, m.E0, m.conn, m.dims, [mat], fixed_nodes=m.fixed_nodes)
    Ke = om.element_tangents(m.E0, 0 * m.E0, 1.0, 0.0)
    nd = 3 * m.conn.shape[1]
    dofs = (3 * m.conn[:, :, None] + np.arange(3)).reshape(m.ne, nd)
    K = sp.coo_matrix((Ke.ravel(), (np.repeat(dofs, nd, axis=1).ravel(), np.tile(dofs, (1, nd)).ravel())),
                      shape=(3 * m.nn, 3 * m.nn)).tocsr()
    fixed = (3 * m.fixed_nodes[:, None] + np.arange(3)).ravel()
    free = np.setdiff1d(np.arange(3 * m.nn), fixed)
    u = np.zeros(3 * m.nn)
    u[free] = spla.spsolve(K[free][:, free].tocsc(), fe.ravel()[free])
    return u.reshape(-1, 3)


@pytest.mark.parametrize("kind", KINDS)
def test_cantilever_bending_matches_euler_bernoulli(kind):
    """A slender cantilever (4 m long, 0.1 m deep, E = 7e8, nu = 0 so no
    Poisson stiffening) under a small tip load deflects by P L^3 / (3 E I):
    the beam's cubic Hermite axis and the shell's incomplete bicubic surface
    carry bending, within 0.1 % at 20 elements along the span (shear
    deformation is what remains)."""
    E = 7e8
    mat = dict(kind="svk", E=E, nu=0.0, rho0=2700.0, eta_d=0.0, lambda_d=0.0)
    if kind == ancf.BEAM:
        m = inputs.beam_ancf3243(20, L=0.2, W=0.1, H=0.1)
        fe = np.zeros_like(m.E0)
        fe[4 * 20, 2] = 1.0
        u = _static_tip_deflection(kind, m, mat, fe)
        tip = [u[4 * 20, 2]]
        I = 0.1 * 0.1 ** 3 / 12
    else:
        m = inputs.shell_ancf3443(20, 1, Lx=4.0, Ly=0.2, H=0.1)
        fe = np.zeros_like(m.E0)
        edge = np.nonzero(np.isclose(m.phys_x[:, 0], 4.0))[0]
        fe[4 * edge, 2] = 0.5
        u = _static_tip_deflection(kind, m, mat, fe)
        tip = u[4 * edge, 2]
        I = 0.2 * 0.1 ** 3 / 12
    eb = 4.0 ** 3 / (3 * E * I)
    for d in tip:
        assert abs(d / eb - 1.0) < 1e-3


@pytest.mark.parametrize("kind", KINDS)
def test_cantilever_first_frequency(kind):
    """Exact mass with the stiffness: the first bending frequency of a 2 m
    cantilever (E = 7e8, rho = 2700, nu = 0; beam 0.1 x 0.1 section in 10
    elements, shell strip 0.2 m wide and 0.1 m thick in 20) is the
    Euler-Bernoulli 1.8751^2 sqrt(E I / (rho A L^4)) within 0.3 %."""
    E, rho = 7e8, 2700.0
    mat = dict(kind="svk", E=E, nu=0.0, rho0=rho, eta_d=0.0, lambda_d=0.0)
    if kind == ancf.BEAM:
        m = inputs.beam_ancf3243(10, L=0.2, W=0.1, H=0.1)
        I, A = 0.1 ** 4 / 12, 0.01
    else:
        m = inputs.shell_ancf3443(20, 1, Lx=2.0, Ly=0.2, H=0.1)
        I, A = 0.2 * 0.1 ** 3 / 12, 0.02
    om = ancf.OracleAncfMesh(kind, m.E0, m.conn, m.dims, [mat], fixed_nodes=m.fixed_nodes)
    w_eb = 1.8751040687 ** 2 * np.sqrt(E * I / (rho * A * 2.0 ** 4))
    w = first_frequencies(om, m.nn, ancf.nen_of(kind), k=1)
    assert abs(w[0] / w_eb - 1.0) < 3e-3
