"""Pins of the oracle's element force and tangent (eq. fint_local,
eq. tangent_block): invariants, the patch test, symmetry, finite-difference
and complex-step derivatives, and the exactly integrated linear stiffness."""
import itertools
from fractions import Fraction
from math import factorial

import numpy as np
import pytest

from oracle import assembly as asm
from oracle import element as el
from oracle import materials as mats
from oracle import t10
from paper_2604_10357_gb300 import inputs

SVK = dict(kind="svk", E=1e7, nu=0.3, rho0=1000.0)
MR = dict(kind="mr", C10=5e5, C01=1e5, kappa=1e8, rho0=1000.0)
SVK_KV = dict(SVK, eta_d=1e3, lambda_d=1e3)
MR_KV = dict(MR, eta_d=1e3, lambda_d=2e3)


def rotation(axis, angle):
    a = np.asarray(axis, float)
    a /= np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K


@pytest.fixture(scope="module")
def box():
    m = inputs.box_t10(3, 2, 2, 0.3, 0.2, 0.2)
    return m


def _om(m, mat):
    return asm.OracleMesh(m.X, m.conn, [mat], fixed_nodes=m.fixed_nodes)


@pytest.mark.parametrize("mat", [SVK, MR, SVK_KV, MR_KV], ids=["svk", "mr", "svk_kv", "mr_kv"])
def test_zero_force_reference_and_rigid_motion(box, mat):
    om = _om(box, mat)
    f0 = om.internal_force(box.X.ravel(), np.zeros(box.nn * 3), 0.0)
    scale = 1e7 * 0.1 ** 2
    assert np.abs(f0).max() < 1e-12 * scale
    R = rotation((1, 2, 3), np.deg2rad(37.0))
    x = box.X @ R.T + np.array([0.3, -0.2, 0.1])
    # rigid spin velocity v = w x (x - c): Fdot = W F, Edot = 0
    w = np.array([0.4, -1.0, 2.0])
    v = np.cross(w[None, :], x - x.mean(0))
    f = om.internal_force(x.ravel(), v.ravel(), 0.0)
    assert np.abs(f).max() < 1e-9 * scale


@pytest.mark.parametrize("mat", [SVK, MR_KV], ids=["svk", "mr_kv"])
def test_force_and_moment_balance(box, mat):
    rng = np.random.default_rng(20)
    om = _om(box, mat)
    x = box.X + 0.01 * rng.normal(size=box.X.shape)
    v = 0.1 * rng.normal(size=box.X.shape)
    f = om.internal_force(x.ravel(), v.ravel(), 0.0).reshape(-1, 3)
    scale = np.abs(f).max()
    assert np.abs(f.sum(0)).max() < 1e-12 * scale * box.nn
    assert np.abs(np.cross(x, f).sum(0)).max() < 1e-12 * scale * box.nn


def _boundary_triangles(conn):
    """Faces of the T10 mesh not shared by two elements, as 6-node triangles
    (3 corners, then the midsides of edges (0,1), (1,2), (0,2))."""
    faces = {}
    corner_sets = ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))
    edge_mid = {(0, 1): 4, (1, 2): 5, (0, 2): 6, (0, 3): 7, (1, 3): 8, (2, 3): 9}
    for e, c in enumerate(conn):
        for fc in corner_sets:
            key = tuple(sorted(int(c[i]) for i in fc))
            a, b, d = fc
            tri = (c[a], c[b], c[d], c[edge_mid[(a, b)]], c[edge_mid[(b, d)]], c[edge_mid[(a, d)]])
            opp = [i for i in range(4) if i not in fc][0]
            faces.setdefault(key, []).append((tri, c[opp]))
    return [v[0] for v in faces.values() if len(v) == 1]


@pytest.mark.parametrize("mat", [SVK, MR], ids=["svk", "mr"])
def test_patch_test_affine_motion(box, mat):
    """q = (I + A) X + b gives a uniform P.  Then f_a = P int grad N_a dV
    = P oint N_a N dA (divergence theorem; exact under the degree-3 rule):
    interior nodes get zero, and on each 6-node boundary triangle of area A_t
    the corners get 0 and every midside (P N) A_t / 3."""
    rng = np.random.default_rng(21)
    A = rng.normal(size=(3, 3))
    A *= 1e-2 / np.linalg.norm(A)
    F = np.eye(3) + A
    x = box.X @ F.T + np.array([1.0, 2.0, 3.0])
    om = _om(box, mat)
    f = om.internal_force(x.ravel(), np.zeros(box.nn * 3), 0.0).reshape(-1, 3)
    P, _, _ = mats.elastic_stress_and_tangent(F, mat, want_tangent=False)
    expect = np.zeros_like(f)
    for tri, opp in _boundary_triangles(box.conn):
        p0, p1, p2 = box.X[tri[0]], box.X[tri[1]], box.X[tri[2]]
        nrm = np.cross(p1 - p0, p2 - p0)
        area = 0.5 * np.linalg.norm(nrm)
        nrm /= np.linalg.norm(nrm)
        if nrm @ (box.X[opp] - p0) > 0:     # make it outward
            nrm = -nrm
        for mid in tri[3:]:
            expect[mid] += (P @ nrm) * area / 3.0
    assert np.abs(f - expect).max() < 1e-9 * np.abs(expect).max()


def _one_element(rng, distort=0.05):
    m = inputs.box_t10(1, 1, 1, 1.0, 1.0, 1.0)
    conn = m.conn[:1]
    X = m.X
    x = X + distort * rng.normal(size=X.shape)
    v = rng.normal(size=X.shape)
    gradN, _, wJ0 = t10.reference_geometry(X, conn)
    return X, conn, x, v, gradN, wJ0


@pytest.mark.parametrize("mat", [SVK, MR, SVK_KV, MR_KV], ids=["svk", "mr", "svk_kv", "mr_kv"])
def test_tangent_matches_complex_step_of_force(mat):
    """alpha K_t + beta D against complex-step derivatives of f_e in x and v.
    For hyperelastic materials K_t = df/dx exactly; with Kelvin-Voigt the
    material part of dP_v/dF at fixed Fdot is left out by design, so the pin
    there is taken with Fdot = 0 (v = 0), where that term vanishes."""
    rng = np.random.default_rng(22)
    X, conn, x, v, gradN, wJ0 = _one_element(rng)
    has_kv = "eta_d" in mat
    if has_kv:
        v = np.zeros_like(v)
    xe, ve = x[conn], v[conn]
    K = el.element_tangent(xe, ve, gradN, wJ0, mat, 1.0, 0.0)[0]
    Kcs = np.zeros((30, 30))
    Dcs = np.zeros((30, 30))
    hstep = 1e-30
    for s in range(30):
        b, k = divmod(s, 3)
        dx = np.zeros((1, 10, 3), complex)
        dx[0, b, k] = 1j * hstep
        Kcs[:, s] = el.element_force(xe + dx, ve.astype(complex), gradN, wJ0, mat).imag.reshape(30) / hstep
        Dcs[:, s] = el.element_force(xe.astype(complex), ve + dx, gradN, wJ0, mat).imag.reshape(30) / hstep
    assert np.abs(K - Kcs).max() < 1e-12 * np.abs(K).max()
    if has_kv:
        D = el.element_tangent(xe, ve, gradN, wJ0, mat, 0.0, 1.0)[0]
        assert np.abs(D - Dcs).max() < 1e-12 * np.abs(D).max()
        assert np.abs(D - D.T).max() < 1e-14 * np.abs(D).max()
        assert np.linalg.eigvalsh(D).min() > -1e-10 * np.abs(D).max()


@pytest.mark.parametrize("mat", [SVK, MR], ids=["svk", "mr"])
def test_tangent_symmetric_and_central_fd(mat):
    rng = np.random.default_rng(23)
    X, conn, x, v, gradN, wJ0 = _one_element(rng, 0.1)
    xe, ve = x[conn], np.zeros_like(x[conn])
    K = el.element_tangent(xe, ve, gradN, wJ0, mat)[0]
    assert np.abs(K - K.T).max() < 1e-14 * np.abs(K).max() * 30
    delta = 1e-6
    Kfd = np.zeros((30, 30))
    for s in range(30):
        b, k = divmod(s, 3)
        dx = np.zeros_like(xe)
        dx[0, b, k] = delta
        Kfd[:, s] = (el.element_force(xe + dx, ve, gradN, wJ0, mat)
                     - el.element_force(xe - dx, ve, gradN, wJ0, mat)).reshape(30) / (2 * delta)
    assert np.abs(K - Kfd).max() < 1e-7 * np.abs(K).max()


def test_force_is_energy_gradient():
    rng = np.random.default_rng(24)
    X, conn, x, v, gradN, wJ0 = _one_element(rng, 0.1)
    for mat in (SVK, MR):
        xe = x[conn]
        f = el.element_force(xe, np.zeros_like(xe), gradN, wJ0, mat)[0]
        g = np.zeros((10, 3))
        for a in range(10):
            for i in range(3):
                dx = np.zeros((1, 10, 3), complex)
                dx[0, a, i] = 1e-30j
                g[a, i] = el.element_energy(xe + dx, gradN, wJ0, mat)[0].imag / 1e-30
        assert np.abs(f - g).max() < 1e-12 * np.abs(f).max()


def _exact_linear_stiffness(X, lam, mu):
    """K_ab,ik = int (grad N_a)_J C_iJkL (grad N_b)_L dV with isotropic C,
    integrated exactly: grad N_a is linear in the barycentrics L,
    grad N_a = sum_c dN_a/dL_c grad L_c, and dN_a/dL_c is affine in L, so the
    integrand is a quadratic polynomial in L integrated monomial by monomial."""
    Xc = X[:4]
    Tm = np.vstack([np.ones(4), Xc.T])
    gradL = np.linalg.inv(Tm)[:, 1:]
    V = np.linalg.det(np.stack([Xc[1] - Xc[0], Xc[2] - Xc[0], Xc[3] - Xc[0]])) / 6
    # grad N_a = sum_m coef[a][m] * (monomial m) with monomials 1, L0..L3
    # corners: (4 L_a - 1) gradL_a ; midsides (i,j): 4 L_j gradL_i + 4 L_i gradL_j
    coef = np.zeros((10, 5, 3))
    for a in range(4):
        coef[a, 0] = -gradL[a]
        coef[a, 1 + a] = 4 * gradL[a]
    for m, (i, j) in enumerate(t10.EDGES):
        coef[4 + m, 1 + j] += 4 * gradL[i]
        coef[4 + m, 1 + i] += 4 * gradL[j]

    def mono_int(m1, m2):
        al = [0, 0, 0, 0]
        for mm in (m1, m2):
            if mm > 0:
                al[mm - 1] += 1
        num = np.prod([factorial(x) for x in al]) * 6
        return float(Fraction(int(num), factorial(sum(al) + 3))) * V

    Imat = np.array([[mono_int(m1, m2) for m2 in range(5)] for m1 in range(5)])
    d = np.eye(3)
    C = (lam * np.einsum("ij,kl->ijkl", d, d)
         + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))
    K = np.einsum("amJ,bnL,mn,iJkL->aibk", coef, coef, Imat, C)
    return K.reshape(30, 30)


def test_linear_stiffness_at_reference_equals_exact_integral():
    """At F = I the SVK tangent is the linear-elastic T10 stiffness; its
    integrand is quadratic, so the degree-3 rule must reproduce the exact
    integral."""
    rng = np.random.default_rng(25)
    Xc = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]]) + 0.15 * rng.normal(size=(4, 3))
    assert np.linalg.det(np.stack([Xc[1] - Xc[0], Xc[2] - Xc[0], Xc[3] - Xc[0]])) > 0
    X = np.concatenate([Xc, np.stack([(Xc[i] + Xc[j]) / 2 for i, j in t10.EDGES])])
    conn = np.arange(10)[None]
    gradN, _, wJ0 = t10.reference_geometry(X, conn)
    K = el.element_tangent(X[conn], np.zeros((1, 10, 3)), gradN, wJ0, SVK)[0]
    lam, mu = mats.lame(SVK["E"], SVK["nu"])
    Kex = _exact_linear_stiffness(X, lam, mu)
    assert np.abs(K - Kex).max() < 1e-12 * np.abs(Kex).max()
    # rigid-body null space: 6 zero eigenvalues
    ev = np.linalg.eigvalsh(Kex)
    assert np.sum(np.abs(ev) < 1e-9 * ev.max()) == 6


@pytest.mark.parametrize("mat", [SVK_KV, MR_KV], ids=["svk_kv", "mr_kv"])
def test_kelvin_voigt_geometric_term_at_nonzero_velocity(mat):
    """The Kelvin-Voigt part of K_t at v != 0: with the viscous stress S_v held
    at its value, the derivative in x of f_a = sum_q wJ0 (P_el(F) + F S_v) n_a
    is the hyperelastic tangent plus the geometric term delta_ik n_a.S_v n_b.
    The oracle's K_t (alpha = 1, beta = 0) must equal that derivative, taken
    here by complex step through the elastic stress and the frozen S_v, so a
    wrong sign or factor of the viscous geometric term fails.  The velocity is
    large enough that the term is ~1e-3 of K (far above the 1e-12 bar)."""
    rng = np.random.default_rng(26)
    X, conn, x, v, gradN, wJ0 = _one_element(rng)
    v = 200.0 * v
    xe, ve = x[conn], v[conn]
    K = el.element_tangent(xe, ve, gradN, wJ0, mat, 1.0, 0.0)[0]
    K0 = el.element_tangent(xe, np.zeros_like(ve), gradN, wJ0, mat, 1.0, 0.0)[0]
    assert np.abs(K - K0).max() > 1e-4 * np.abs(K).max()          # the term is really exercised
    F0 = el.kinematics(xe, gradN)
    _, Sv0 = mats.kv_stress(F0, el.kinematics(ve, gradN), mat["eta_d"], mat["lambda_d"])

    def f_frozen(xc):
        F = el.kinematics(xc, gradN)
        P_el, _, _ = mats.elastic_stress_and_tangent(F, mat, want_tangent=False)
        P = P_el + F @ Sv0
        return np.einsum("eqiJ,eqaJ,eq->eai", P, gradN, wJ0)

    Kcs = np.zeros((30, 30))
    for s in range(30):
        b, k = divmod(s, 3)
        dx = np.zeros((1, 10, 3), complex)
        dx[0, b, k] = 1e-30j
        Kcs[:, s] = f_frozen(xe + dx).imag.reshape(30) / 1e-30
    assert np.abs(K - Kcs).max() < 1e-12 * np.abs(K).max()
    # the same term by brute force: K - K_el(v = 0) = sum_q wJ0 delta_ik n_a.S_v n_b
    geo = np.einsum("eqaJ,eqJL,eqbL,eq->eab", gradN, Sv0, gradN, wJ0)[0]
    dK = (K - K0).reshape(10, 3, 10, 3)
    assert np.abs(dK - np.einsum("ab,ik->aibk", geo, np.eye(3))).max() < 1e-9 * np.abs(geo).max()
