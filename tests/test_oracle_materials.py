"""Pins of the oracle's constitutive laws: stress-free reference, rigid
rotations, small-strain limits, the Mooney-Rivlin uniaxial closed forms,
energy consistency and complex-step / finite-difference derivatives."""
import numpy as np
import pytest

from oracle import materials as mats

LAM, MU = mats.lame(1e7, 0.3)
MR = dict(C10=5e5, C01=1e5, kappa=1e8)


def rotation(axis, angle):
    a = np.asarray(axis, float)
    a /= np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K


R37 = rotation((1, 2, 3), np.deg2rad(37.0))


def rand_F(rng, amp=0.2):
    return np.eye(3) + amp * rng.normal(size=(3, 3))


def isotropic_C(lam, mu):
    d = np.eye(3)
    return (lam * np.einsum("ij,kl->ijkl", d, d)
            + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))


def cstep_dP(Pfun, F, h=1e-30):
    """dP_iJ/dF_kL by the complex step (no subtractive cancellation)."""
    A = np.zeros((3, 3, 3, 3))
    for k in range(3):
        for L in range(3):
            Fc = F.astype(complex)
            Fc[k, L] += 1j * h
            A[:, :, k, L] = Pfun(Fc).imag / h
    return A


def cstep_dW(Wfun, F, h=1e-30):
    P = np.zeros((3, 3))
    for k in range(3):
        for L in range(3):
            Fc = F.astype(complex)
            Fc[k, L] += 1j * h
            P[k, L] = Wfun(Fc).imag / h
    return P


# ----------------------------------------------------------------- SVK

def test_svk_zero_at_identity_and_rigid_rotation():
    P, _ = mats.svk_stress(np.eye(3), LAM, MU)
    assert np.abs(P).max() == 0.0
    P, _ = mats.svk_stress(R37, LAM, MU)
    assert np.abs(P).max() < 1e-8 * MU


def test_svk_small_strain_tangent_is_isotropic_hooke():
    A = mats.svk_tangent(np.eye(3), np.zeros((3, 3)), LAM, MU)
    assert np.abs(A - isotropic_C(LAM, MU)).max() < 1e-9 * MU


def test_svk_stress_is_energy_gradient_and_tangent_is_stress_gradient():
    rng = np.random.default_rng(10)
    for _ in range(5):
        F = rand_F(rng)
        P, S = mats.svk_stress(F, LAM, MU)
        assert np.abs(cstep_dW(lambda G: mats.svk_energy(G, LAM, MU), F) - P).max() < 1e-12 * MU
        A = mats.svk_tangent(F, S, LAM, MU)
        Acs = cstep_dP(lambda G: mats.svk_stress(G, LAM, MU)[0], F)
        assert np.abs(A - Acs).max() < 1e-12 * np.abs(A).max()
        # major symmetry of a hyperelastic tangent
        assert np.abs(A - A.transpose(2, 3, 0, 1)).max() < 1e-12 * np.abs(A).max()


# ----------------------------------------------------------------- Mooney-Rivlin

def mrP(F):
    return mats.mr_stress(F, **MR)


def test_mr_zero_at_identity():
    assert np.abs(mrP(np.eye(3))).max() < 1e-9


def test_mr_small_strain_limit():
    """At F = I: isotropic with shear modulus mu = 2(C10 + C01), bulk kappa."""
    A = mats.mr_tangent(np.eye(3), **MR)
    mu = 2 * (MR["C10"] + MR["C01"])
    lam = MR["kappa"] - 2.0 * mu / 3.0
    assert np.abs(A - isotropic_C(lam, mu)).max() < 1e-12 * MR["kappa"]


def test_mr_uniaxial_isochoric_closed_form():
    """F = diag(s, s^-1/2, s^-1/2), J = 1: sigma11 - sigma22 = 2(s^2 - 1/s)(C10 + C01/s)."""
    for s in (0.7, 0.9, 1.1, 1.5, 2.0):
        F = np.diag([s, s ** -0.5, s ** -0.5])
        sigma = mrP(F) @ F.T / np.linalg.det(F)
        expect = 2 * (s * s - 1 / s) * (MR["C10"] + MR["C01"] / s)
        assert abs((sigma[0, 0] - sigma[1, 1]) - expect) < 1e-12 * abs(expect)


def test_mr_traction_free_uniaxial():
    """Uniaxial stretch s with free lateral faces: solve sigma22(s, t) = 0 for
    the lateral stretch t by a scalar Newton iteration, then the axial Cauchy
    stress must equal the closed form of the isochoric split at J = s t^2:
    sigma11 - sigma22 depends on the deviatoric terms only."""
    for s in (0.8, 1.2, 1.6):
        t = s ** -0.5
        for _ in range(60):
            F = np.diag([s, t, t])
            r = (mrP(F) @ F.T)[1, 1]
            Fp = np.diag([s, t + 1e-7, t + 1e-7])
            dr = ((mrP(Fp) @ Fp.T)[1, 1] - r) / 1e-7
            t -= r / dr
            if abs(r) < 1e-6:
                break
        F = np.diag([s, t, t])
        J = s * t * t
        sig = mrP(F) @ F.T / J
        assert abs(sig[1, 1]) < 1e-6 * MR["kappa"] * 1e-3
        # closed form of the Cauchy deviator difference for diag(s, t, t):
        # sigma11 - sigma22 = (2/J)[C10 J^-2/3 (s^2 - t^2) + C01 J^-4/3 (s^2 - t^2) t^2]
        expect = (2 / J) * (MR["C10"] * J ** (-2 / 3) * (s * s - t * t)
                            + MR["C01"] * J ** (-4 / 3) * (s * s - t * t) * t * t)
        assert abs(sig[0, 0] - sig[1, 1] - expect) < 1e-10 * abs(expect)


def test_mr_energy_stress_tangent_consistency():
    rng = np.random.default_rng(11)
    for _ in range(5):
        F = rand_F(rng, 0.15)
        P = mrP(F)
        Pcs = cstep_dW(lambda G: mats.mr_energy(G, **MR), F)
        assert np.abs(P - Pcs).max() < 1e-12 * max(1.0, np.abs(P).max())
        A = mats.mr_tangent(F, **MR)
        Acs = cstep_dP(mrP, F)
        assert np.abs(A - Acs).max() < 1e-12 * np.abs(A).max()
        assert np.abs(A - A.transpose(2, 3, 0, 1)).max() < 1e-12 * np.abs(A).max()


def test_mr_objectivity():
    rng = np.random.default_rng(12)
    F = rand_F(rng, 0.15)
    assert np.abs(mrP(R37 @ F) - R37 @ mrP(F)).max() < 1e-9 * np.abs(mrP(F)).max()


# ----------------------------------------------------------------- Kelvin-Voigt

def test_kv_rigid_spin_has_no_viscous_stress():
    rng = np.random.default_rng(13)
    W = rng.normal(size=(3, 3))
    W = W - W.T                               # spin
    for F in (np.eye(3), R37):
        Fdot = W @ F                          # v = w x x  =>  Fdot = W F
        Pv, _ = mats.kv_stress(F, Fdot, 1e3, 1e3)
        assert np.abs(Pv).max() < 1e-12


def test_kv_velocity_tangent_is_derivative():
    rng = np.random.default_rng(14)
    F = rand_F(rng)
    Fdot = rng.normal(size=(3, 3))
    D = mats.kv_tangent(F, 1e3, 2e3)
    Dcs = cstep_dP(lambda G: mats.kv_stress(F.astype(complex), G, 1e3, 2e3)[0], Fdot)
    assert np.abs(D - Dcs).max() < 1e-12 * np.abs(D).max()
