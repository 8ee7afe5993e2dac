"""Pins of the oracle's T10 element pieces (shape functions, Keast rule,
reference geometry, exact mass) against closed forms and brute force."""
import itertools
from fractions import Fraction
from math import factorial

import numpy as np
import pytest

from oracle import t10


def _all_monomials(max_deg):
    for a in itertools.product(range(max_deg + 1), repeat=4):
        if sum(a) <= max_deg:
            yield a


def test_keast5_exact_to_degree_3():
    """Keast's 5-point rule integrates every barycentric monomial of degree <= 3
    exactly: int L^a dV / V = a! 3! / (|a|+3)! (Dirichlet integral)."""
    for a in _all_monomials(3):
        exact = float(Fraction(np.prod([factorial(x) for x in a]) * 6, factorial(sum(a) + 3)))
        quad = sum(t10.KEAST5_WFRAC[q] * np.prod(t10.KEAST5_L[q] ** np.array(a))
                   for q in range(5))
        assert abs(quad - exact) < 1e-15, (a, quad, exact)


def test_keast5_not_exact_at_degree_4():
    """... and is not exact for L0^4 (so the degree-3 claim is tight: a mistyped
    point that happened to raise the degree would be caught here)."""
    a = (4, 0, 0, 0)
    exact = float(Fraction(factorial(4) * 6, factorial(7)))
    quad = sum(t10.KEAST5_WFRAC[q] * t10.KEAST5_L[q][0] ** 4 for q in range(5))
    assert abs(quad - exact) > 1e-4
    assert abs(t10.KEAST5_WFRAC.sum() - 1.0) < 1e-15
    assert np.allclose(t10.KEAST5_L.sum(1), 1.0)


def _node_barycentrics():
    L = np.zeros((10, 4))
    for i in range(4):
        L[i, i] = 1.0
    for m, (i, j) in enumerate(t10.EDGES):
        L[4 + m, i] = L[4 + m, j] = 0.5
    return L


def test_shape_functions_kronecker_and_partition_of_unity():
    Ln = _node_barycentrics()
    N = np.stack([t10.shape_values(L) for L in Ln])
    assert np.allclose(N, np.eye(10), atol=1e-15)
    rng = np.random.default_rng(0)
    for _ in range(20):
        L = rng.dirichlet(np.ones(4))
        assert abs(t10.shape_values(L).sum() - 1.0) < 1e-14
        assert np.abs(t10.shape_dxi(L).sum(0)).max() < 1e-14


def test_shape_gradient_matches_finite_difference():
    rng = np.random.default_rng(1)
    L = rng.dirichlet(np.ones(4))
    xi = L[1:]
    G = t10.shape_dxi(L)
    eps = 1e-6
    for j in range(3):
        dxi = np.zeros(3)
        dxi[j] = eps
        Lp = np.concatenate([[1 - (xi + dxi).sum()], xi + dxi])
        Lm = np.concatenate([[1 - (xi - dxi).sum()], xi - dxi])
        fd = (t10.shape_values(Lp) - t10.shape_values(Lm)) / (2 * eps)
        assert np.abs(fd - G[:, j]).max() < 1e-9


def _random_tet(rng):
    while True:
        Xc = rng.normal(size=(4, 3))
        if np.linalg.det(np.stack([Xc[1] - Xc[0], Xc[2] - Xc[0], Xc[3] - Xc[0]])) > 0.1:
            break
    X = np.concatenate([Xc, np.stack([(Xc[i] + Xc[j]) / 2 for i, j in t10.EDGES])])
    return X, np.arange(10)[None, :]


def test_reference_geometry_straight_tet_closed_form():
    """For a straight-sided T10 the isoparametric gradients equal the closed
    form: corners (4L_a - 1) grad L_a, midsides 4 (L_i grad L_j + L_j grad L_i),
    and J0 = 6V at every point."""
    rng = np.random.default_rng(2)
    X, conn = _random_tet(rng)
    gradN, J0, wJ0 = t10.reference_geometry(X, conn)
    Xc = X[:4]
    # barycentric gradients: rows of the inverse of [[1,1,1,1],[x],[y],[z]]
    Tm = np.vstack([np.ones(4), Xc.T])
    gradL = np.linalg.inv(Tm)[:, 1:]                 # (4, 3)
    V = np.linalg.det(np.stack([Xc[1] - Xc[0], Xc[2] - Xc[0], Xc[3] - Xc[0]])) / 6
    for q in range(5):
        L = t10.KEAST5_L[q]
        expect = np.zeros((10, 3))
        for a in range(4):
            expect[a] = (4 * L[a] - 1) * gradL[a]
        for m, (i, j) in enumerate(t10.EDGES):
            expect[4 + m] = 4 * (L[i] * gradL[j] + L[j] * gradL[i])
        assert np.abs(gradN[0, q] - expect).max() < 1e-12
        assert abs(J0[0, q] - 6 * V) < 1e-12
    assert abs(wJ0.sum() - V) < 1e-14


def test_gradients_reproduce_linear_fields():
    """sum_a X_a (x) grad N_a = I (the reference configuration has F = I)."""
    rng = np.random.default_rng(3)
    X, conn = _random_tet(rng)
    gradN, _, _ = t10.reference_geometry(X, conn)
    F = np.einsum("ai,qaJ->qiJ", X, gradN[0])
    assert np.abs(F - np.eye(3)).max() < 1e-13


# Closed form of the consistent mass of the 10-node tetrahedron (standard
# result of exact integration of products of quadratic shape functions), in
# units of rho V / 420: corner diagonal 6, corner-corner 1, corner with a
# midside on an edge through it -4, corner with a midside on the opposite
# edges -6, midside diagonal 32, midsides on edges sharing a node 16, midsides
# on opposite edges 8.
def _mass_closed_form():
    M = np.zeros((10, 10))
    for a in range(10):
        for b in range(10):
            if a < 4 and b < 4:
                M[a, b] = 6 if a == b else 1
            elif a < 4 or b < 4:
                c, m = (a, b) if a < 4 else (b, a)
                M[a, b] = -4 if c in t10.EDGES[m - 4] else -6
            else:
                if a == b:
                    M[a, b] = 32
                else:
                    shared = set(t10.EDGES[a - 4]) & set(t10.EDGES[b - 4])
                    M[a, b] = 16 if shared else 8
    return M / 420.0


def test_exact_mass_matches_closed_form():
    assert np.abs(t10._UNIT_MASS - _mass_closed_form()).max() < 1e-15


def test_mass_spd_and_total():
    rng = np.random.default_rng(4)
    X, conn = _random_tet(rng)
    Me = t10.element_mass(X, conn, 7.0)[0]
    V = t10.element_volumes(X, conn)[0]
    assert abs(Me.sum() - 7.0 * V) < 1e-13
    assert np.linalg.eigvalsh(Me).min() > 0
    # the 5-point rule would make it indefinite (why the oracle integrates exactly)
    Mq = sum(t10.KEAST5_WFRAC[q] * np.outer(t10.shape_values(t10.KEAST5_L[q]),
                                             t10.shape_values(t10.KEAST5_L[q]))
             for q in range(5))
    assert np.linalg.eigvalsh(Mq).min() < 0
