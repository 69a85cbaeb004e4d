"""Pins of the oracle's tables against closed forms (no GPU).

Gauss rules of Eq. 3 and the tet rules of the far field are checked against
textbook values and exact monomial integrals; the direction table against the
exact half-sphere moments that fix the prefactor pi/16 of Eq. 3.
"""
import math

import numpy as np
import pytest


def test_gauss_legendre_closed_forms(orc):
    """Closed-form Gauss-Legendre nodes and weights for n = 1..5 (textbook roots of P_n)."""
    r30, r70 = math.sqrt(30.0), math.sqrt(70.0)
    table = {
        1: ([0.0], [2.0]),
        2: ([-1 / math.sqrt(3), 1 / math.sqrt(3)], [1.0, 1.0]),
        3: ([-math.sqrt(0.6), 0.0, math.sqrt(0.6)], [5 / 9, 8 / 9, 5 / 9]),
        4: ([-math.sqrt(3 / 7 + 2 / 7 * math.sqrt(1.2)), -math.sqrt(3 / 7 - 2 / 7 * math.sqrt(1.2)),
             math.sqrt(3 / 7 - 2 / 7 * math.sqrt(1.2)), math.sqrt(3 / 7 + 2 / 7 * math.sqrt(1.2))],
            [(18 - r30) / 36, (18 + r30) / 36, (18 + r30) / 36, (18 - r30) / 36]),
        5: ([-math.sqrt(5 + 2 * math.sqrt(10 / 7)) / 3, -math.sqrt(5 - 2 * math.sqrt(10 / 7)) / 3, 0.0,
             math.sqrt(5 - 2 * math.sqrt(10 / 7)) / 3, math.sqrt(5 + 2 * math.sqrt(10 / 7)) / 3],
            [(322 - 13 * r70) / 900, (322 + 13 * r70) / 900, 128 / 225, (322 + 13 * r70) / 900,
             (322 - 13 * r70) / 900]),
    }
    for n, (nodes, weights) in table.items():
        t, w = orc.gauss_legendre(n)
        assert np.allclose(t, nodes, atol=2e-16, rtol=0), n
        assert np.allclose(w, weights, atol=4e-16, rtol=0), n


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16, 33, 64, 128, 256])
def test_gauss_legendre_monomials(orc, n):
    t, w = orc.gauss_legendre(n)
    assert np.all(np.diff(t) > 0)
    for m in range(0, 2 * n):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.dot(w, t**m) - exact) < 2e-14 * max(1.0, n / 16)
    if n <= 32:
        # degree 2n is not integrated exactly (guards against an over-clever rule)
        assert abs(np.dot(w, t ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-15


@pytest.mark.parametrize("alpha", [0, 1, 2])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_gauss_jacobi_moments(orc, k, alpha):
    u, w = orc.gauss_jacobi01(k, alpha)
    assert np.all((u > 0) & (u < 1))
    for m in range(0, 2 * k):
        exact = math.factorial(m) * math.factorial(alpha) / math.factorial(m + alpha + 1)
        assert abs(np.dot(w, u**m) - exact) < 1e-14


def _dirichlet(a, b, c):
    """int over the unit simplex of xi1^a xi2^b xi3^c divided by its volume 1/6."""
    return 6.0 * math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)


@pytest.mark.parametrize("order,degree", [(1, 1), (4, 2), (8, 3), (27, 5), (64, 7)])
def test_tet_rule_exact_to_its_degree(orc, order, degree):
    bary, w = orc.tet_rule(order)
    assert bary.shape == (order, 4)
    assert np.allclose(bary.sum(axis=1), 1.0, atol=1e-15)
    assert np.all(bary > 0)
    assert abs(w.sum() - 1.0) < 1e-14
    xi = bary[:, 1:]
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            for c in range(degree + 1 - a - b):
                got = np.dot(w, xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c)
                assert abs(got - _dirichlet(a, b, c)) < 1e-14, (a, b, c)
    # and one monomial of the next degree is not exact
    worst = max(
        abs(np.dot(w, xi[:, 0] ** a * xi[:, 1] ** (degree + 1 - a)) - _dirichlet(a, degree + 1 - a, 0))
        for a in range(degree + 2)
    )
    assert worst > 1e-6


def test_four_point_rule_constants(orc):
    bary, w = orc.tet_rule(4)
    a = (5 + 3 * math.sqrt(5)) / 20
    b = (5 - math.sqrt(5)) / 20
    for q in range(4):
        expect = np.full(4, b)
        expect[q] = a
        assert np.allclose(bary[q], expect, atol=1e-16)
    assert np.allclose(w, 0.25)


def test_unsupported_tet_rule(orc):
    with pytest.raises(ValueError):
        orc.tet_rule(5)


@pytest.mark.parametrize("n_phi,n_theta", [(16, 8), (16, 16), (24, 32)])
def test_direction_table_half_sphere_moments(orc, n_phi, n_theta):
    """sum k_nm s s^T equals (1/4pi) int over the half sphere of s s^T = I/6.

    With the printed 1/(16 pi^2) instead of pi/16 this sum is off by pi^3;
    a theta range over the full circle would double it.
    """
    s, k = orc.directions(n_phi, n_theta)
    assert np.allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-15)
    assert np.all(s[:, 1] >= 0)  # theta in [0, pi]: the y >= 0 half
    assert np.all(k > 0)
    M = (k[:, None, None] * s[:, :, None] * s[:, None, :]).sum(axis=0)
    tol = 1e-12 if min(n_phi, n_theta) >= 16 else 1e-6
    assert np.allclose(M, np.eye(3) / 6.0, atol=tol)
    # sum k -> (1/4pi) * 2pi = 1/2
    assert abs(k.sum() - 0.5) < (1e-12 if n_phi >= 16 else 1e-6)


def test_direction_table_layout(orc):
    s, k = orc.directions(3, 2)
    tN, wN = orc.gauss_legendre(3)
    tM, wM = orc.gauss_legendre(2)
    phi = (1 + tN) * np.pi / 2
    theta = (1 + tM) * np.pi / 2
    for n in range(3):
        for m in range(2):
            l = n * 2 + m
            assert np.allclose(s[l], [np.sin(phi[n]) * np.cos(theta[m]), np.sin(phi[n]) * np.sin(theta[m]),
                                      np.cos(phi[n])], atol=1e-16)
            assert abs(k[l] - np.pi / 16 * np.sin(phi[n]) * wN[n] * wM[m]) < 1e-16


def test_moller_trumbore_hand_cases(orc):
    p0, p1, p2 = [0, 0, 0], [1, 0, 0], [0, 1, 0]
    hit, t, u, v = orc.moller_trumbore([0.2, 0.3, 1.0], [0, 0, -1], p0, p1, p2)
    assert hit and abs(t - 1.0) < 1e-15 and abs(u - 0.2) < 1e-15 and abs(v - 0.3) < 1e-15
    # behind the origin: negative directed distance (the full line is used)
    hit, t, u, v = orc.moller_trumbore([0.2, 0.3, -2.0], [0, 0, -1], p0, p1, p2)
    assert hit and abs(t + 2.0) < 1e-15
    # two-sided: reversed winding gives the same distance, swapped area coordinates
    hit, t2, u2, v2 = orc.moller_trumbore([0.2, 0.3, 1.0], [0, 0, -1], p0, p2, p1)
    assert hit and abs(t2 - 1.0) < 1e-15 and abs(u2 - 0.3) < 1e-15 and abs(v2 - 0.2) < 1e-15
    # outside the triangle
    assert not orc.moller_trumbore([0.8, 0.8, 1.0], [0, 0, -1], p0, p1, p2)[0]
    assert not orc.moller_trumbore([-0.1, 0.3, 1.0], [0, 0, -1], p0, p1, p2)[0]
    # parallel to the plane
    assert not orc.moller_trumbore([0.2, 0.3, 1.0], [1, 0, 0], p0, p1, p2)[0]
    # oblique direction, hit point on the plane z = 0 at (0.5, 0.25, 0)
    d = np.array([0.3, -0.05, -1.0])
    o = np.array([0.5, 0.25, 0.0]) - 2.5 * d
    hit, t, u, v = orc.moller_trumbore(o, d, p0, p1, p2)
    assert hit and abs(t - 2.5) < 1e-14 and abs(u - 0.5) < 1e-14 and abs(v - 0.25) < 1e-14


def test_tet_geometry(orc):
    # regular tetrahedron of edge a: circumradius a sqrt(6)/4, volume a^3/(6 sqrt 2)
    a = 0.7
    v = a / math.sqrt(2) * np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]]) / 2 * math.sqrt(2)
    edge = np.linalg.norm(v[0] - v[1])
    c, rho, h, vol = orc.tet_geometry(v)
    assert np.allclose(c, 0, atol=1e-16)
    assert abs(rho - edge * math.sqrt(6) / 4) < 1e-15
    assert abs(h - edge) < 1e-15
    assert abs(vol - edge**3 / (6 * math.sqrt(2))) < 1e-15
    # Kuhn tet of a cube of side s: circumradius = half the cube diagonal
    s = 0.25
    v = np.array([[0, 0, 0], [s, 0, 0], [s, s, 0], [s, s, s]])
    c, rho, h, vol = orc.tet_geometry(v)
    assert abs(rho - math.sqrt(3) * s / 2) < 1e-15
    assert abs(vol - s**3 / 6) < 1e-16
    assert np.allclose(c, [0.75 * s, 0.5 * s, 0.25 * s])
