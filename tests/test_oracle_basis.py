"""Pins for the oracle's harmonic basis (Eq. "harmonic": B_n^m = r^n Y_n^m).

The basis is checked against scipy's spherical harmonics (a library routine
the oracle does not use), against the addition theorem, and against the two
defining properties of solid harmonics: homogeneity of degree n and a zero
Laplacian.
"""
import math

import numpy as np
import pytest

import oracle


def _scipy_Y(n, m, theta, phi):
    from scipy import special
    if hasattr(special, "sph_harm_y"):
        return special.sph_harm_y(n, m, theta, phi)
    return special.sph_harm(m, n, phi, theta)


def _norm(n, m):
    return math.sqrt((2 * n + 1) / (4 * math.pi) * math.factorial(n - m) / math.factorial(n + m))


@pytest.fixture(scope="module")
def pts():
    g = np.random.default_rng(11)
    p = g.normal(size=(40, 3))
    p *= (0.2 + 1.1 * g.random((40, 1))) / np.linalg.norm(p, axis=1, keepdims=True)
    return p


def test_matches_scipy_spherical_harmonics(pts):
    P, Rs = 12, 1.3
    B = oracle.basis(pts, P, Rs)
    r = np.linalg.norm(pts, axis=1)
    theta = np.arccos(pts[:, 2] / r)
    phi = np.arctan2(pts[:, 1], pts[:, 0])
    rho = r / Rs
    for n in range(P + 1):
        for m in range(-n, n + 1):
            k = n * n + n + m
            Y = _scipy_Y(n, abs(m), theta, phi)
            ref = (Y.real if m >= 0 else Y.imag) / (_norm(n, abs(m)) * (-1) ** abs(m))
            np.testing.assert_allclose(B[:, k], rho**n * ref, rtol=1e-10, atol=1e-12 * _scale(n))


def _scale(n):
    return max(1.0, float(np.prod(np.arange(1, 2 * n, 2))))


def test_addition_theorem(pts):
    # sum_m Y_nm(u) Y_nm(v)^* = (2n+1)/(4 pi) P_n(u.v), written in the real form
    P = 10
    u = pts / np.linalg.norm(pts, axis=1, keepdims=True)
    Bu = oracle.basis(u, P, 1.0)
    v = np.roll(u, 1, axis=0)
    Bv = oracle.basis(v, P, 1.0)
    from scipy.special import eval_legendre
    for n in range(P + 1):
        acc = np.zeros(len(u))
        for m in range(-n, n + 1):
            k = n * n + n + m
            w = _norm(n, abs(m)) ** 2 * (2.0 if m != 0 else 1.0)
            acc += w * Bu[:, k] * Bv[:, k]
        ref = (2 * n + 1) / (4 * math.pi) * eval_legendre(n, np.sum(u * v, axis=1))
        np.testing.assert_allclose(acc, ref, rtol=1e-11, atol=1e-12)


def test_homogeneous_of_degree_n(pts):
    P = 9
    B1 = oracle.basis(pts, P, 1.0)
    B2 = oracle.basis(0.37 * pts, P, 1.0)
    for n in range(P + 1):
        sl = slice(n * n, (n + 1) * (n + 1))
        np.testing.assert_allclose(B2[:, sl], 0.37**n * B1[:, sl], rtol=1e-12, atol=1e-300)


def test_laplacian_vanishes(pts):
    # a fourth-order central difference of the Laplacian of every basis function
    P, h = 8, 1e-2
    x = pts[:10]
    lap = -3 * 2.5 * oracle.basis(x, P, 1.0)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        lap += (-1 / 12) * (oracle.basis(x + 2 * e, P, 1.0) + oracle.basis(x - 2 * e, P, 1.0))
        lap += (4 / 3) * (oracle.basis(x + e, P, 1.0) + oracle.basis(x - e, P, 1.0))
    lap /= h * h
    B = oracle.basis(x, P, 1.0)
    scale = np.abs(B).max(axis=0) + 1.0
    assert np.all(np.abs(lap) < 1e-5 * scale)


def test_origin_is_constant_only():
    B = oracle.basis(np.zeros((1, 3)), 5, 2.0)
    assert B[0, 0] == 1.0 and np.all(B[0, 1:] == 0.0)
