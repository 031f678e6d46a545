"""Pins for the oracle's geometry: Fibonacci integration (Sec. II.B),
monitoring points (Sec. II.A and II.C), the in-set of Sec. II.A, the least-
squares solver and the plain Coulomb sums."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import hsma

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- quadrature
@pytest.mark.parametrize("F2", [89, 377, 987])
def test_quadrature_weights_sum_to_sphere_area(F2):
    R = 1.7
    dirs, w = oracle.quadrature(F2, hsma.fib_predecessor(F2), R)
    assert dirs.shape == (2 * (F2 + 1), 3)
    np.testing.assert_allclose(np.linalg.norm(dirs, axis=1), 1.0, rtol=0, atol=1e-15)
    assert abs(w.sum() - 4 * math.pi * R * R) < 1e-12 * 4 * math.pi * R * R
    # the two pole nodes carry zero weight
    assert w[0] == 0.0 and w[1] == 0.0 and abs(w[-1]) < 1e-15 and abs(w[-2]) < 1e-15


def test_quadrature_integrates_harmonics_to_zero():
    # int Y_nm dS = 0 for n >= 1; and int (B_n^m)^2 dS matches scipy-free closed form
    F2 = 987
    dirs, w = oracle.quadrature(F2, hsma.fib_predecessor(F2), 1.0)
    B = oracle.basis(dirs, 10, 1.0)
    integ = w @ B
    assert abs(integ[0] - 4 * math.pi) < 1e-12
    # relative to each (unnormalised) column's size
    assert np.abs(integ[1:] / np.abs(B[:, 1:]).max(axis=0)).max() < 1e-12
    # int z^2 dS = 4 pi/3, int z^4 dS = 4 pi/5 on the unit sphere
    assert abs(w @ dirs[:, 2] ** 2 - 4 * math.pi / 3) < 1e-9
    assert abs(w @ dirs[:, 2] ** 4 - 4 * math.pi / 5) < 1e-9


def test_quadrature_converges_fast():
    # error of a smooth non-polynomial integrand drops quickly with F2 (Sec. II.B)
    def f(d):
        return np.exp(d[:, 0] + 0.3 * d[:, 1] - 0.5 * d[:, 2])
    # exact: int exp(k.u) dS = 4 pi sinh|k|/|k|
    k = math.sqrt(1 + 0.09 + 0.25)
    exact = 4 * math.pi * math.sinh(k) / k
    errs = []
    for F2 in (55, 144, 377):
        dirs, w = oracle.quadrature(F2, hsma.fib_predecessor(F2), 1.0)
        errs.append(abs(w @ f(dirs) - exact))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-9


def test_image_count_matches_paper():
    g = json.load(open(os.path.join(GOLD, "fibonacci_counts.json")))
    for F2, No in g["pairs"]:
        dirs, _ = oracle.quadrature(F2, hsma.fib_predecessor(F2), 1.0)
        assert 3 * dirs.shape[0] == No
    F2 = g["plateau"]["F2_min"]
    assert 6 * (F2 + 1) > g["plateau"]["N_o_above"]
    assert hsma.fib_from_points(2000) == (377, 233)
    assert hsma.fib_from_points(8000) == (1597, 987)
    assert hsma.fib_from_points(6000) == (987, 610)


# ---------------------------------------------------------------- monitoring
def test_monitor_sphere():
    nm, R0 = 200, math.sqrt(3) / 2
    x = oracle.monitor_sphere(nm, R0)
    np.testing.assert_allclose(np.linalg.norm(x, axis=1), R0, rtol=1e-14)
    # heights evenly spaced (the latitude grid), covering both hemispheres
    np.testing.assert_allclose(np.diff(x[:, 2]), 2 * R0 / nm, rtol=1e-9)
    assert abs(x.mean(axis=0)).max() < 0.02 * R0
    # azimuth advances by 2 pi w per point, w = (sqrt5 - 1)/2
    az = np.arctan2(x[:, 1], x[:, 0])
    w = (math.sqrt(5) - 1) / 2
    d = np.mod(np.diff(az) - 2 * math.pi * w, 2 * math.pi)
    assert np.all(np.minimum(d, 2 * math.pi - d) < 1e-9)


def test_wrap_into_box():
    L = np.array([1.0, 1.0, 2.0])
    x = oracle.monitor_sphere(300, 0.5 * np.linalg.norm(L))
    xt = oracle.wrap_into_box(x, L)
    assert np.all(np.abs(xt) <= 0.5 * L + 1e-15)
    k = (x - xt) / L
    np.testing.assert_allclose(k, np.round(k), atol=1e-12)


def test_monitor_faces():
    L = np.array([1.0, 1.0, 2.0])
    K = 1500
    x = oracle.monitor_faces(K, L)
    assert x.shape == (K, 3)
    on_wall = np.isclose(np.abs(x), 0.5 * L, rtol=0, atol=1e-15)
    assert np.all(on_wall.sum(axis=1) == 1)
    assert np.all(np.abs(x) <= 0.5 * L + 1e-15)
    # counts in proportion to area: faces normal to z have area 1, others 2
    nz = np.sum(on_wall[:, 2])
    assert abs(nz - K * 2 / 10) <= 1


def test_periodic_fit_on_box_faces_is_singular():
    """Why the periodic monitoring points sit on the circumsphere (Sec. II.A):
    with points on the box faces, each paired with its periodic partner on
    the opposite face, every harmonic that is even in x, in y and in z takes
    equal values at both points of each pair, so its column of the fitting
    matrix Phi(x) - Phi(x~) vanishes and its coefficient is undetermined.
    Which harmonics are even is found by reflecting random points, not from
    the face matrix; the circumsphere matrix of the same order has full rank."""
    L = np.array([1.0, 1.0, 1.0])
    P, K, Rs = 8, 600, 1.5
    g = np.random.default_rng(11)
    # K points on the three lower faces (the upper ones are their partners)
    pts = []
    for a in range(3):
        p = g.uniform(-0.5, 0.5, size=(K // 3, 3)) * L
        p[:, a] = -0.5 * L[a]
        pts.append(p)
    x = np.concatenate(pts)
    xt = oracle.wrap_into_box(x, L)
    np.testing.assert_allclose(np.abs(x - xt).sum(axis=1), 1.0, rtol=0, atol=1e-15)
    M = (oracle.basis(x, P, Rs) - oracle.basis(xt, P, Rs))[:, 1:]
    zero = np.abs(M).max(axis=0) <= 1e-13 * np.abs(M).max()
    r = g.standard_normal((64, 3))
    B = oracle.basis(r, P, Rs)
    even = np.ones(B.shape[1], dtype=bool)
    for a in range(3):
        rr = r.copy()
        rr[:, a] = -rr[:, a]
        even &= np.abs(oracle.basis(rr, P, Rs) - B).max(axis=0) <= 1e-12 * np.abs(B).max()
    assert np.array_equal(zero, even[1:])
    assert zero.sum() >= 5
    # the circumsphere placement: full column rank, well conditioned
    xs = oracle.monitor_sphere(K, 0.5 * np.linalg.norm(L))
    Ms = (oracle.basis(xs, P, Rs) - oracle.basis(oracle.wrap_into_box(xs, L), P, Rs))[:, 1:]
    Ms = Ms / np.linalg.norm(Ms, axis=0)
    sv = np.linalg.svd(Ms, compute_uv=False)
    assert sv[0] / sv[-1] < 1e3


# ---------------------------------------------------------------- in-set
def test_num_shells_brute_force():
    for Rs, La in [(1.5, 1.0), (3.464, 2.0), (2.121, 1.0), (2.121, 2.0), (0.9, 1.0)]:
        k = oracle.num_shells(Rs, La)
        # smallest possible |x + k L| for x in [-L/2, L/2) is (|k| - 1/2) L
        assert (k - 0.5) * La < Rs <= (k + 0.5) * La


@pytest.mark.parametrize("bc", [0, 1])
def test_inset_is_exactly_the_images_inside_the_sphere(bc):
    g = np.random.default_rng(3)
    L = np.array([1.0, 1.0, 2.0])
    n = 37
    c = (g.random((n, 3)) - 0.5) * L
    q = g.standard_normal(n)
    Rs = 0.5 * np.linalg.norm(L) * 1.6
    xyz, qq, src, sh = oracle.inset(c, q, L, bc, Rs)
    assert np.array_equal(xyz[:n], c) and np.array_equal(qq[:n], q)
    # brute force over a generous shell range
    want = set()
    for k in itertools.product(range(-4, 5), repeat=3):
        k = np.array(k)
        s = (-1.0) ** np.abs(k) if bc == 1 else np.ones(3)
        sign = (-1.0) ** np.abs(k).sum() if bc == 1 else 1.0
        p = c * s + k * L
        inside = np.linalg.norm(p, axis=1) < Rs
        for j in np.nonzero(inside)[0]:
            want.add((tuple(np.round(p[j], 12)), round(sign * q[j], 12)))
    got = {(tuple(np.round(xyz[i], 12)), round(qq[i], 12)) for i in range(len(qq))}
    assert got == want and len(got) == len(qq)
    assert np.all(np.linalg.norm(xyz, axis=1) < Rs)


# ---------------------------------------------------------------- least squares
def test_lstsq_matches_numpy():
    g = np.random.default_rng(7)
    A = g.standard_normal((300, 40)) * np.logspace(0, 3, 40)
    b = g.standard_normal(300)
    x, _ = oracle.lstsq(A, b)
    ref = np.linalg.lstsq(A, b, rcond=None)[0]
    np.testing.assert_allclose(x, ref, rtol=1e-11)
    # the residual is orthogonal to the columns (normal equations)
    r = b - A @ x
    assert np.abs(A.T @ r).max() < 1e-10 * np.abs(A).max() * np.abs(b).max()


def test_lstsq_recovers_planted_solution():
    g = np.random.default_rng(8)
    # columns scaled over 8 decades: equilibration keeps every component exact
    A = g.standard_normal((120, 25)) * np.logspace(0, 8, 25)
    x0 = g.standard_normal(25) / np.logspace(0, 8, 25)
    x, _ = oracle.lstsq(A, A @ x0)
    np.testing.assert_allclose(x, x0, rtol=1e-11)


def test_lstsq_rejects_zero_column():
    A = np.ones((10, 3))
    A[:, 1] = 0.0
    with pytest.raises(np.linalg.LinAlgError):
        oracle.lstsq(A, np.ones(10))


# ---------------------------------------------------------------- Coulomb sums
def test_coulomb_cube_centre_closed_form():
    a = 0.7
    corners = np.array(list(itertools.product((-a / 2, a / 2), repeat=3)))
    q = np.full(8, 1.5)
    pot, fld = oracle.coulomb(corners, q, np.zeros((1, 3)))
    assert abs(pot[0] - 8 * 1.5 / (math.sqrt(3) * a / 2)) < 1e-13
    assert np.abs(fld).max() < 1e-13


def test_coulomb_field_is_minus_gradient():
    g = np.random.default_rng(9)
    s = g.random((50, 3))
    q = g.standard_normal(50)
    t = g.random((5, 3)) + 2.0
    _, fld = oracle.coulomb(s, q, t)
    h = 1e-4
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = -(oracle.coulomb(s, q, t + e, field=False) - oracle.coulomb(s, q, t - e, field=False)) / (2 * h)
        np.testing.assert_allclose(fld[:, a], fd, rtol=1e-6, atol=1e-9)


def test_coulomb_skip_and_threads():
    g = np.random.default_rng(10)
    s = g.random((200, 3))
    q = g.standard_normal(200)
    t = s[:30]
    p1, f1 = oracle.coulomb(s, q, t, tskip=np.arange(30))
    p4, f4 = oracle.coulomb(s, q, t, tskip=np.arange(30), nthreads=4)
    assert np.array_equal(p1, p4) and np.array_equal(f1, f4)
    # skipping the own copy equals removing that source
    for i in (0, 17):
        keep = np.arange(200) != i
        pr, fr = oracle.coulomb(s[keep], q[keep], t[i:i + 1])
        np.testing.assert_allclose(p1[i], pr[0], rtol=1e-14)
        np.testing.assert_allclose(f1[i], fr[0], rtol=1e-13)
    # a coincident source that is not skipped gives a non-finite result
    p, _ = oracle.coulomb(s, q, t[:1])
    assert not np.isfinite(p[0])
