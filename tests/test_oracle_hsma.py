"""End-to-end pins for the HSMA oracle against quantities the paper and the
mathematics fix independently of HSMA:

* the NaCl Madelung constant the paper quotes (Sec. III, first example), both
  through an Ewald sum and through HSMA, with HSMA inside the truncation bound
  of Sec. II.A and converging geometrically in P;
* Ewald sums on small random neutral periodic boxes (energy and forces);
* the grounded box of Sec. III (second example) against the exact
  doubled-cell image lattice;
* force balance (Sec. III), translation invariance;
* the harmonic surface mapping on its own: a planted exterior charge, a
  constant exterior potential, zero net charge of each dipole pair.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import checks, hsma
from paper_1806_04801_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")
MADELUNG = json.load(open(os.path.join(GOLD, "madelung_nacl.json")))
THREE = json.load(open(os.path.join(GOLD, "dirichlet_three_charges.json")))


def _nacl():
    xyz, q, a = checks.nacl_lattice(MADELUNG["n_side"], MADELUNG["L"])
    return xyz, q, a, np.full(3, MADELUNG["L"])


def test_madelung_by_ewald():
    xyz, q, a, L = _nacl()
    _, fld, U = checks.ewald_periodic(xyz, q, L)
    M = checks.madelung_from_energy(U, len(q), a)
    assert abs(M - MADELUNG["madelung_constant"]) < 1e-12
    assert np.abs(fld).max() < 1e-12  # every ion sits at a centre of symmetry


def test_madelung_by_hsma_converges_within_bound():
    xyz, q, a, L = _nacl()
    alpha = MADELUNG["alpha"]
    Rs = hsma.alpha_to_rs(L, alpha)
    d0 = len(q) / np.prod(L)
    errs = []
    for P in (8, 12, 16, 20, 25):
        out, _ = hsma.hsma(xyz, q, L, hsma.PERIODIC, P, Rs, 2 * P * P, F2=MADELUNG["F2"])
        M = checks.madelung_from_energy(out["energy"], len(q), a)
        err = abs(M - MADELUNG["madelung_constant"])
        # |dM| = 2a |dU|/N <= a * eps_potl
        assert err <= a * hsma.error_bound_potential(alpha, P, Rs, d0, 1.0)
        errs.append(err)
    assert errs[-1] < 1e-11
    # geometric convergence: the observed rate per degree is at least ~1/alpha
    slope = (math.log(errs[3]) - math.log(errs[0])) / (20 - 8)
    assert slope < -math.log(alpha) * 0.8


@pytest.mark.parametrize("n,seed", [(2, 1), (8, 2), (32, 3), (64, 4)])
def test_periodic_against_ewald(n, seed):
    L = np.ones(3)
    xyz, q = inputs.random_neutral(n, L, seed)
    _, fld, U = checks.ewald_periodic(xyz, q, L)
    Rs = hsma.alpha_to_rs(L, 2.0)
    out, _ = hsma.hsma(xyz, q, L, hsma.PERIODIC, 25, Rs, 2 * 25 * 25, F2=987)
    assert abs(out["energy"] - U) <= 1e-9 * abs(U)
    F = q[:, None] * fld
    assert np.abs(out["forces"] - F).max() <= 1e-8 * np.abs(F).max()
    # the gradient bound of Sec. II.A at a coarser order
    out8, _ = hsma.hsma(xyz, q, L, hsma.PERIODIC, 8, Rs, 128, F2=987)
    bound = hsma.error_bound_gradient(2.0, 8, Rs, n / 1.0, 1.0)
    assert np.abs(out8["forces"] - F).max() <= bound


def test_force_balance_and_translation():
    L = np.ones(3)
    xyz, q = inputs.random_neutral(40, L, 12)
    Rs = hsma.alpha_to_rs(L, 2.0)
    out, plan = hsma.hsma(xyz, q, L, hsma.PERIODIC, 20, Rs, 800, F2=610)
    Fmax = np.abs(out["forces"]).max()
    assert np.abs(out["forces"].sum(axis=0)).max() < 1e-6 * Fmax
    shifted = np.mod(xyz + np.array([0.31, -0.17, 0.55]), 1.0)
    out2 = hsma.energy_forces(shifted, q, plan)
    assert abs(out2["energy"] - out["energy"]) < 1e-7 * abs(out["energy"])
    np.testing.assert_allclose(out2["forces"], out["forces"], rtol=0, atol=1e-6 * Fmax)


@pytest.mark.parametrize("alpha,P,tol", [(2.0, 16, 1e-7), (2.0, 20, 1e-9), (3.0, 20, 1e-9)])
def test_grounded_three_charges_exact(alpha, P, tol):
    L = np.full(3, THREE["L"])
    c = np.array(THREE["positions_centred"])
    q = np.array(THREE["charges"])
    xyz = c + 0.5 * L
    pot, fld, U = checks.grounded_box_exact(xyz, q, L)
    Rs = hsma.alpha_to_rs(L, alpha)
    out, plan = hsma.hsma(xyz, q, L, hsma.GROUNDED, P, Rs, 2 * P * P, F2=987, dr_rel=THREE["dr_rel"])
    assert abs(out["energy"] - U) <= tol * abs(U)
    F = q[:, None] * fld
    assert np.abs(out["forces"] - F).max() <= 100 * tol * np.abs(F).max()


def test_grounded_exact_pin_vanishes_on_walls():
    # the doubled-cell lattice gives zero potential on every wall
    L = np.array([1.0, 1.0, 2.0])
    g = np.random.default_rng(4)
    xyz = 0.1 + g.random((4, 3)) * (L - 0.2)
    q = np.array([1.0, -2.0, 0.5, 0.7])
    c = xyz - 0.5 * L
    pos, chg = [], []
    import itertools
    for p in itertools.product((0, 1), repeat=3):
        s = np.array([(-1.0) ** pa for pa in p])
        pos.append(c * s + np.array(p) * L)
        chg.append(q * (-1.0) ** sum(p))
    pos, chg = np.concatenate(pos), np.concatenate(chg)
    wall = oracle.monitor_faces(60, L)
    # potential at wall points from the periodic 2L lattice, by Ewald with test charges
    allpos = np.concatenate([pos, wall])
    allq = np.concatenate([chg, np.zeros(len(wall))])
    pot, _, _ = checks.ewald_periodic(allpos, allq, 2 * L)
    assert np.abs(pot[len(chg):]).max() < 1e-12 * np.abs(pot[:len(chg)]).max()


def _plan_for_mapping(P=14, F2=987, bc=hsma.PERIODIC):
    L = np.ones(3)
    Rs = hsma.alpha_to_rs(L, 2.0)
    return hsma.make_plan(L, bc, P, Rs, 2 * P * P, F2)


def test_mapping_reproduces_exterior_charge():
    # Sec. II.B on its own: fit a planted exterior potential, map it to surface
    # images, evaluate inside the box
    plan = _plan_for_mapping()
    src = np.array([[2.3, -0.9, 1.1]]) * plan.Rs / 1.0
    qs = np.array([1.7])
    pts = oracle.monitor_sphere(400, 0.5 * math.sqrt(3))
    B = oracle.basis(pts, plan.P, plan.Rs)
    A, _ = oracle.lstsq(B, oracle.coulomb(src, qs, pts, field=False))
    img_xyz, img_q, _, _ = hsma.surface_images(plan, A)
    g = np.random.default_rng(2)
    tgt = g.random((30, 3)) - 0.5
    phi, fld = oracle.coulomb(img_xyz, img_q, tgt)
    ref_phi, ref_fld = oracle.coulomb(src, qs, tgt)
    assert np.abs(phi - ref_phi).max() < 1e-8 * np.abs(ref_phi).max()
    assert np.abs(fld - ref_fld).max() < 1e-7 * np.abs(ref_fld).max()


def test_mapping_of_constant_and_charge_balance():
    plan = _plan_for_mapping(P=6, F2=377)
    A = np.zeros((plan.P + 1) ** 2)
    A[0] = 1.0 / plan.Bq[0, 0]  # Phi_out = 1 everywhere
    img_xyz, img_q, phi_s, sigma = hsma.surface_images(plan, A)
    assert np.abs(sigma).max() == 0.0
    g = np.random.default_rng(3)
    phi = oracle.coulomb(img_xyz, img_q, g.random((20, 3)) - 0.5, field=False)
    # a constant maps to a constant, up to the O(dr^2) dipole approximation
    assert np.abs(phi - 1.0).max() < 1e-8
    # random harmonic: each dipole pair carries zero net charge, sigma-images sum to ~0 (Gauss)
    A = g.standard_normal((plan.P + 1) ** 2)
    img_xyz, img_q, _, _ = hsma.surface_images(plan, A)
    nd = len(plan.weights)
    np.testing.assert_allclose(img_q[nd:2 * nd] + img_q[2 * nd:], 0.0, atol=1e-12 * np.abs(img_q).max())
    assert abs(img_q[:nd].sum()) < 1e-10 * np.abs(img_q[:nd]).sum()


def test_nonneutral_periodic_rejected():
    L = np.ones(3)
    plan = _plan_for_mapping(P=4, F2=89)
    with pytest.raises(ValueError):
        hsma.energy_forces(np.full((2, 3), 0.3), np.array([1.0, 0.5]), plan)


def test_series_far_field_matches_surface_images():
    # the two ways of bringing the fitted far field to the particles agree to
    # the mapping accuracy (quadrature + O(dr^2)), and the series' field is
    # minus the gradient of its potential
    L = np.ones(3)
    xyz, q = inputs.random_neutral(24, L, 33)
    Rs = hsma.alpha_to_rs(L, 2.0)
    plan = hsma.make_plan(L, hsma.PERIODIC, 14, Rs, 2 * 14 * 14, 987)
    img = hsma.energy_forces(xyz, q, plan)
    ser = hsma.energy_forces_series(xyz, q, plan)
    assert abs(ser["energy"] - img["energy"]) <= 1e-9 * abs(img["energy"])
    np.testing.assert_allclose(ser["phi_out"], img["phi_out"], rtol=0, atol=1e-9 * np.abs(img["phi_out"]).max())
    np.testing.assert_allclose(ser["e_out"], img["e_out"], rtol=0, atol=1e-7 * np.abs(img["e_out"]).max())
    # both against Ewald
    _, fld, U = checks.ewald_periodic(xyz, q, L)
    assert abs(ser["energy"] - U) <= 1e-7 * abs(U)


def test_structure_factor_ewald_equals_pairwise_ewald():
    L = np.array([1.0, 1.0, 1.3])
    xyz, q = inputs.random_neutral(20, L, 44)
    p1, f1, U1 = checks.ewald_periodic(xyz, q, L)
    p2, f2, U2 = checks.ewald_periodic_fast(xyz, q, L)
    np.testing.assert_allclose(p2, p1, rtol=0, atol=1e-12 * np.abs(p1).max())
    np.testing.assert_allclose(f2, f1, rtol=0, atol=1e-11 * np.abs(f1).max())
    xyz, q, a = checks.nacl_lattice(MADELUNG["n_side"], MADELUNG["L"])
    _, _, U = checks.ewald_periodic_fast(xyz, q, np.full(3, MADELUNG["L"]))
    assert abs(checks.madelung_from_energy(U, len(q), a) - MADELUNG["madelung_constant"]) < 1e-12
