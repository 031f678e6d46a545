"""The oracle's cell-list Ewald sum (the reference of the large-N study of
Sec. III) pinned to the plain Ewald sum and to the NaCl Madelung constant."""
import json
import os

import numpy as np

from paper_1806_04801_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_cell_list_ewald_matches_plain_ewald():
    import oracle
    from oracle import checks
    xyz, q = I.random_neutral(600, (1.0, 1.0, 1.0), 31)
    pick = np.array([0, 5, 77, 599])
    pot_ref, fld_ref, U_ref = checks.ewald_periodic_fast(xyz, q, np.ones(3))
    U, pot, fld = oracle.ewald_cells(xyz, q, np.ones(3), pick=pick)
    assert abs(U - U_ref) <= 1e-11 * abs(U_ref)
    np.testing.assert_allclose(pot, pot_ref[pick], rtol=0, atol=1e-10)
    np.testing.assert_allclose(fld, fld_ref[pick], rtol=0, atol=1e-8)
    # the picked-particles-only form gives the same potentials and fields
    U2, pot2, fld2 = oracle.ewald_cells(xyz, q, np.ones(3), pick=pick, energy=False)
    assert U2 is None
    np.testing.assert_allclose(pot2, pot, rtol=0, atol=1e-12)
    np.testing.assert_allclose(fld2, fld, rtol=0, atol=1e-10)
    # a rectangular box (cells per axis differ)
    L = np.array([1.0, 1.3, 0.8])
    xyz, q = I.random_neutral(400, L, 32)
    pot_ref, _, U_ref = checks.ewald_periodic_fast(xyz, q, L)
    U, pot, _ = oracle.ewald_cells(xyz, q, L, pick=np.arange(5))
    # |U| (33) is a cancellation of terms of order sum q^2 (400): compare on that scale
    assert abs(U - U_ref) <= 1e-11 * max(abs(U_ref), float(np.sum(q * q)))
    np.testing.assert_allclose(pot, pot_ref[:5], rtol=0, atol=1e-10)


def test_cell_list_ewald_madelung():
    import oracle
    from oracle import checks
    g = json.load(open(os.path.join(GOLD, "madelung_nacl.json")))
    xyz, q, a = checks.nacl_lattice(g["n_side"], g["L"])
    U, _, _ = oracle.ewald_cells(xyz, q, np.full(3, g["L"]))
    assert abs(checks.madelung_from_energy(U, len(q), a) - g["madelung_constant"]) < 1e-11


def test_cell_list_ewald_translation_invariance():
    """Shifting every charge by the same vector (with wrapping) leaves the
    energy unchanged: the cell lists and the minimum image are consistent."""
    import oracle
    xyz, q = I.lattice_random_sign(12, 1.0, seed_offset=512)
    U0, _, _ = oracle.ewald_cells(xyz, q, np.ones(3))
    U1, _, _ = oracle.ewald_cells(np.mod(xyz + np.array([0.37, -0.21, 0.55]), 1.0), q, np.ones(3))
    assert abs(U1 - U0) <= 1e-11 * abs(U0)
