"""The paper's accuracy studies (Sec. III) run on the GPU path.

* NaCl Madelung constant (first example: 64 unit charges, L = 2, periodic,
  alpha = 2, F2 = 987) over P: the GPU value matches the oracle's at every P,
  stays inside the truncation bound of Sec. II.A and converges at ~alpha^-P;
* the grounded three-charge box (second example, Delta r = 1e-4 Rs) against
  the exact doubled-cell image lattice;
* forces (third example): the lattice forces vanish by symmetry, the grounded
  forces match the exact lattice;
* random-sign charges on a lattice (large-N example, alpha = 2, P = 25)
  against an Ewald sum;
* error against the number of surface images N_o = 6 (F2 + 1) (first and
  second examples, Fig. 2a/2c, and the large-N example, Fig. 4a): the curves
  flatten once N_o > 3600 (F2 >= 610), where the quadrature stops being the
  leading error;
* random-sign lattices of 1k to 512k charges (Fig. 4a) against the oracle's
  cell-list Ewald sum: energies up to 64k, forces on sampled charges at all
  sizes; and the error against P for two alpha (Fig. 4b).
Each study prints its table (pytest -s)."""
import json
import math
import os

import numpy as np
import pytest

from gpu_common import rel_energy_err, to_dev
from paper_1806_04801_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available()
    from paper_1806_04801_gb300 import build
    build.build()


def hs():
    from paper_1806_04801_gb300 import hsma
    return hsma


def test_madelung_convergence():
    from oracle import checks, hsma as oh
    g = json.load(open(os.path.join(GOLD, "madelung_nacl.json")))
    xyz, q, a = checks.nacl_lattice(g["n_side"], g["L"])
    L = np.full(3, g["L"])
    alpha = g["alpha"]
    Rs = oh.alpha_to_rs(L, alpha)
    d0 = len(q) / np.prod(L)
    rows = []
    for P in (8, 12, 16, 20, 25):
        K = 2 * P * P
        res = {}
        for prec in ("fp64", "fp32"):
            with hs().Plan(L, I.PERIODIC, P, Rs, 0, K, precision=prec, fib_F2=g["F2"]) as plan:
                U, F, _, _ = plan.energy_forces(*to_dev(xyz, q))
                res[prec] = (checks.madelung_from_energy(U, len(q), a), float(np.abs(F.cpu().numpy()).max()))
        ref = oh.energy_forces(xyz, q, oh.make_plan(L, I.PERIODIC, P, Rs, K, g["F2"]))
        M_or = checks.madelung_from_energy(ref["energy"], len(q), a)
        M64, F64 = res["fp64"]
        err = abs(M64 - g["madelung_constant"])
        assert abs(M64 - M_or) <= 1e-10 * M_or, (P, M64, M_or)
        assert err <= a * oh.error_bound_potential(alpha, P, Rs, d0, 1.0)
        rows.append((P, M64, err, abs(res["fp32"][0] - g["madelung_constant"]), F64))
    print("\nMadelung (alpha=2, F2=987): P, M_gpu_fp64, |err| fp64, |err| fp32, max|F| fp64")
    for r in rows:
        print(f"  {r[0]:3d} {r[1]:.15f} {r[2]:.3e} {r[3]:.3e} {r[4]:.3e}")
    errs = [r[2] for r in rows]
    assert errs[-1] < 1e-11
    assert (math.log(errs[3]) - math.log(errs[0])) / 12 < -0.8 * math.log(alpha)
    # lattice forces vanish by symmetry: they converge like the energy
    assert rows[-1][4] < 1e-8 and rows[-1][4] < rows[0][4]


def test_dirichlet_three_charges():
    from oracle import checks, hsma as oh
    g = json.load(open(os.path.join(GOLD, "dirichlet_three_charges.json")))
    L = np.full(3, g["L"])
    q = np.array(g["charges"])
    xyz = np.array(g["positions_centred"]) + 0.5 * L
    _, fld, U_exact = checks.grounded_box_exact(xyz, q, L)
    F_exact = q[:, None] * fld
    Rs = oh.alpha_to_rs(L, 2.0)
    rows = []
    for P in (8, 12, 16, 20):
        with hs().Plan(L, I.GROUNDED, P, Rs, 0, 2 * P * P, precision="fp64", fib_F2=987,
                       dr_rel=g["dr_rel"]) as plan:
            U, F, _, _ = plan.energy_forces(*to_dev(xyz, q))
        F = F.cpu().numpy()
        rows.append((P, U, abs(U - U_exact) / abs(U_exact), float(np.abs(F - F_exact).max())))
    print(f"\nDirichlet 3-charge box (alpha=2, dr=1e-4 Rs), exact U = {U_exact:.15f}: P, U, rel err, max|dF|")
    for r in rows:
        print(f"  {r[0]:3d} {r[1]:.15f} {r[2]:.3e} {r[3]:.3e}")
    assert rows[-1][2] < 1e-9 and rows[-1][3] < 1e-7
    assert rows[0][2] > rows[-1][2] and rows[0][3] > rows[-1][3]


@pytest.mark.parametrize("n_side", [10, 12])
def test_random_sign_lattice_against_ewald(n_side):
    from oracle import checks, hsma as oh
    xyz, q = I.lattice_random_sign(n_side, 1.0, seed_offset=500 + n_side)
    L = np.ones(3)
    _, fld, U = checks.ewald_periodic_fast(xyz, q, L)
    F_ref = q[:, None] * fld
    Rs = oh.alpha_to_rs(L, 2.0)
    out = {}
    for prec in ("fp64", "fp32"):
        with hs().Plan(L, I.PERIODIC, 25, Rs, 0, 2 * 25 * 25, precision=prec, fib_F2=987) as plan:
            Ug, Fg, _, _ = plan.energy_forces(*to_dev(xyz, q))
        Fg = Fg.cpu().numpy()
        out[prec] = (rel_energy_err(Ug, U, q), float(np.sqrt(np.mean((Fg - F_ref) ** 2) / np.mean(F_ref ** 2))))
    print(f"\nrandom-sign lattice {n_side}^3 vs Ewald (alpha=2, P=25): "
          f"fp64 energy {out['fp64'][0]:.2e} force {out['fp64'][1]:.2e}; "
          f"fp32 energy {out['fp32'][0]:.2e} force {out['fp32'][1]:.2e}")
    assert out["fp64"][0] < 1e-9 and out["fp64"][1] < 1e-7
    assert out["fp32"][0] < 1e-6 and out["fp32"][1] < 1e-5


F2_SWEEP = [89, 144, 233, 377, 610, 987, 1597]  # N_o = 540 ... 9588


def _plateau_checks(table, F2s, plateau_from, what, floor=1e-11):
    """Rows of errors over F2: beyond plateau_from every error is within 10%
    (plus a rounding floor) of the one at the largest F2; the smallest F2
    leaves a far larger error where the expansion itself is accurate."""
    for P, errs in table:
        last = errs[-1]
        for F2, e in zip(F2s, errs):
            if F2 >= plateau_from:
                assert e <= 1.1 * last + floor, (what, P, F2, e, last)
        if last < 1e-6:
            assert errs[0] > 10.0 * last, (what, P, errs)


def test_madelung_error_vs_surface_images():
    """Fig. 2a: the NaCl Madelung error against N_o for five P (alpha = 2):
    flat once F2 >= 610 (N_o > 3600).  The GPU FP64 value equals the
    oracle's at every (P, F2) of two orders, so each F2's Fibonacci nodes and
    weights are checked too."""
    from oracle import checks, hsma as oh
    g = json.load(open(os.path.join(GOLD, "madelung_nacl.json")))
    xyz, q, a = checks.nacl_lattice(g["n_side"], g["L"])
    L = np.full(3, g["L"])
    Rs = oh.alpha_to_rs(L, 2.0)
    table = []
    for P in (8, 12, 16, 20, 25):
        errs = []
        for F2 in F2_SWEEP:
            with hs().Plan(L, I.PERIODIC, P, Rs, 0, 2 * P * P, precision="fp64", fib_F2=F2) as plan:
                U = plan.energy_forces(*to_dev(xyz, q))[0]
            M = checks.madelung_from_energy(U, len(q), a)
            if P in (12, 20):
                ref = oh.energy_forces(xyz, q, oh.make_plan(L, I.PERIODIC, P, Rs, 2 * P * P, F2))
                assert abs(U - ref["energy"]) <= 1e-10 * abs(ref["energy"]), (P, F2)
            errs.append(abs(M - g["madelung_constant"]))
        table.append((P, errs))
    print("\nMadelung |error| vs F2 " + str(F2_SWEEP) + " (alpha = 2), rows P = 8, 12, 16, 20, 25")
    for P, errs in table:
        print(f"  P={P:2d} " + " ".join(f"{e:.2e}" for e in errs))
    _plateau_checks(table, F2_SWEEP, 610, "madelung")


def test_dirichlet_error_vs_surface_images():
    """Fig. 2c: the grounded three-charge box (Delta r = 1e-4 Rs) against the
    exact image lattice, over N_o for four P: flat once F2 >= 610."""
    from oracle import checks, hsma as oh
    g = json.load(open(os.path.join(GOLD, "dirichlet_three_charges.json")))
    L = np.full(3, g["L"])
    q = np.array(g["charges"])
    xyz = np.array(g["positions_centred"]) + 0.5 * L
    _, _, U_exact = checks.grounded_box_exact(xyz, q, L)
    Rs = oh.alpha_to_rs(L, 2.0)
    table = []
    for P in (8, 12, 16, 20):
        errs = []
        for F2 in F2_SWEEP:
            with hs().Plan(L, I.GROUNDED, P, Rs, 0, 2 * P * P, precision="fp64", fib_F2=F2,
                           dr_rel=g["dr_rel"]) as plan:
                U = plan.energy_forces(*to_dev(xyz, q))[0]
            errs.append(abs(U - U_exact) / abs(U_exact))
        table.append((P, errs))
    print("\nGrounded 3-charge box, relative energy error vs F2 " + str(F2_SWEEP) + ", rows P = 8, 12, 16, 20")
    for P, errs in table:
        print(f"  P={P:2d} " + " ".join(f"{e:.2e}" for e in errs))
    _plateau_checks(table, F2_SWEEP, 610, "dirichlet", floor=5e-10)


def _lattice_case(n_side):
    import oracle
    xyz, q = I.lattice_random_sign(n_side, 1.0, seed_offset=500 + n_side)
    n = len(q)
    pick = np.linspace(0, n - 1, 64).astype(np.int64)
    U_ref, pot_ref, fld_ref = oracle.ewald_cells(xyz, q, np.ones(3), pick=pick, energy=n_side <= 40)
    return xyz, q, pick, U_ref, pot_ref, q[pick, None] * fld_ref


def _lattice_errors(xyz, q, pick, U_ref, pot_ref, F_ref, prec, F2, P=25, alpha=2.0):
    from oracle import hsma as oh
    L = np.ones(3)
    with hs().Plan(L, I.PERIODIC, P, oh.alpha_to_rs(L, alpha), 0, 2 * P * P, precision=prec,
                   fib_F2=F2) as plan:
        U, F, pot, _ = plan.energy_forces(*to_dev(xyz, q), potentials=True)
    F = F.cpu().numpy()[pick]
    pot = pot.cpu().numpy()[pick]
    # the periodic potential is fixed up to a constant (A_00 = 0): compare it
    # with the Ewald potential after removing the mean over the sampled charges
    dp = (pot - pot.mean()) - (pot_ref - pot_ref.mean())
    return {"energy": None if U_ref is None else abs(U - U_ref) / abs(U_ref),
            "force": float(np.sqrt(np.mean((F - F_ref) ** 2) / np.mean(F_ref ** 2))),
            "pot": float(np.sqrt(np.mean(dp ** 2) / np.mean((pot_ref - pot_ref.mean()) ** 2)))}


def test_random_sign_lattices_error_vs_surface_images():
    """Fig. 4a: random-sign lattices of 1k and 8k charges (alpha = 2, P = 25)
    against the Ewald sum over N_o: the same curve for both sizes, flat once
    F2 >= 987 at this P."""
    rows = []
    for n_side in (10, 20):
        case = _lattice_case(n_side)
        errs = [_lattice_errors(*case, "fp64", F2)["energy"] for F2 in F2_SWEEP]
        rows.append((n_side ** 3, errs))
    print("\nrandom-sign lattices vs Ewald, relative energy error vs F2 " + str(F2_SWEEP) + " (alpha 2, P 25)")
    for n, errs in rows:
        print(f"  N={n:6d} " + " ".join(f"{e:.2e}" for e in errs))
    _plateau_checks(rows, F2_SWEEP, 987, "lattice", floor=1e-10)
    for n, errs in rows:
        assert errs[F2_SWEEP.index(987)] < 1e-9 and errs[0] > 1e-3, (n, errs)


def test_random_sign_lattices_up_to_512k():
    """Fig. 4a at N_o = 5928 for N = 1k, 8k, 64k and 512k charges: energies
    against the Ewald sum up to 64k (FP64 and the FP32 pair sums), forces
    and potential differences of 64 sampled charges at every size."""
    rows = []
    for n_side in (10, 20, 40, 80):
        case = _lattice_case(n_side)
        precs = ("fp64", "fp32") if n_side <= 40 else ("fp32",)
        for prec in precs:
            e = _lattice_errors(*case, prec, 987)
            rows.append((n_side ** 3, prec, e))
            tol = {"fp64": (1e-9, 1e-8, 1e-8), "fp32": (1e-6, 1e-5, 1e-5)}[prec]
            if e["energy"] is not None:
                assert e["energy"] < tol[0], (n_side, prec, e)
            assert e["force"] < tol[1] and e["pot"] < tol[2], (n_side, prec, e)
    print("\nrandom-sign lattices vs Ewald (alpha 2, P 25, N_o 5928): N, precision, energy, force, potential")
    for n, prec, e in rows:
        en = "   --   " if e["energy"] is None else f"{e['energy']:.2e}"
        print(f"  {n:7d} {prec} {en} {e['force']:.2e} {e['pot']:.2e}")


def test_random_sign_lattice_error_vs_order():
    """Fig. 4b: 8000 random-sign charges against the Ewald sum over P for
    alpha = 1.5 and 2 (N_o = 5928, FP64): the error falls at least at about
    the rate alpha^-P of the Sec. II.A estimate, and the larger alpha is more
    accurate at every P."""
    case = _lattice_case(20)
    errs = {}
    for alpha in (1.5, 2.0):
        errs[alpha] = [_lattice_errors(*case, "fp64", 987, P=P, alpha=alpha)["energy"] for P in (8, 12, 16, 20, 25)]
    print("\nrandom-sign lattice 20^3 vs Ewald, relative energy error for P = 8, 12, 16, 20, 25")
    for alpha, e in errs.items():
        print(f"  alpha={alpha}: " + " ".join(f"{x:.2e}" for x in e))
    for alpha, e in errs.items():
        assert all(b < a for a, b in zip(e, e[1:])), (alpha, e)
        assert (math.log(e[-1]) - math.log(e[0])) / 17 < -0.8 * math.log(alpha), (alpha, e)
    assert all(a2 < a1 for a1, a2 in zip(errs[1.5], errs[2.0]))
