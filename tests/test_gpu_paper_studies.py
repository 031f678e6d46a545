"""The paper's accuracy studies (Sec. III) run on the GPU path.

* NaCl Madelung constant (first example: 64 unit charges, L = 2, periodic,
  alpha = 2, F2 = 987) over P: the GPU value matches the oracle's at every P,
  stays inside the truncation bound of Sec. II.A and converges at ~alpha^-P;
* the grounded three-charge box (second example, Delta r = 1e-4 Rs) against
  the exact doubled-cell image lattice;
* forces (third example): the lattice forces vanish by symmetry, the grounded
  forces match the exact lattice;
* random-sign charges on a lattice (large-N example, alpha = 2, P = 25)
  against an Ewald sum.
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
