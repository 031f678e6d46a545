"""Independent checkers for the HSMA oracle (test infrastructure only).

These do not use any part of the HSMA pipeline; they compute the exact
electrostatics of the paper's model problems by other means:

* ``ewald_periodic`` -- Ewald summation of the periodic sum of Sec. II
  (conducting surroundings, the convention a strictly periodic potential
  implies);
* ``grounded_box_exact`` -- the conducting-wall box of Eq. "diel" at
  gamma = -1.  Its image lattice is the 2L-periodic lattice of the eight
  reflections s∘r + p∘L (p in {0,1}^3, s_a = (-1)^p_a, charge (-1)^{|p|} q); that
  cell is neutral and odd under every wall reflection, so its periodic
  potential vanishes on the walls and is the Dirichlet solution;
* ``madelung_from_energy`` -- the NaCl Madelung constant from a lattice energy
  (Sec. III, first example).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import ewald, ewald_sf


def _ewald_params(L):
    L = np.asarray(L, dtype=np.float64)
    nreal = 3
    beta = 3.0 / float(L.min())  # erfc(beta * 2 Lmin) ~ 2e-17
    kcut = 2.0 * beta * math.sqrt(math.log(1e17))
    kmax = int(math.ceil(kcut * float(L.max()) / (2.0 * math.pi))) + 1
    return beta, nreal, kmax


def ewald_periodic(xyz, q, L):
    """Potential (self excluded), field and energy of a neutral periodic cell."""
    beta, nreal, kmax = _ewald_params(L)
    pot, fld = ewald(xyz, q, L, beta, nreal, kmax)
    q = np.asarray(q, dtype=np.float64)
    return pot, fld, 0.5 * float(np.dot(q, pot))


def grounded_box_exact(xyz_box, q, L):
    """Exact potential, field and energy for charges in a grounded box.

    xyz_box: positions in the box frame [0, L_a); they are centred first.
    """
    L = np.asarray(L, dtype=np.float64)
    c = np.asarray(xyz_box, dtype=np.float64).reshape(-1, 3) - 0.5 * L
    q = np.asarray(q, dtype=np.float64)
    pos, chg = [], []
    for p in itertools.product((0, 1), repeat=3):
        s = np.array([(-1.0) ** pa for pa in p])
        pos.append(c * s + np.array(p) * L)
        chg.append(q * (-1.0) ** sum(p))
    pos = np.concatenate(pos)
    chg = np.concatenate(chg)
    pot, fld, _ = ewald_periodic(pos, chg, 2.0 * L)
    n = q.shape[0]
    pot, fld = pot[:n], fld[:n]
    return pot, fld, 0.5 * float(np.dot(q, pot))


def nacl_lattice(n_side: int, L: float):
    """NaCl-like lattice: n_side^3 unit charges at cell centres of an
    n_side^3 grid of side L, alternating sign (box frame [0, L))."""
    a = L / n_side
    idx = np.array(list(itertools.product(range(n_side), repeat=3)), dtype=np.float64)
    xyz = (idx + 0.5) * a
    q = (-1.0) ** idx.sum(axis=1)
    return xyz, q, a


def madelung_from_energy(U, n_ions: int, a: float, qabs: float = 1.0):
    """U = -(N/2) M q^2 / a for a rock-salt lattice, so M = -2 a U / (N q^2)."""
    return -2.0 * a * U / (n_ions * qabs * qabs)


def ewald_periodic_fast(xyz, q, L):
    """ewald_periodic with the structure-factor reciprocal sum (for a few
    thousand charges)."""
    beta, nreal, kmax = _ewald_params(L)
    pot, fld = ewald_sf(xyz, q, L, beta, nreal, kmax)
    q = np.asarray(q, dtype=np.float64)
    return pot, fld, 0.5 * float(np.dot(q, pot))
