"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds only random-number generation and workload shapes; it
contains none of the method's arithmetic, so both the CUDA path and the CPU
oracle can be fed from it.

Positions are in the box frame [0, L_a).  Every generator is deterministic in
its seed (numpy PCG64).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 1806_04801
PERIODIC = 0
GROUNDED = 1


@dataclass(frozen=True)
class Workload:
    """Plan parameters of one workload: box, boundary, harmonic order p,
    auxiliary-sphere radius R, requested surface points Q, monitoring points."""
    name: str
    box: tuple
    bc: int
    p: int
    R: float
    Q: int
    Kmon: int


def _rs_sqrt3(box):
    # auxiliary radius sqrt(3) x circumradius (= 1.5 L for a cube)
    return math.sqrt(3.0) * 0.5 * math.sqrt(sum(b * b for b in box))


# The five workload shapes (cubic periodic boxes at L = 1 and a 1x1x2 grounded
# cavity).  R = 1.5 L for the cube; sqrt(3) x circumradius for the cavity.
SMALL_PERIODIC = Workload("periodic-N1000-p8", (1.0, 1.0, 1.0), PERIODIC, 8, 1.5, 2000, 600)
LARGE_PERIODIC = Workload("periodic-N100000-p12", (1.0, 1.0, 1.0), PERIODIC, 12, 1.5, 8000, 2000)
GROUNDED_CAVITY = Workload("grounded-1x1x2-N20000-p10", (1.0, 1.0, 2.0), GROUNDED, 10,
                           _rs_sqrt3((1.0, 1.0, 2.0)), 6000, 1500)
BATCH_PERIODIC = Workload("batched-256-periodic-p10", (1.0, 1.0, 1.0), PERIODIC, 10, 1.5, 6000, 1500)
SERVING_PERIODIC = Workload("serving-periodic-p10", (1.0, 1.0, 1.0), PERIODIC, 10, 1.5, 6000, 1500)


def rng(seed_offset: int = 0) -> np.random.Generator:
    """The PCG64 generator of seed 1806_04801 + seed_offset."""
    return np.random.default_rng(SEED_BASE + seed_offset)


def uniform_pm1(n: int, box, seed_offset: int = 0, margin: float = 0.0):
    """n uniform positions (optional wall margin) with n/2 charges +1 and n/2
    charges -1 in random order (n rounded up to even)."""
    n = n + (n % 2)
    g = rng(seed_offset)
    box = np.asarray(box, dtype=np.float64)
    xyz = margin + g.random((n, 3)) * (box - 2.0 * margin)
    q = np.concatenate([np.ones(n // 2), -np.ones(n // 2)])
    g.shuffle(q)
    return xyz, q


def uniform_gauss(n: int, box, seed_offset: int = 0):
    """n uniform positions with charges N(0,1) minus their mean (neutral)."""
    g = rng(seed_offset)
    box = np.asarray(box, dtype=np.float64)
    xyz = g.random((n, 3)) * box
    q = g.standard_normal(n)
    q -= q.mean()
    return xyz, q


def small_periodic():
    """1000 charges, +-1, uniform in the unit periodic box."""
    return uniform_pm1(1000, SMALL_PERIODIC.box, seed_offset=0)


def large_periodic(n: int = 100_000):
    """100000 charges N(0,1) mean-subtracted, uniform in the unit periodic box."""
    return uniform_gauss(n, LARGE_PERIODIC.box, seed_offset=1)


def grounded_cavity(n: int = 20_000):
    """20000 charges +-1 uniform in the 1x1x2 box with a 0.05 wall margin."""
    return uniform_pm1(n, GROUNDED_CAVITY.box, seed_offset=2, margin=0.05)


def log_uniform_sizes(count: int, lo: int, hi: int, seed_offset: int):
    """count sizes log-uniform in [lo, hi], rounded to integers and up to even."""
    g = rng(seed_offset)
    n = np.exp(g.uniform(math.log(lo), math.log(hi), size=count))
    n = np.round(n).astype(np.int64)
    return n + (n % 2)


def batch_periodic(count: int = 256, lo: int = 500, hi: int = 50_000, seed_offset: int = 3):
    """Independent periodic unit boxes with log-uniform sizes, +-1 charges."""
    sizes = log_uniform_sizes(count, lo, hi, seed_offset)
    systems = [uniform_pm1(int(n), BATCH_PERIODIC.box, seed_offset=1000 + 7 * i + seed_offset)
               for i, n in enumerate(sizes)]
    return systems


def poisson_trace(count: int, rate_hz: float = 2000.0, lo: int = 1000, hi: int = 200_000,
                  seed_offset: int = 4):
    """Arrival times (s) of a Poisson stream and the sizes of its systems."""
    g = rng(seed_offset)
    gaps = g.exponential(1.0 / rate_hz, size=count)
    t = np.cumsum(gaps) - gaps[0]
    sizes = log_uniform_sizes(count, lo, hi, seed_offset + 100)
    return t, sizes


def nacl_lattice(n_side: int = 4, L: float = 2.0):
    """Rock-salt arrangement: unit charges of alternating sign at the cell
    centres of an n_side^3 grid (the lattice of the paper's first example)."""
    a = L / n_side
    idx = np.array(list(itertools.product(range(n_side), repeat=3)), dtype=np.float64)
    return (idx + 0.5) * a, (-1.0) ** idx.sum(axis=1)


def lattice_random_sign(n_side: int, L: float = 1.0, seed_offset: int = 5):
    """Unit charges of random sign on a uniform lattice, neutral overall
    (the paper's large-N accuracy workload)."""
    n = n_side**3
    g = rng(seed_offset)
    a = L / n_side
    idx = np.array(list(itertools.product(range(n_side), repeat=3)), dtype=np.float64)
    q = np.concatenate([np.ones(n // 2), -np.ones(n - n // 2)])
    if n % 2:
        q[-1] = 0.0
    g.shuffle(q)
    return (idx + 0.5) * a, q


def random_neutral(n: int, box, seed_offset: int):
    """Small random neutral periodic box, alternating +-1 (n even)."""
    g = rng(seed_offset)
    box = np.asarray(box, dtype=np.float64)
    xyz = g.random((n, 3)) * box
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    return xyz, q
