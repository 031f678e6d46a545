"""The HSMA algorithm of arXiv:1806.04801, Sec. II, composed from the oracle's
FP64 primitives in the order the paper gives.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Preparation step (Sec. II.C, Table I): monitoring points, fitting matrix and
its least-squares factorisation, integration points and the mapping matrix.
Update step (Sec. II.C): images inside the auxiliary sphere, the right-hand
side of the least-squares problem, the coefficients A_nm, the surface images
Q_j (Sec. II.B) and finally energies and forces.

Readings of points the paper leaves open:
  * periodic monitoring points: the Fibonacci latitude grid on the circumsphere
    of the box; the fitting residual is Phi(x_i) - Phi(x~_i) (Sec. II.A);
  * the n = 0 column of the periodic fitting matrix is identically zero
    (B_0^0 is constant), so A_00 is undetermined and set to 0: a constant
    shift of the potential does not change energy or forces of a neutral
    system;
  * grounded (conducting) walls are the gamma = -1 limit of Eq. "diel" with a
    Dirichlet residual v_i = Phi(x_i) on the walls;
  * the Fibonacci integration formula is used literally (its two pole nodes
    carry zero weight);
  * Delta r = 1e-5 Rs (periodic) and 1e-4 Rs (grounded), Sec. III;
  * energy U = 1/2 sum_i q_i [Phi_in'(r_i) + Phi_out(r_i)] and force
    F_i = q_i E(r_i), where Phi_in' skips only the particle's own copy.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import basis, coulomb, inset, lstsq, monitor_faces, monitor_sphere, quadrature, wrap_into_box

PERIODIC = 0
GROUNDED = 1


def fibonacci_numbers(limit: int = 10**7):
    """Fibonacci numbers 1, 2, 3, 5, ... up to limit (the F2 candidates of Sec. II.B)."""
    a, b = 1, 2
    out = [1, 2]
    while b < limit:
        a, b = b, a + b
        out.append(b)
    return out


def fib_from_points(Q: int):
    """F2 whose 6(F2+1) image count (Sec. II.B) is nearest to Q (ties to the
    larger), and its predecessor F1."""
    fib = fibonacci_numbers()
    best = None
    for i in range(1, len(fib)):
        d = abs(6 * (fib[i] + 1) - Q)
        if best is None or d < best[0] or (d == best[0] and fib[i] > best[1]):
            best = (d, fib[i], fib[i - 1])
    return best[1], best[2]


def fib_predecessor(F2: int) -> int:
    """F1: the Fibonacci number before F2 (azimuth step of the Fibonacci integration, Sec. II.B)."""
    fib = fibonacci_numbers(F2 + 1)
    if F2 not in fib:
        raise ValueError("F2 must be a Fibonacci number")
    i = fib.index(F2)
    return fib[i - 1] if i > 0 else 1


def degree_of_index(nb: int):
    """Degree n of basis index k = n^2 + n + m."""
    return np.floor(np.sqrt(np.arange(nb) + 0.5)).astype(np.int64)


@dataclass
class Plan:
    """Matrices and point sets of the preparation step (Sec. II.C, Table I upper half)."""
    box: np.ndarray
    bc: int
    P: int
    Rs: float
    Kmon: int
    F2: int
    F1: int
    dr: float
    x_mon: np.ndarray
    x_mon_partner: np.ndarray | None
    M: np.ndarray
    dirs: np.ndarray
    weights: np.ndarray
    Bq: np.ndarray
    extra: dict = field(default_factory=dict)


def make_plan(box, bc: int, P: int, Rs: float, Kmon: int, F2: int, dr_rel: float | None = None) -> Plan:
    """Preparation step (Sec. II.C): independent of the charges."""
    L = np.asarray(box, dtype=np.float64)
    R0 = 0.5 * float(np.linalg.norm(L))
    if not Rs > R0:
        raise ValueError("the auxiliary sphere must enclose the box (alpha > 1)")
    if dr_rel is None:
        dr_rel = 1e-5 if bc == PERIODIC else 1e-4
    F1 = fib_predecessor(F2)
    if bc == PERIODIC:
        x = monitor_sphere(Kmon, R0)
        xt = wrap_into_box(x, L)
        M = (basis(x, P, Rs) - basis(xt, P, Rs))[:, 1:]
    else:
        x = monitor_faces(Kmon, L)
        xt = None
        M = basis(x, P, Rs)
    dirs, w = quadrature(F2, F1, Rs)
    Bq = basis(Rs * dirs, P, Rs)
    return Plan(L, bc, P, Rs, Kmon, F2, F1, dr_rel * Rs, x, xt, M, dirs, w, Bq)


def centre_positions(xyz, L, bc: int):
    """Box frame [0, L_a) -> centred frame [-L_a/2, L_a/2); periodic inputs are
    wrapped first, grounded inputs must lie strictly inside the box."""
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    L = np.asarray(L, dtype=np.float64)
    if bc == PERIODIC:
        xyz = xyz - np.floor(xyz / L) * L
    else:
        if np.any(xyz <= 0.0) or np.any(xyz >= L):
            raise ValueError("grounded box: particle on or outside a wall")
    return xyz - 0.5 * L


def surface_images(plan: Plan, A):
    """Sec. II.B: from the harmonic coefficients to the N_o = 6(F2+1) point
    images on the spheres Rs - dr/2, Rs, Rs + dr/2 (literal three-surface form).

    sigma(r') = (1/r') sum n A_nm B_nm(r')          (surface charge)
    mu^pm = Rs^2 Phi_out / (dr (Rs pm dr/2)^2)      (two charge layers)
    Quadrature weights on a sphere of radius R scale as R^2, so each node
    carries charge w sigma / 4pi on Rs, +w Phi_out / (4 pi dr) on Rs - dr/2 and
    -w Phi_out / (4 pi dr) on Rs + dr/2.
    """
    nb = plan.Bq.shape[1]
    n = degree_of_index(nb)
    phi_s = plan.Bq @ A
    sigma = (plan.Bq @ (n * A)) / plan.Rs
    Rm = plan.Rs - 0.5 * plan.dr
    Rp = plan.Rs + 0.5 * plan.dr
    q_sigma = plan.weights * sigma / (4.0 * math.pi)
    mu_m = plan.Rs**2 * phi_s / (plan.dr * Rm**2)
    mu_p = plan.Rs**2 * phi_s / (plan.dr * Rp**2)
    q_inner = plan.weights * (Rm / plan.Rs) ** 2 * mu_m / (4.0 * math.pi)
    q_outer = -plan.weights * (Rp / plan.Rs) ** 2 * mu_p / (4.0 * math.pi)
    pos = np.concatenate([plan.Rs * plan.dirs, Rm * plan.dirs, Rp * plan.dirs])
    chg = np.concatenate([q_sigma, q_inner, q_outer])
    return pos, chg, phi_s, sigma


def energy_forces(xyz, q, plan: Plan, nthreads: int = 1, sample=None) -> dict:
    """Update step of Sec. II.C for one configuration.

    sample: optional particle indices; when given, potentials and forces are
    evaluated only there (the fit still uses the full in-set) and no energy is
    returned.
    """
    L = plan.box
    q = np.asarray(q, dtype=np.float64)
    n = q.shape[0]
    if plan.bc == PERIODIC and abs(q.sum()) > 1e-12 * max(np.abs(q).sum(), 1e-300):
        raise ValueError("periodic system must be neutral")
    c = centre_positions(xyz, L, plan.bc)

    # 1. images inside the auxiliary sphere (first n entries are the sources)
    s_xyz, s_q, _, _ = inset(c, q, L, plan.bc, plan.Rs)

    # 2. Phi_in and its field at the particles (own copy skipped)
    idx = np.arange(n) if sample is None else np.asarray(sample, dtype=np.int64)
    phi_in, e_in = coulomb(s_xyz, s_q, c[idx], tskip=idx, field=True, nthreads=nthreads)

    # 3. right-hand side of the least-squares problem (Sec. II.A)
    phi_x = coulomb(s_xyz, s_q, plan.x_mon, field=False, nthreads=nthreads)
    if plan.bc == PERIODIC:
        phi_xt = coulomb(s_xyz, s_q, plan.x_mon_partner, field=False, nthreads=nthreads)
        b = phi_xt - phi_x
    else:
        phi_xt = None
        b = -phi_x

    # 4. coefficients A_nm (A_00 = 0 for the periodic case)
    a, rdiag = lstsq(plan.M, b)
    A = np.concatenate([[0.0], a]) if plan.bc == PERIODIC else a

    # 5. surface images and 6. their potential and field at the particles
    img_xyz, img_q, phi_s, sigma = surface_images(plan, A)
    phi_out, e_out = coulomb(img_xyz, img_q, c[idx], field=True, nthreads=nthreads)

    # 7. energy and forces
    pot = phi_in + phi_out
    forces = q[idx, None] * (e_in + e_out)
    out = dict(pot=pot, forces=forces, phi_in=phi_in, phi_out=phi_out, e_in=e_in, e_out=e_out,
               A=A, b=b, phi_mon=phi_x, phi_mon_partner=phi_xt, n_inset=s_xyz.shape[0],
               n_images=img_xyz.shape[0], img_xyz=img_xyz, img_q=img_q, phi_surface=phi_s,
               sigma=sigma, lstsq_rdiag=rdiag, index=idx)
    out["energy"] = 0.5 * float(np.dot(q, pot)) if sample is None else None
    return out


def hsma(xyz, q, box, bc: int, P: int, Rs: float, Kmon: int, Q: int | None = None,
         F2: int | None = None, dr_rel: float | None = None, nthreads: int = 1, sample=None):
    """Convenience: plan + update in one call (Q -> F2 via fib_from_points)."""
    if F2 is None:
        F2, _ = fib_from_points(Q)
    plan = make_plan(box, bc, P, Rs, Kmon, F2, dr_rel)
    return energy_forces(xyz, q, plan, nthreads=nthreads, sample=sample), plan


def alpha_to_rs(box, alpha: float) -> float:
    """Rs = alpha R0 with R0 the circumradius of the box (Sec. II.A, Appendix)."""
    return alpha * 0.5 * float(np.linalg.norm(np.asarray(box, dtype=np.float64)))


def error_bound_potential(alpha, P, Rs, d0, qmax):
    """Truncation bound on the potential (Sec. II.A, the first error estimate)."""
    return 4 * math.pi * d0 * Rs**2 * qmax / ((alpha - 1) * (P - 2)) * alpha ** (-P)


def error_bound_gradient(alpha, P, Rs, d0, qmax):
    """Truncation bound on each gradient component (Sec. II.A and Appendix)."""
    return 4 * math.pi * d0 * Rs * qmax / ((alpha - 1) * (P - 2)) * (P + alpha / (alpha - 1)) * alpha ** (-(P - 1))


def series_far_field(plan: Plan, A, pts, h: float = 1e-4):
    """Phi_out = sum_k A_k B_k(r) evaluated directly at points (Eq.
    "harmonic"), and E_out = -grad Phi_out by fourth-order central
    differences with step h (relative to Rs).  The alternative to the
    surface images of Sec. II.B for bringing the fitted far field to the
    particles."""
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
    phi = basis(pts, plan.P, plan.Rs) @ A
    step = h * plan.Rs
    field = np.empty_like(pts)
    for a in range(3):
        e = np.zeros(3)
        e[a] = step
        f = lambda d: basis(pts + d * e, plan.P, plan.Rs) @ A  # noqa: E731
        deriv = (-f(2) + 8 * f(1) - 8 * f(-1) + f(-2)) / (12 * step)
        field[:, a] = -deriv
    return phi, field


def energy_forces_series(xyz, q, plan: Plan, nthreads: int = 1) -> dict:
    """The update step with the far field evaluated as the fitted series at
    each particle instead of through surface images (same in-set, fit and
    energy/force definitions as energy_forces)."""
    out = energy_forces(xyz, q, plan, nthreads=nthreads)
    c = centre_positions(xyz, plan.box, plan.bc)
    phi_s, e_s = series_far_field(plan, out["A"], c)
    q = np.asarray(q, dtype=np.float64)
    pot = out["phi_in"] + phi_s
    res = dict(out)
    res.update(pot=pot, phi_out=phi_s, e_out=e_s, forces=q[:, None] * (out["e_in"] + e_s),
               energy=0.5 * float(np.dot(q, pot)))
    return res
