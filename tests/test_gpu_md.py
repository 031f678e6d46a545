"""MD update loop over HSMA forces: a periodic ionic crystal with a
repulsive core, integrated with velocity Verlet; the plan (and its CUDA graph)
is reused every step.  The total energy must be conserved to the accuracy of
the integrator, which needs the HSMA forces to be minus the gradient of the
HSMA energy -- a check of the force/energy pair that no single-point test
makes."""
import numpy as np
import pytest

from paper_1806_04801_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _repulsion(L, sigma=0.08, eps=1.0):
    import torch

    def f(x):
        d = x[:, None, :] - x[None, :, :]
        d = d - L * torch.round(d / L)  # minimum image (box >> cutoff)
        r2 = (d * d).sum(-1)
        n = x.shape[0]
        r2 = r2 + torch.eye(n, dtype=x.dtype, device=x.device) * 1e6
        s6 = (sigma * sigma / r2) ** 3
        e = eps * s6 * s6  # r^-12 core
        u = 0.5 * e.sum()
        coef = (12.0 * e / r2)[..., None]
        return u, (coef * d).sum(1)
    return f


def test_velocity_verlet_conserves_energy():
    import torch
    from paper_1806_04801_gb300 import build, hsma, md
    assert torch.cuda.is_available()
    build.build()
    L = 1.0
    xyz, q = I.nacl_lattice(6, L)  # 216 ions, rock-salt arrangement
    g = np.random.default_rng(7)
    xyz = xyz + 0.01 * g.standard_normal(xyz.shape)
    v = 0.5 * g.standard_normal(xyz.shape)
    v -= v.mean(axis=0)
    dev = torch.device("cuda")
    x_t = torch.as_tensor(xyz, device=dev)
    q_t = torch.as_tensor(q, device=dev)
    v_t = torch.as_tensor(v, device=dev)
    with hsma.Plan((L, L, L), I.PERIODIC, 14, 1.5, 6000, 500, precision="fp64") as plan:
        sim = md.VelocityVerlet(plan, x_t, q_t, v_t, 1.0, dt=2e-5, box=(L, L, L), short_range=_repulsion(L))
        e0 = sim.u + sim.kinetic()
        launches0 = hsma.kernel_launches()
        traj = sim.step(200)
        per_step = (hsma.kernel_launches() - launches0) / 200
    tot = np.array([u + k for u, k in traj])
    kin = np.array([k for _, k in traj])
    drift = np.abs(tot - e0).max()
    assert drift <= 2e-4 * kin.mean(), (drift, kin.mean())
    assert per_step >= 10  # the whole update step runs on the device every step


def _configs(xyz, skin, seed):
    """Four configurations from xyz: the start, a small displacement, one in
    which particles near the x = 0 wall cross it (wrapped by the caller), and
    one in which a single particle has moved by more than the skin."""
    g = np.random.default_rng(seed)
    d1 = g.uniform(-0.3 * skin, 0.3 * skin, xyz.shape)
    c1 = np.mod(xyz + d1, 1.0)
    d2 = d1.copy()
    near = xyz[:, 0] < 0.2 * skin
    d2[near, 0] -= 0.4 * skin
    c2 = np.mod(xyz + d2, 1.0)
    c3 = c2.copy()
    c3[7] = np.mod(c3[7] + np.array([1.6 * skin, 0.0, 0.0]), 1.0)
    return [xyz, c1, c2, c3], int(near.sum())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_reused_inset_matches_a_fresh_one(prec):
    """In-set reuse (hsma_plan_set_inset_skin): steps that reuse the list --
    including one where particles crossed a periodic wall and were wrapped by
    the caller -- give the energy and forces of a plan that builds its in-set
    from scratch; a particle moved by more than the skin is detected and the
    step redone with a new list."""
    import torch
    from gpu_common import assert_within, errors
    from paper_1806_04801_gb300 import build, hsma
    build.build()
    w = I.SMALL_PERIODIC
    xyz, q = I.uniform_pm1(3000, w.box, seed_offset=430)
    skin = 0.05
    configs, crossing = _configs(xyz, skin, 431)
    assert crossing > 0
    dq = torch.as_tensor(q).cuda()
    tol = "fp64" if prec == "fp64" else "fp32"
    with hsma.Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec) as ref, \
            hsma.Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec) as pl:
        pl.set_inset_skin(skin)
        for k, x in enumerate(configs):
            dx = torch.as_tensor(x).cuda()
            U0, F0, _, ns0 = ref.energy_forces(dx, dq)
            U1, F1, _, ns1 = pl.energy_forces(dx, dq)
            assert_within(errors(F1.cpu().numpy(), F0.cpu().numpy(), U1, U0), tol, f"configuration {k}")
            assert ns1 >= ns0  # candidates outside the sphere ride along with charge 0
        assert pl.inset_stats() == {"builds": 2, "reuses": 2, "stale": 1}


def test_reused_inset_grounded_box():
    """The same for the grounded cavity (images are reflections, particles
    stay inside the box)."""
    import torch
    from gpu_common import assert_within, errors
    from paper_1806_04801_gb300 import build, hsma
    build.build()
    w = I.Workload("grounded-small", (1.0, 1.0, 2.0), I.GROUNDED, 8, I.GROUNDED_CAVITY.R, 2000, 600)
    xyz, q = I.uniform_pm1(2000, w.box, seed_offset=432, margin=0.05)
    g = np.random.default_rng(433)
    dq = torch.as_tensor(q).cuda()
    with hsma.Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp64") as ref, \
            hsma.Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp64") as pl:
        pl.set_inset_skin(0.04)
        for k in range(3):
            x = xyz + g.uniform(-0.01, 0.01, xyz.shape) * k
            dx = torch.as_tensor(x).cuda()
            U0, F0, _, _ = ref.energy_forces(dx, dq)
            U1, F1, _, _ = pl.energy_forces(dx, dq)
            assert_within(errors(F1.cpu().numpy(), F0.cpu().numpy(), U1, U0), "fp64", f"step {k}")
        assert pl.inset_stats() == {"builds": 1, "reuses": 2, "stale": 0}


def _oracle_verlet(xyz, q, v, dt, nsteps, w):
    """Velocity Verlet driven by the oracle's energy and forces (FP64 on the
    host), the same update as md.VelocityVerlet; returns positions and
    potential energies after each step."""
    from oracle import hsma as oh
    F2, _ = oh.fib_from_points(w.Q)
    plan = oh.make_plan(w.box, w.bc, w.p, w.R, w.Kmon, F2)
    x = xyz.copy()
    v = v.copy()
    r = oh.energy_forces(x, q, plan)
    f = r["forces"]
    out = []
    for _ in range(nsteps):
        a = f
        x = np.mod(x + dt * v + 0.5 * dt * dt * a, 1.0)
        r = oh.energy_forces(x, q, plan)
        v = v + 0.5 * dt * (a + r["forces"])
        f = r["forces"]
        out.append((x.copy(), r["energy"]))
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_md_trajectory_against_the_oracle(prec):
    """Five velocity-Verlet steps of 216 ions from one start state: the GPU
    loop (in-set reuse on, with a skin small enough that the list is rebuilt
    within the five steps) against the same integration driven by the
    oracle's forces.  Positions and energies agree at each step within the
    precision's tolerance."""
    import torch
    from paper_1806_04801_gb300 import build, hsma, md
    build.build()
    w = I.SMALL_PERIODIC
    xyz, q = I.nacl_lattice(6, 1.0)
    g = np.random.default_rng(434)
    xyz = np.mod(xyz + 0.02 * g.standard_normal(xyz.shape), 1.0)
    v = 2.0 * g.standard_normal(xyz.shape)
    v -= v.mean(axis=0)
    dt = 2e-4
    ref = _oracle_verlet(xyz, q, v, dt, 5, w)
    dev = torch.device("cuda")
    with hsma.Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec) as plan:
        sim = md.VelocityVerlet(plan, torch.as_tensor(xyz, device=dev), torch.as_tensor(q, device=dev),
                                torch.as_tensor(v, device=dev), 1.0, dt=dt, box=w.box, skin=0.002)
        traj = []
        for _ in range(5):
            (u, _), = sim.step(1)
            traj.append((sim.x.cpu().numpy(), u))
        stats = plan.inset_stats()
    assert stats["builds"] >= 2 and stats["reuses"] >= 1, stats
    tol_x, tol_u = (1e-11, 1e-10) if prec == "fp64" else (1e-8, 1e-6)
    for k, ((xg, ug), (xo, uo)) in enumerate(zip(traj, ref)):
        dxk = np.abs(xg - xo)
        dxk = np.minimum(dxk, 1.0 - dxk)  # a particle that wrapped on one side only
        assert dxk.max() <= tol_x, (k, dxk.max())
        assert abs(ug - uo) <= tol_u * abs(uo), (k, ug, uo)
