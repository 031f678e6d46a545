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
