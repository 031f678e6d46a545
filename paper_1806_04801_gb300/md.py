"""Molecular-dynamics update loop over HSMA forces.

The paper's stated use of the method (Sec. III timing discussion and the
concluding remarks): the electrostatics of every MD step.  The loop keeps one
plan -- its fitting pseudo-inverse and integration matrices stay resident, and
the update step's CUDA graph is replayed each step -- and integrates with
velocity Verlet on device tensors.  Positions stay in the box frame (periodic
coordinates are wrapped after each drift).  A caller-supplied short-range
term (e.g. a repulsive core) is added to the electrostatic energy and forces.
With a skin, the plan reuses its in-set between steps (the sort and the image
generation run only when some particle has moved by the skin since the last
build; hsma_plan_set_inset_skin).
"""
from __future__ import annotations


class VelocityVerlet:
    """x(t+dt) = x + v dt + F dt^2 / 2m;  v(t+dt) = v + (F(t) + F(t+dt)) dt / 2m.

    plan:        hsma.Plan (its precision and boundary apply)
    xyz, q, v:   CUDA float64 tensors (n, 3), (n,), (n, 3)
    mass:        scalar or (n,) tensor
    short_range: optional callable xyz -> (energy, forces) on the same device
    skin:        if given, the plan's in-set reuse skin (0 switches it off)
    """

    def __init__(self, plan, xyz, q, v, mass, dt: float, box, periodic: bool = True, short_range=None,
                 skin=None):
        import torch
        self.torch = torch
        self.plan = plan
        if skin is not None:
            plan.set_inset_skin(skin)
        self.x = xyz.clone()
        self.q = q
        self.v = v.clone()
        self.m = mass if not hasattr(mass, "shape") else mass.reshape(-1, 1)
        self.dt = float(dt)
        self.L = torch.as_tensor(box, dtype=torch.float64, device=xyz.device)
        self.periodic = periodic
        self.short_range = short_range
        self.u, self.f = self._forces()

    def _forces(self):
        u, f, _, _ = self.plan.energy_forces(self.x, self.q)
        if self.short_range is not None:
            us, fs = self.short_range(self.x)
            u = u + float(us)
            f = f + fs
        return u, f

    def kinetic(self) -> float:
        """Kinetic energy sum m v^2 / 2 (FP64)."""
        return float(0.5 * (self.m * self.v * self.v).sum())

    def step(self, nsteps: int = 1):
        """Advance nsteps; returns [(potential, kinetic)] after each step."""
        out = []
        for _ in range(nsteps):
            a = self.f / self.m
            self.x += self.dt * self.v + 0.5 * self.dt * self.dt * a
            if self.periodic:
                self.x = self.torch.remainder(self.x, self.L)
            u_new, f_new = self._forces()
            self.v += 0.5 * self.dt * (a + f_new / self.m)
            self.u, self.f = u_new, f_new
            out.append((self.u, self.kinetic()))
        return out
