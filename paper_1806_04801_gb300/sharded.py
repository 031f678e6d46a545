"""Target sharding of one system over several GPUs (host logic).

One process per GPU.  Every rank holds all particles and a plan with the same
parameters.  The update step (Sec. II.C) then needs only two small exchanges:

  1. near-field sums for the rank's own targets (a slice of the particles
     and of the monitoring points);
  2. sum of the monitoring potentials over the ranks (n_mon_targets doubles);
  3. fit, surface images and far field at the rank's own particles (the fit
     is repeated on every rank: it is tiny), then -- on the device -- the
     owned particles' potentials, forces and the part's energy;
  4. sum of the parts' energies over the ranks (one double).  Forces stay
     with the rank that owns the particle (gather them if the caller wants
     them in one place).

This module does none of the method's arithmetic: it moves arrays between
the stages and calls the all-reduce.  The compute backend is any object with
``near(xyz, q, part, nparts)`` -> (index, phi_in, E_in, phi_mon) and
``far(xyz, q, phi_mon, phi_in, E_in, part, nparts)`` -> (index, potentials,
forces, energy of the part); ``GpuBackend`` wraps a plan of the CUDA library
(hsma_shard_near / hsma_shard_far).  The communicator needs
``allreduce_sum(numpy array) -> numpy array``; ``TorchComm`` uses
torch.distributed (NCCL or gloo).
"""
from __future__ import annotations

import numpy as np


class GpuBackend:
    """The CUDA library's split update step (hsma_shard_near / hsma_shard_far)."""

    def __init__(self, plan):
        self.plan = plan

    def near(self, xyz, q, part, nparts):
        """Stage 1 on this rank's slice (hsma_shard_near): owned indices, Phi_in, E_in and the monitoring potentials."""
        return self.plan.shard_near(xyz, q, part, nparts)

    def far(self, xyz, q, phi_mon, phi_in, e_in, part, nparts):
        """Stage 3 on this rank's slice (hsma_shard_far): potentials, forces and the part's energy, from the
        summed monitoring potentials and this part's near-stage results."""
        return self.plan.shard_far(xyz, q, phi_mon, phi_in, e_in, part, nparts)


class TorchComm:
    """Sum-reductions over a torch.distributed process group."""

    def __init__(self, group=None, device=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.device = device

    @property
    def rank(self):
        """This process's rank in the process group."""
        return self.dist.get_rank(self.group)

    @property
    def size(self):
        """Number of ranks."""
        return self.dist.get_world_size(self.group)

    def allreduce_sum(self, a):
        """Element-wise sum of a numpy array over the ranks."""
        import torch
        t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64))
        if self.device is not None:
            t = t.to(self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t.cpu().numpy()


def shard_update(backend, xyz, q, comm, part=None, nparts=None):
    """The target-sharded update step on this rank.  Returns (U, index,
    forces of the owned particles, potentials of the owned particles)."""
    part = comm.rank if part is None else part
    nparts = comm.size if nparts is None else nparts
    idx, phi_in, e_in, phi_mon = backend.near(xyz, q, part, nparts)
    phi_mon = comm.allreduce_sum(phi_mon)
    idx2, pot, forces, u_part = backend.far(xyz, q, phi_mon, phi_in, e_in, part, nparts)
    if not np.array_equal(idx, idx2):
        raise RuntimeError("near and far stages disagree on the owned particles")
    u = comm.allreduce_sum(np.array([u_part]))[0]
    return float(u), idx, forces, pot


def shard_update_local(backend, xyz, q, nparts):
    """All parts of the sharded step in one process (stage by stage), for a
    single device or for tests: the two all-reduces become sums over the
    parts' arrays."""
    near = [backend.near(xyz, q, p, nparts) for p in range(nparts)]
    phi_mon = np.sum([r[3] for r in near], axis=0)
    n = len(q)
    forces = np.zeros((n, 3))
    pot = np.zeros(n)
    u_parts = []
    seen = np.zeros(n, dtype=np.int64)
    for p in range(nparts):
        idx, phi_in, e_in, _ = near[p]
        idx2, pot_p, f_p, u_p = backend.far(xyz, q, phi_mon, phi_in, e_in, p, nparts)
        if not np.array_equal(idx, idx2):
            raise RuntimeError("near and far stages disagree on the owned particles")
        pot[idx] = pot_p
        forces[idx] = f_p
        u_parts.append(u_p)
        seen[idx] += 1
    if not np.all(seen == 1):
        raise RuntimeError("the parts do not cover every particle exactly once")
    return float(np.sum(u_parts)), forces, pot
