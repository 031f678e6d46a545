"""Target sharding of one system over ranks (host logic), on CPU ranks.

Two gloo processes run paper_1806_04801_gb300.sharded.shard_update with a
compute backend built from the FP64 oracle (the test stands it in for the
CUDA library, which needs a GPU); their exchanges are real torch.distributed
all-reduces.  The sharded energy and forces must equal the unsharded oracle's, and a rank
that fails before the exchange must end the others' step with an error.
"""
import os
import socket
import tempfile

import numpy as np

from paper_1806_04801_gb300 import inputs as I


class OracleBackend:
    """near/far stages of the update step computed by the oracle, owning the
    particle slice [p n / P, (p + 1) n / P) and the same slice of the
    monitoring targets (order: x_i, then their partners)."""

    def __init__(self, w):
        from oracle import hsma as oh
        self.oh = oh
        self.w = w
        F2, _ = oh.fib_from_points(w.Q)
        self.plan = oh.make_plan(w.box, w.bc, w.p, w.R, w.Kmon, F2)
        mon = [self.plan.x_mon] + ([self.plan.x_mon_partner] if self.plan.bc == oh.PERIODIC else [])
        self.mon = np.concatenate(mon)

    def _inset(self, xyz, q):
        import oracle
        c = self.oh.centre_positions(xyz, self.plan.box, self.plan.bc)
        s_xyz, s_q, _, _ = oracle.inset(c, q, self.plan.box, self.plan.bc, self.plan.Rs)
        return c, s_xyz, s_q

    def near(self, xyz, q, part, nparts):
        import oracle
        n = len(q)
        c, s_xyz, s_q = self._inset(xyz, q)
        idx = np.arange(part * n // nparts, (part + 1) * n // nparts)
        phi, fld = oracle.coulomb(s_xyz, s_q, c[idx], tskip=idx, field=True)
        nm = len(self.mon)
        mlo, mhi = part * nm // nparts, (part + 1) * nm // nparts
        phi_mon = np.zeros(nm)
        phi_mon[mlo:mhi] = oracle.coulomb(s_xyz, s_q, self.mon[mlo:mhi], field=False)
        return idx, phi, fld, phi_mon

    def far(self, xyz, q, phi_mon, phi_in, e_in, part, nparts):
        import oracle
        oh = self.oh
        n = len(q)
        c, _, _ = self._inset(xyz, q)
        K = self.plan.Kmon
        b = phi_mon[K:] - phi_mon[:K] if self.plan.bc == oh.PERIODIC else -phi_mon
        a, _ = oracle.lstsq(self.plan.M, b)
        A = np.concatenate([[0.0], a]) if self.plan.bc == oh.PERIODIC else a
        img_xyz, img_q, _, _ = oh.surface_images(self.plan, A)
        idx = np.arange(part * n // nparts, (part + 1) * n // nparts)
        phi, fld = oracle.coulomb(img_xyz, img_q, c[idx], field=True)
        qi = np.asarray(q, dtype=np.float64)[idx]
        pot = phi_in + phi
        return idx, pot, qi[:, None] * (e_in + fld), 0.5 * float(np.dot(qi, pot))


WORKLOAD = I.Workload("sharded-test", (1.0, 1.0, 1.0), I.PERIODIC, 6, 1.5, 600, 200)


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    from paper_1806_04801_gb300 import sharded
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        xyz, q = I.uniform_pm1(300, WORKLOAD.box, seed_offset=400)
        U, idx, F, pot = sharded.shard_update(OracleBackend(WORKLOAD), xyz, q, sharded.TorchComm())
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), U=U, idx=idx, F=F, pot=pot)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reproduce_the_unsharded_step():
    import torch.multiprocessing as mp
    from oracle import hsma as oh
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_worker, args=(world, _free_port(), d), nprocs=world, join=True)
        parts = [np.load(os.path.join(d, f"r{r}.npz")) for r in range(world)]
    xyz, q = I.uniform_pm1(300, WORKLOAD.box, seed_offset=400)
    F2, _ = oh.fib_from_points(WORKLOAD.Q)
    ref = oh.energy_forces(xyz, q, oh.make_plan(WORKLOAD.box, WORKLOAD.bc, WORKLOAD.p, WORKLOAD.R, WORKLOAD.Kmon, F2))
    # every rank holds the same all-reduced energy
    for p in parts:
        assert abs(float(p["U"]) - ref["energy"]) <= 1e-12 * abs(ref["energy"])
    F = np.zeros_like(ref["forces"])
    seen = np.zeros(len(q), dtype=int)
    for p in parts:
        F[p["idx"]] = p["F"]
        seen[p["idx"]] += 1
    assert np.all(seen == 1)
    np.testing.assert_allclose(F, ref["forces"], rtol=0, atol=1e-12 * np.abs(ref["forces"]).max())


def test_local_driver_with_oracle_backend_any_part_count():
    from oracle import hsma as oh
    from paper_1806_04801_gb300 import sharded
    xyz, q = I.uniform_pm1(200, WORKLOAD.box, seed_offset=401)
    F2, _ = oh.fib_from_points(WORKLOAD.Q)
    ref = oh.energy_forces(xyz, q, oh.make_plan(WORKLOAD.box, WORKLOAD.bc, WORKLOAD.p, WORKLOAD.R, WORKLOAD.Kmon, F2))
    for nparts in (1, 3, 7):
        U, F, pot = sharded.shard_update_local(OracleBackend(WORKLOAD), xyz, q, nparts)
        assert abs(U - ref["energy"]) <= 1e-12 * abs(ref["energy"])
        np.testing.assert_allclose(F, ref["forces"], rtol=0, atol=1e-12 * np.abs(ref["forces"]).max())


class _DyingBackend:
    """Stands in for a rank whose near-field stage fails (a host-side
    fault: the exception a failed device call would raise)."""

    def near(self, xyz, q, part, nparts):
        raise RuntimeError("injected failure in the near-field stage")

    def far(self, xyz, q, phi_mon, phi_in, e_in, part, nparts):
        raise AssertionError("not reached")


def _worker_one_rank_fails(rank, world, port, out_dir):
    import time
    from datetime import timedelta
    import torch.distributed as dist
    from paper_1806_04801_gb300 import sharded
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                            timeout=timedelta(seconds=10))
    xyz, q = I.uniform_pm1(200, WORKLOAD.box, seed_offset=404)
    backend = OracleBackend(WORKLOAD) if rank == 0 else _DyingBackend()
    t0 = time.time()
    try:
        sharded.shard_update(backend, xyz, q, sharded.TorchComm())
        outcome = "completed"
    except Exception as e:  # recorded for the parent, which checks it
        outcome = f"{type(e).__name__}: {e}".replace("\n", " ")[:300]
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{time.time() - t0:.3f}\n{outcome}\n")


def test_a_failing_rank_ends_the_sharded_step_with_an_error_on_the_others():
    """Rank 1 fails before the exchange of the monitoring potentials and
    leaves; rank 0's all-reduce then ends with an error (the peer's closed
    connection, at the latest the process group's 10 s timeout) instead of
    waiting for ever.  Host-side failure only: no device is involved."""
    import multiprocessing as mpl
    ctx = mpl.get_context("spawn")
    with tempfile.TemporaryDirectory() as d:
        port = _free_port()
        procs = [ctx.Process(target=_worker_one_rank_fails, args=(r, 2, port, d)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        alive = [p for p in procs if p.is_alive()]
        for p in alive:  # only the processes this test started
            p.terminate()
            p.join(timeout=10)
        assert not alive, "a rank was still running after 120 s"
        res = {}
        for r in range(2):
            with open(os.path.join(d, f"r{r}.txt")) as f:
                t, outcome = f.read().splitlines()[:2]
            res[r] = (float(t), outcome)
    assert "injected failure" in res[1][1]
    assert res[0][1] != "completed", res[0]
    assert res[0][0] < 60.0, res[0]
