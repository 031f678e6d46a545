"""Batched and served update steps on the GPU.

* the CUDA-graph path gives bit-identical results to direct launches;
* a batch of uneven systems (the 256-box workload, full size) agrees with
  the FP64 path system by system, and sampled systems agree with the oracle;
* the serving loop returns, for a request submitted alone and the same
  request submitted in a mix with concurrent traffic, the same result within
  the reduced-precision tolerance; oversize requests fail cleanly.
"""
import threading

import numpy as np
import pytest

from gpu_common import TOL, energy_floor, errors, rel_energy_err, rms, to_dev
from paper_1806_04801_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available()
    from paper_1806_04801_gb300 import build
    build.build()


def hs():
    from paper_1806_04801_gb300 import hsma
    return hsma


def test_graph_and_direct_launches_agree():
    w = I.SMALL_PERIODIC
    xyz, q = I.small_periodic()
    dx, dq = to_dev(xyz, q)
    res = {}
    for graphs in (False, True):
        with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32", use_graphs=graphs) as plan:
            out = [plan.energy_forces(dx, dq) for _ in range(3)]
            res[graphs] = out
            for U, F, _, _ in out[1:]:
                assert U == out[0][0] and bool((F == out[0][1]).all())
            # a different shape re-captures, then the first shape still replays correctly
            x2, q2 = I.uniform_pm1(700, w.box, seed_offset=61)
            plan.energy_forces(*to_dev(x2, q2))
            U3, F3, _, _ = plan.energy_forces(dx, dq)
            assert U3 == out[0][0] and bool((F3 == out[0][1]).all())
    assert res[True][0][0] == res[False][0][0]
    assert bool((res[True][0][1] == res[False][0][1]).all())


@pytest.fixture(scope="module")
def batch256():
    systems = I.batch_periodic()
    xyz = np.concatenate([s[0] for s in systems])
    q = np.concatenate([s[1] for s in systems])
    off = np.concatenate([[0], np.cumsum([len(s[1]) for s in systems])])
    return systems, xyz, q, off


@pytest.mark.slow
def test_batched_256_boxes_full_size(batch256):
    systems, xyz, q, off = batch256
    w = I.BATCH_PERIODIC
    dx, dq = to_dev(xyz, q)
    out = {}
    for prec in ("fp32", "fp64"):
        with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec) as plan:
            E, F, _, st = plan.energy_forces_batched(dx, dq, off)
            assert np.all(st == 0)
            out[prec] = (E, F.cpu().numpy())
    E32, F32 = out["fp32"]
    E64, F64 = out["fp64"]
    # relative energy error; the denominator is floored at the self-image
    # energy scale, because some random +-1 draws have energies that cancel to
    # far below their natural size (e.g. U = -12 for 2542 charges)
    rel = np.array([rel_energy_err(E32[i], E64[i], systems[i][1]) for i in range(len(systems))])
    assert rel.max() <= 1e-6, (rel.max(), int(rel.argmax()))
    # and systems of ordinary energy meet the plain relative bound
    plain = np.array([abs(E64[i]) >= energy_floor(systems[i][1]) for i in range(len(systems))])
    assert plain.sum() >= 64
    assert (np.abs(E32 - E64) / np.abs(E64))[plain].max() <= 1e-6
    for i in range(len(systems)):
        sl = slice(off[i], off[i + 1])
        assert rms(F32[sl] - F64[sl]) <= 1e-5 * rms(F64[sl]), i
    # sampled systems against the oracle (smallest, largest)
    from oracle import hsma as oh
    F2, _ = oh.fib_from_points(w.Q)
    oplan = oh.make_plan(w.box, w.bc, w.p, w.R, w.Kmon, F2)
    sizes = np.diff(off)
    for i in (int(sizes.argmin()), int(sizes.argmax())):
        sx, sq = systems[i]
        sample = None if len(sq) < 3000 else np.linspace(0, len(sq) - 1, 40).astype(np.int64)
        ref = oh.energy_forces(sx, sq, oplan, nthreads=16, sample=sample)
        sl = slice(off[i], off[i + 1])
        idx = ref["index"]
        e = errors(F32[sl][idx], ref["forces"])
        assert e["force_rms"] <= TOL["fp32"]["force_rms"], (i, e)
        if sample is None:
            assert rel_energy_err(E32[i], ref["energy"], sq) <= 1e-6


def _mixed_traffic(server, systems, first, results):
    for j, (sx, sq) in enumerate(systems):
        t = server.submit(sx, sq)
        results.append((first + j, t))


@pytest.mark.parametrize("prec", ["fp32", "fp32_tc"])
def test_serving_alone_and_in_mix_agree(prec):
    """A request served alone and inside concurrent traffic (continuous
    batching over two lanes) agrees within the reduced-form tolerance; so
    does every mixed request with a direct call.  With the tensor-core fit the
    product spans whatever systems share the batch."""
    w = I.SERVING_PERIODIC
    target_x, target_q = I.uniform_pm1(12000, w.box, seed_offset=70)
    others = [I.uniform_pm1(int(n), w.box, seed_offset=71 + i) for i, n in
              enumerate([1000, 30000, 5000, 2000, 60000, 800, 15000, 4000, 9000, 3000])]
    with hs().Server(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec, lanes=2, max_batch=8) as srv:
        t = srv.submit(target_x, target_q)
        code, E_alone, F_alone, info = srv.result(t, n=len(target_q))
        assert code == 0 and info["batch_size"] == 1
        # the same request inside concurrent traffic
        tickets = []
        th = threading.Thread(target=_mixed_traffic, args=(srv, others[:5], 0, tickets))
        th.start()
        t2 = srv.submit(target_x, target_q)
        _mixed_traffic(srv, others[5:], 5, tickets)
        th.join()
        code, E_mix, F_mix, info2 = srv.result(t2, n=len(target_q))
        assert code == 0
        assert rel_energy_err(E_mix, E_alone, target_q) <= TOL["fp32"]["energy"]
        assert rms(F_mix - F_alone) <= TOL["fp32"]["force_rms"] * rms(F_alone)
        # every mixed request agrees with a direct single-system call
        with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec) as plan:
            for j, tk in tickets:
                sx, sq = others[j]
                code, E, F, inf = srv.result(tk, n=len(sq))
                assert code == 0
                U1, F1, _, _ = plan.energy_forces(sx, sq)
                assert rel_energy_err(E, U1, sq) <= TOL["fp32"]["energy"]
                assert rms(F - F1) <= TOL["fp32"]["force_rms"] * rms(F1)
        st = srv.stats()
        assert st["completed"] == 12 and st["failed"] == 0


def test_serving_rejects_requests_beyond_budget():
    w = I.SERVING_PERIODIC
    with hs().Server(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, lanes=1, hbm_budget_bytes=64 << 20) as srv:
        big = I.uniform_pm1(200000, w.box, seed_offset=80)
        small = I.uniform_pm1(1000, w.box, seed_offset=81)
        tb = srv.submit(*big)
        ts = srv.submit(*small)
        code_b, _, _, _ = srv.result(tb, n=len(big[1]))
        code_s, E, _, _ = srv.result(ts, n=len(small[1]))
        assert code_b == -11
        assert code_s == 0 and np.isfinite(E)
        # a ticket is collected once
        assert srv.result(ts, n=1)[0] == -9


def test_autotuner_and_both_kernel_variants(tmp_path):
    """Both work decompositions of the pair kernel give the same physics (to
    FP32 rounding); the autotuner picks one, records it, and a new plan loads
    it back from the cache."""
    w = I.BATCH_PERIODIC
    systems = [I.uniform_pm1(int(n), w.box, seed_offset=90 + i) for i, n in enumerate([600, 3000, 9000, 1200])]
    xyz = np.concatenate([s[0] for s in systems])
    q = np.concatenate([s[1] for s in systems])
    off = np.concatenate([[0], np.cumsum([len(s[1]) for s in systems])])
    dx, dq = to_dev(xyz, q)
    res = {}
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32") as plan:
        for var in (4, 5, 2, 12, 13, 14, 15, 16, 17):
            for ips in (8, 48):
                plan.set_tuning(var, ips)
                E, F, _, st = plan.energy_forces_batched(dx, dq, off)
                assert np.all(st == 0)
                res[(var, ips)] = (E, F.cpu().numpy())
        E0, F0 = res[(4, 8)]
        for k, (E, F) in res.items():
            for i in range(len(systems)):
                sl = slice(off[i], off[i + 1])
                assert rel_energy_err(E[i], E0[i], systems[i][1]) <= 1e-6, k
                assert rms(F[sl] - F0[sl]) <= 1e-5 * rms(F0[sl]), k
        plan.set_tuning(None, None)
        cache = str(tmp_path / "tune.jsonl")
        best = plan.autotune(dx, dq, off, cache_path=cache)
        assert best["pair_variant"] in (14, 17, 12, 13, 2) and best["items_per_slot"] in (8, 16, 24, 48) and best["ms"] > 0
        assert plan.get_tuning(off)["pair_variant"] == best["pair_variant"]
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32") as plan2:
        assert (plan2.get_tuning(off)["pair_variant"], plan2.get_tuning(off)["items_per_slot"]) == (17, 48)  # defaults
        assert plan2.load_tuning(cache) == 1
        t2 = plan2.get_tuning(off)
        assert (t2["pair_variant"], t2["items_per_slot"]) == (best["pair_variant"], best["items_per_slot"])
        E, F, _, _ = plan2.energy_forces_batched(dx, dq, off)
        for i in range(len(systems)):
            assert rel_energy_err(E[i], E0[i], systems[i][1]) <= 1e-6


def test_serving_cancellation():
    """Requests withdrawn while queued report the cancellation code and never
    run; the rest of the stream is served normally."""
    w = I.SERVING_PERIODIC
    reqs = [I.uniform_pm1(int(n), w.box, seed_offset=120 + i) for i, n in enumerate([60000] * 2 + [2000] * 10)]
    with hs().Server(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, lanes=1, max_batch=1) as srv:
        tickets = [srv.submit(*r) for r in reqs]
        # the tail is still queued behind the two large requests: withdraw every other one
        withdrawn = [t for i, t in enumerate(tickets) if i >= 4 and i % 2 == 0]
        codes = {t: srv.cancel(t) for t in withdrawn}
        for t, (x, q) in zip(tickets, reqs):
            code, E, F, info = srv.result(t, n=len(q))
            if t in withdrawn and codes[t] == 0:
                assert code == -12
            else:
                assert code == 0 and np.isfinite(E)
        st = srv.stats()
        assert st["cancelled"] == sum(1 for c in codes.values() if c == 0) >= 1
        assert st["completed"] + st["cancelled"] == len(reqs)


def test_preemptible_pair_work_gives_the_same_results():
    """One CTA per work item (the serving bulk lanes' mode) against the
    persistent grid.  These systems are small enough that both modes take the
    smallest chunk (four tiles), so the items and the fixed-order reduction
    are the same and the FP32 pair sums with the FP64 fit are bit-identical."""
    w = I.BATCH_PERIODIC
    systems = [I.uniform_pm1(int(n), w.box, seed_offset=140 + i) for i, n in enumerate([900, 5000, 20000])]
    xyz = np.concatenate([s[0] for s in systems])
    q = np.concatenate([s[1] for s in systems])
    off = np.concatenate([[0], np.cumsum([len(s[1]) for s in systems])])
    dx, dq = to_dev(xyz, q)
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32") as plan:
        E0, F0, _, _ = plan.energy_forces_batched(dx, dq, off)
        plan.set_preemptible(True)
        E1, F1, _, _ = plan.energy_forces_batched(dx, dq, off)
        assert np.array_equal(E0, E1) and bool((F0 == F1).all())
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32_tc") as plan:
        E0, F0, _, _ = plan.energy_forces_batched(dx, dq, off)
        plan.set_preemptible(True)  # the tensor-core fit on a quarter of the SMs: other sum grouping
        E1, F1, _, _ = plan.energy_forces_batched(dx, dq, off)
        for i in range(len(systems)):
            assert rel_energy_err(E1[i], E0[i], systems[i][1]) <= 1e-7


def test_preemptible_pair_work_on_finer_items():
    """At 1e5 charges the preemptible mode cuts its items 8x finer than the
    persistent grid's, so the same pair sums are grouped differently: equal
    up to summation order (measured: energy identical, forces within 2e-11 of
    the RMS force)."""
    w = I.LARGE_PERIODIC
    xyz, q = I.large_periodic(100_000)
    dx, dq = to_dev(xyz, q)
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32") as plan:
        plan.set_tuning(17, 48)
        U0, F0, _, _ = plan.energy_forces(dx, dq)
        plan.set_preemptible(True)
        U1, F1, _, _ = plan.energy_forces(dx, dq)
    F0, F1 = F0.cpu().numpy(), F1.cpu().numpy()
    assert abs(U1 - U0) <= 1e-12 * abs(U0)
    assert np.abs(F1 - F0).max() <= 1e-9 * np.sqrt(np.mean(F0 ** 2))


def test_medium_and_small_requests_overtake_a_large_batch():
    """Three classes: express (small, highest priority), medium lanes (middle
    priority, preemptible) and bulk (lowest, preemptible).  A medium request
    submitted while a large one runs finishes long before it; a small one
    submitted while both run finishes before the medium one; all three agree
    with direct calls."""
    import time
    w = I.SERVING_PERIODIC
    big = I.uniform_pm1(200000, w.box, seed_offset=152)
    medium = I.uniform_pm1(40000, w.box, seed_offset=153)
    small = I.uniform_pm1(2000, w.box, seed_offset=154)
    with hs().Server(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32", lanes=3, max_batch=4,
                     express_lanes=1, express_max_n=20000, mid_lanes=1, mid_max_n=60000) as srv:
        tb = srv.submit(*big)
        time.sleep(0.03)  # the large request is on the GPU
        tm = srv.submit(*medium)
        time.sleep(0.002)
        ts = srv.submit(*small)
        code_s, E_s, F_s, info_s = srv.result(ts)
        code_m, E_m, F_m, info_m = srv.result(tm)
        code_b, E_b, F_b, info_b = srv.result(tb)
    assert code_s == 0 and code_m == 0 and code_b == 0
    print(f"\nlarge {info_b['latency_ms']:.1f} ms, medium {info_m['latency_ms']:.1f} ms, "
          f"small {info_s['latency_ms']:.1f} ms")
    assert info_m["latency_ms"] < 0.5 * (info_b["latency_ms"] - 30.0), (info_m, info_b)
    assert info_s["latency_ms"] < info_m["latency_ms"], (info_s, info_m)
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32") as plan:
        for (sx, sq), E, F in ((small, E_s, F_s), (medium, E_m, F_m), (big, E_b, F_b)):
            U1, F1, _, _ = plan.energy_forces(sx, sq)
            assert rel_energy_err(E, U1, sq) <= TOL["fp32"]["energy"]
            assert rms(F - F1) <= TOL["fp32"]["force_rms"] * rms(F1)


def test_small_request_overtakes_a_large_batch():
    """Express lane (high-priority stream) and bulk lane (preemptible pair
    work): a small request submitted while a large one runs finishes long
    before it, and both agree with direct calls."""
    import time
    w = I.SERVING_PERIODIC
    big = I.uniform_pm1(200000, w.box, seed_offset=150)
    small = I.uniform_pm1(2000, w.box, seed_offset=151)
    with hs().Server(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32", lanes=2, max_batch=4,
                     express_lanes=1, express_max_n=20000) as srv:
        tb = srv.submit(*big)
        time.sleep(0.03)  # the large request is on the GPU
        ts = srv.submit(*small)
        code_s, E_s, F_s, info_s = srv.result(ts)
        code_b, E_b, F_b, info_b = srv.result(tb)
    assert code_s == 0 and code_b == 0
    print(f"\nlarge request {info_b['latency_ms']:.1f} ms, small request behind it {info_s['latency_ms']:.1f} ms")
    assert info_s["latency_ms"] < 0.5 * (info_b["latency_ms"] - 30.0), (info_s, info_b)
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32") as plan:
        for (sx, sq), E, F in ((small, E_s, F_s), (big, E_b, F_b)):
            U1, F1, _, _ = plan.energy_forces(sx, sq)
            assert rel_energy_err(E, U1, sq) <= TOL["fp32"]["energy"]
            assert rms(F - F1) <= TOL["fp32"]["force_rms"] * rms(F1)
