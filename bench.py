"""Benchmark of the HSMA hot path on GB300.

A step is one full update step (in-set, near-field sums at particles and
monitoring points, fit, surface images and their sums, energy and forces) of
one periodic system of 100000 charges (p = 12, 2000 monitoring points,
Q = 8000 -> F2 = 1597, Rs = 1.5 L), FP32 pair sums with double-float
accumulation, FP64 fit and energy.  Inputs are resident in HBM when the timed
region starts; L2 is flushed (a 256 MB write) between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own system (weak scaling; no collective on
the data path).  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("systems/sec and pair-interactions/s vs FP32 roofline at rel. energy err ≤1e-6; p50/p99")
FP32_LANES_PER_SM = 128          # FP32 lanes per SM (GB300)
OPS_POT_FIELD = 13               # FP32 lane instructions per potential+field pair (minimal form)
OPS_POT = 7                      # FP32 lane instructions per potential-only pair
RECIPE_SMS = 152
RECIPE_MAX_SM_MHZ = 2070.0
# DRAM bytes (read + write) of one full-size pair_fp32_kernel launch of the
# periodic N=100000 workload, from the ncu capture summarised in
# profiles/pair_fp32_kernel_periodic_N100000_dram.md (current kernel build),
# keyed by (N, pair variant, items per slot) of the captured launch.
PAIR_FP32_TRAFFIC_BYTES = {(100_000, 17, 48): 361.16e6, (100_000, 14, 48): 356.89e6,
                           (100_000, 17, 96): 726.99e6, (100_000, 14, 96): 710.68e6}
OPS_SURFACE = 45                 # FP32 lane instructions per particle-direction pair of the surface kernel


def parse():
    """Command-line options (the contract's --gpus/--steps/--warmup, --impl, workloads and tuning)."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32_tc", choices=["fp32", "fp64", "fp32_tc"],
                    help="fp32_tc (default): FP32 pair sums with double-float accumulation, split-BF16 "
                         "tensor-core fit + one refinement; fp32: the same with an FP64 fit; fp64: parity form")
    ap.add_argument("--n", "--particles", dest="n", type=int, default=100_000,
                    help="particles of the periodic workload (--particles under torchrun, where --n is ambiguous)")
    ap.add_argument("--no-check", action="store_true", help="skip the FP64 accuracy check")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and serving summaries")
    ap.add_argument("--workload", default="periodic",
                    choices=["periodic", "batched", "serving", "grounded", "basis", "paper", "md"])
    ap.add_argument("--basis-points", type=int, default=4_000_000, help="points of the basis workload")
    ap.add_argument("--requests", type=int, default=200, help="serving: requests in the Poisson trace")
    ap.add_argument("--tuning", default=None,
                    help="V,I: fix the pair kernel variant and items per slot instead of autotuning "
                         "(profiling runs use this so the captured launch is the timed configuration)")
    return ap.parse_args()


# ------------------------------------------------------- batched workload
def measured_hbm_gbs():
    """HBM copy bandwidth measured on this machine (generated file), else
    the recorded fallback."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def run_basis(steps: int, warmup: int, n: int = 4_000_000, p: int = 12, Rs: float = 1.5):
    """The harmonic basis of Eq. "harmonic" (orthonormal real solid harmonics,
    N_b = (p + 1)^2 FP64 values per point) at n points spread over the
    auxiliary sphere's ball: the per-point evaluation behind the plan's
    matrices and the direct series evaluation, timed through hsma_basis in
    both forms -- the double-float recurrence on the FP32 pipe (the headline)
    and the FP64 recurrence."""
    import torch
    from paper_1806_04801_gb300 import hsma
    g = torch.Generator(device="cuda").manual_seed(1806_04801 + 5)
    pts = (torch.rand(n, 3, dtype=torch.float64, device="cuda", generator=g) - 0.5) * (2.0 * Rs / math.sqrt(3.0))

    def timed(precision, k):
        for _ in range(warmup):
            out = hsma.basis(pts, p, Rs, precision=precision)
            del out
        torch.cuda.synchronize()
        times = []
        for _ in range(k):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = hsma.basis(pts, p, Rs, precision=precision)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            del out
        return float(np.median(times))

    ms = timed("fp32", steps)
    ms64 = timed("fp64", max(1, min(steps, 5)))
    nb = (p + 1) * (p + 1)
    written = n * nb * 8.0
    hbm, how = measured_hbm_gbs()
    # FP64 operations of the FP64 form per point (fully normalised
    # recurrence): per (n, m) with n >= m + 2 four (a_nm z, b_nm r2, a product
    # and a fused multiply-add), one per stored value (Pbar C_m or S_m), one
    # per order for E_m z, six per power of (x + i y), three for r2
    pairs = sum(max(0, p - m - 1) for m in range(p + 1))
    fp64_ops = 4 * pairs + nb + (p + 1) + 6 * p + 3
    gbs = written / (ms / 1000.0) / 1e9
    return {"workload": f"basis-N{n}-p{p} (points uniform in a cube inside the Rs = {Rs} ball)",
            "points": n, "p": p, "N_b": nb, "ms": ms, "points_per_s": n / (ms / 1000.0),
            "arithmetic": "double-float (FP32 pairs), FP64 output",
            "fp64_recurrence": {"ms": ms64, "points_per_s": n / (ms64 / 1000.0),
                                "achieved_gbs": written / (ms64 / 1000.0) / 1e9,
                                "hbm_frac": written / (ms64 / 1000.0) / 1e9 / hbm,
                                "fp64_ops_per_point": fp64_ops,
                                "achieved_fp64_tops": n * fp64_ops / (ms64 / 1000.0) / 1e12},
            "speedup_vs_fp64_recurrence": ms64 / ms,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "traffic": None, "peak_source": f"HBM copy bandwidth, {how}",
                         "algorithmic_bytes": "8 N_b bytes written per point (the 24-byte point read is ~2%)",
                         "note": "timed through hsma_basis (launch + stream synchronisation included)"}}


def run_paper_config(steps: int, warmup: int, precision: str, n_side: int = 47):
    """The configuration of the paper's timing study (Sec. III): unit charges
    of random sign on a uniform lattice (47^3 = 103823 sites, about the
    paper's N = 100k), periodic, alpha = 1.3, P = 25, N_o = 5928 (F2 = 987);
    the paper reports under 1 s per HSMA step there on two Tesla P100 or two
    K80 GPUs (precision not stated)."""
    import torch
    from paper_1806_04801_gb300 import hsma
    from paper_1806_04801_gb300 import inputs as I
    L = (1.0, 1.0, 1.0)
    alpha, P = 1.3, 25
    Rs = alpha * 0.5 * math.sqrt(3.0)
    xyz, q = I.lattice_random_sign(n_side, 1.0, seed_offset=500 + n_side)
    dx, dq = torch.as_tensor(xyz).cuda(), torch.as_tensor(q).cuda()
    with hsma.Plan(L, I.PERIODIC, P, Rs, 5928, 2 * P * P, precision=precision, fib_F2=987, profile=True) as plan:
        plan.autotune(dx, dq)
        for _ in range(warmup):
            plan.energy_forces(dx, dq)
        torch.cuda.synchronize()
        times = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            U, _, _, ns = plan.energy_forces(dx, dq)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        info = plan.info()
    ms = float(np.median(times))
    return {"workload": f"paper timing configuration: lattice {n_side}^3 random +-1, periodic, alpha 1.3 "
                        f"(Rs = {Rs:.4f} L), P = 25, N_o = {info['n_images']}, Kmon = {2 * P * P}",
            "N": int(len(q)), "n_inset": int(ns), "ms_per_step": ms, "systems_per_s": 1000.0 / ms,
            "precision": precision, "energy": float(U),
            "paper": "under 1 s per step on 2x Tesla P100 or 2x Tesla K80 (Sec. III; precision not stated)"}


def run_series_far_field(dx, dq, w, precision: str, tuning: dict, images_ms: float, U_images: float):
    """The far field by the fitted series evaluated at every particle
    (O(N N_b)) instead of the surface images (O(N N_o)), on the headline
    system: its time beside the images' and the energy difference between
    the two (the images' quadrature and dipole-layer error)."""
    from paper_1806_04801_gb300 import hsma
    with hsma.Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=precision, profile=True,
                   far_field="series") as ps:
        ps.set_tuning(tuning["pair_variant"], tuning["items_per_slot"])
        ps.energy_forces(dx, dq)
        best, U = None, None
        for _ in range(3):
            U = float(ps.energy_forces(dx, dq)[0])
            t = ps.last_timings()
            best = t if best is None or t[7] < best[7] else best
    return {"far_field_ms": best[5], "step_ms": best[7], "images_far_field_ms": images_ms,
            "energy": U, "rel_energy_diff_vs_images": abs(U - U_images) / abs(U_images)}


def run_md(steps: int = 20, sizes=(4000, 100_000), precision: str = "fp32_tc"):
    """Repeated update steps of one moving system, as in molecular dynamics
    (the paper's application, Sec. III and IV): ms per step with the in-set
    rebuilt every step (skin 0) and with the in-set reused between steps
    (hsma_plan_set_inset_skin), and the cost of a step that builds the
    reusable list.  The particles drift along fixed random directions, at
    most 0.9 skin over the run (no rebuild is due)."""
    import torch
    from paper_1806_04801_gb300 import hsma
    from paper_1806_04801_gb300 import inputs as I
    w = I.LARGE_PERIODIC
    skin = 0.02
    out = []
    for n in sizes:
        xyz, q = I.large_periodic(n)
        g = np.random.default_rng(9)
        u = g.standard_normal((n, 3))
        u *= (0.9 * skin / steps) / np.linalg.norm(u, axis=1, keepdims=True)
        x0 = torch.as_tensor(xyz).cuda()
        du = torch.as_tensor(u).cuda()
        dq = torch.as_tensor(q).cuda()
        row = {"N": n, "steps": steps, "skin": skin}
        with hsma.Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=precision) as plan:
            for label, sk in (("rebuild_every_step", 0.0), ("reuse", skin)):
                plan.set_inset_skin(sk)
                plan.energy_forces(x0, dq)          # builds the list (reuse) / warms the graph
                plan.energy_forces(torch.remainder(x0 + 0.5 * du, 1.0), dq)
                times = []
                for t in range(steps):
                    xt = torch.remainder(x0 + t * du, 1.0)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    plan.energy_forces(xt, dq)
                    e1.record()
                    e1.synchronize()
                    times.append(e0.elapsed_time(e1))
                row[label + "_ms"] = float(np.median(times))
            # a step that builds the list: the first one after the skin is set again
            plan.set_inset_skin(skin)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.energy_forces(x0, dq)
            e1.record()
            e1.synchronize()
            row["build_step_ms"] = e0.elapsed_time(e1)
            row["inset_stats"] = plan.inset_stats()
        row["speedup_reuse"] = row["rebuild_every_step_ms"] / row["reuse_ms"]
        out.append(row)
    return {"workload": "md-periodic-p12 (N charges drifting < 0.9 skin, fp32_tc)", "precision": precision,
            "rows": out}


def fixed_tuning(args):
    """(pair variant, items per slot) from --tuning, or None (autotune)."""
    if not args.tuning:
        return None
    v, i = (int(t) for t in args.tuning.split(","))
    return v, i


def run_batched(plan_fp32, plan_fp64, steps: int, warmup: int, flush, fp64_systems: int = 24, fixed=None):
    """256 periodic boxes of log-uniform size in one batched update step
    (persistent launch over all systems, CUDA graph), against the plain
    one-system-per-launch FP64 path."""
    import torch
    from paper_1806_04801_gb300 import inputs as I
    systems = I.batch_periodic()
    xyz = np.concatenate([s[0] for s in systems])
    q = np.concatenate([s[1] for s in systems])
    off = np.concatenate([[0], np.cumsum([len(s[1]) for s in systems])])
    dx = torch.as_tensor(xyz).cuda()
    dq = torch.as_tensor(q).cuda()

    def timed():
        for _ in range(warmup):
            plan_fp32.energy_forces_batched(dx, dq, off)
        torch.cuda.synchronize()
        times = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            E, F, _, st = plan_fp32.energy_forces_batched(dx, dq, off)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        return float(np.median(times)), E
    plan_fp32.set_tuning(4, 24)  # the scalar loop, for reference
    ms_scalar, _ = timed()
    plan_fp32.set_tuning(None, None)  # the library's untuned default
    ms_default, _ = timed()
    if fixed is None:
        plan_fp32.set_tuning(None, None)
        tuning = plan_fp32.autotune(dx, dq, off)
    else:
        plan_fp32.set_tuning(*fixed)
        tuning = {"pair_variant": fixed[0], "items_per_slot": fixed[1], "ms": None, "fixed": True}
    ms, E32 = timed()
    # the plain paths: one system per call (FP64, and FP32 for reference), on
    # a sample of systems
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(len(systems), size=min(fp64_systems, len(systems)), replace=False))
    t64 = t32 = 0.0
    rel, rel_raw = [], []
    sizes = np.diff(off)

    def one(plan, sx, sq):
        plan.energy_forces(sx, sq)  # warm (plan workspace, graph)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        U, _, _, _ = plan.energy_forces(sx, sq)
        e1.record()
        e1.synchronize()
        return U, e0.elapsed_time(e1)
    per_system = []
    for i in pick:
        sx = torch.as_tensor(systems[i][0]).cuda()
        sq = torch.as_tensor(systems[i][1]).cuda()
        U64, dt = one(plan_fp64, sx, sq)
        t64 += dt
        t32 += one(plan_fp32, sx, sq)[1]
        floor = 0.5 * 2.837297479 * float(np.sum(systems[i][1] ** 2))
        rel.append(abs(E32[i] - U64) / max(abs(U64), floor))
        rel_raw.append(abs(E32[i] - U64) / abs(U64))
        per_system.append({"system": int(i), "N": int(sizes[i]), "U_fp64": float(U64),
                           "abs_err": float(abs(E32[i] - U64)), "rel_err": rel_raw[-1],
                           "abs_U_over_floor": abs(U64) / floor})
    # the fit of the whole batch (one product over all 256 right-hand sides):
    # FP64 on the CUDA cores vs split-BF16 on the tensor cores (tcgen05)
    from paper_1806_04801_gb300 import hsma
    wb = I.BATCH_PERIODIC
    fit_ms, e_fit = {}, {}
    for prec, key in (("fp32", "fp64_fit"), ("fp32_tc", "tensor_core_fit")):
        with hsma.Plan(wb.box, wb.bc, wb.p, wb.R, wb.Q, wb.Kmon, precision=prec, profile=True) as pf:
            pf.set_tuning(tuning["pair_variant"], tuning["items_per_slot"])
            pf.energy_forces_batched(dx, dq, off)
            best = None
            for _ in range(3):
                e_fit[key], _, _, _ = pf.energy_forces_batched(dx, dq, off)
                t = pf.last_timings()[3]
                best = t if best is None else min(best, t)
            fit_ms[key] = best
    fit_dev = max(abs(a - b) / max(abs(b), 0.5 * 2.837297479 * float(np.sum(systems[i][1] ** 2)))
                  for i, (a, b) in enumerate(zip(e_fit["tensor_core_fit"], e_fit["fp64_fit"])))
    # scale the sampled FP64 time to all systems by their share of pair work (~ N^2)
    w_all = float(np.sum(sizes.astype(np.float64) ** 2 + 3000.0 * sizes))
    w_pick = float(np.sum(sizes[pick].astype(np.float64) ** 2 + 3000.0 * sizes[pick]))
    t64_all = t64 * w_all / w_pick
    t32_all = t32 * w_all / w_pick
    return {"workload": "batched-256-periodic-p10 (N log-uniform in [500, 50000], +-1)",
            "systems": len(systems), "particles": int(off[-1]), "ms_per_batch": ms,
            "autotuned": tuning, "ms_per_batch_default_tuning": ms_default,
            "ms_per_batch_scalar_variant_4_24": ms_scalar,
            "systems_per_s": len(systems) / (ms / 1000.0),
            "fp64_one_system_per_launch_systems_per_s": len(systems) / (t64_all / 1000.0),
            "fp32_one_system_per_launch_systems_per_s": len(systems) / (t32_all / 1000.0),
            "sampled_systems_for_single_paths": int(len(pick)),
            "speedup_vs_fp64_single": t64_all / ms,
            "max_rel_energy_err_vs_fp64": float(max(rel_raw)),
            "max_rel_energy_err_vs_fp64_floored": float(max(rel)),
            "max_rel_energy_err_vs_fp64_where_abs_U_above_floor": float(max(
                [r["rel_err"] for r in per_system if r["abs_U_over_floor"] >= 1.0] or [0.0])),
            "systems_over_1e-6": [r for r in per_system if r["rel_err"] > 1e-6],
            "energy_err_note": ("plain |U32 - U64| / |U64| per system; floored: denominator max(|U|, 1/2 |xi| "
                                "sum q^2 / L), xi = -2.837297 (the energy scale of the periodic self-images)"),
            "per_system": per_system,
            "precision": f"{plan_fp32.precision}: fp32 pair sums ({'split-BF16 tensor-core' if plan_fp32.precision == 'fp32_tc' else 'fp64'} fit), CUDA graph",
            "fit_ms_per_batch": fit_ms,
            "tensor_core_fit_max_rel_energy_dev": float(fit_dev)}


# ------------------------------------------------------ grounded workload
def run_grounded(steps: int, warmup: int):
    """The 1x1x2 conducting cavity: 20000 charges, p = 10, Kmon = 1500,
    Q = 6000, FP32 pair sums with the split-BF16 tensor-core fit and one
    refinement step; accuracy against the FP64 GPU path."""
    import torch
    from paper_1806_04801_gb300 import hsma
    from paper_1806_04801_gb300 import inputs as I
    w = I.GROUNDED_CAVITY
    xyz, q = I.grounded_cavity()
    dx = torch.as_tensor(xyz).cuda()
    dq = torch.as_tensor(q).cuda()
    with hsma.Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32_tc") as plan:
        plan.autotune(dx, dq)
        for _ in range(warmup):
            plan.energy_forces(dx, dq)
        times = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            U, F, _, ns = plan.energy_forces(dx, dq)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    with hsma.Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp64") as p64:
        U64, F64, _, _ = p64.energy_forces(dx, dq)
    ms = float(np.median(times))
    n = len(q)
    return {"workload": "grounded-1x1x2-N20000-p10 (fp32 pair sums, split-BF16 tensor-core fit + refinement)",
            "ms_per_step": ms, "systems_per_s": 1000.0 / ms, "N_s": int(ns),
            "pair_interactions_per_s": (n * (ns - 1) + 1500 * ns) / (ms / 1000.0),
            "rel_energy_err_vs_fp64": abs(U - U64) / abs(U64),
            "rms_force_err_rel_vs_fp64": float((F - F64).pow(2).mean().sqrt() / F64.pow(2).mean().sqrt())}


# ------------------------------------------------------- serving workload
def run_serving(n_requests: int, rate_hz: float = 2000.0, sweep: bool = True, lanes: int = 4, max_batch: int = 32,
                express_lanes: int = 1, express_max_n: int = 20000, mid_lanes: int = 1, mid_max_n: int = 60000):
    """Poisson stream of periodic boxes with N log-uniform in [1000, 200000]:
    requests are submitted at their arrival times to the continuous-batching
    server; latency is submit -> result.  One express lane (high-priority
    stream) serves requests of at most express_max_n particles, one medium
    lane (middle priority, preemptible pair work) those up to mid_max_n, the
    bulk lanes the rest with preemptible pair work.  Besides p50/p99 of the
    latency, each request's slowdown -- its latency over the time the same
    request takes alone through a plan with host buffers -- is reported:
    with N spanning 200x the latency percentiles mostly restate the size
    mix, the slowdown shows the queueing."""
    import threading
    from paper_1806_04801_gb300 import hsma
    from paper_1806_04801_gb300 import inputs as I
    w = I.SERVING_PERIODIC

    # time alone (one request, host buffers) over the size range, for the slowdown
    sizes_ref = [1000, 3000, 10000, 30000, 100000, 200000]
    alone = []
    with hsma.Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32_tc") as pl:
        for n in sizes_ref:
            x, q = I.uniform_pm1(n, w.box, seed_offset=9000 + n)
            pl.energy_forces(x, q)
            ts = []
            for _ in range(3):
                t0 = time.perf_counter()
                pl.energy_forces(x, q)
                ts.append((time.perf_counter() - t0) * 1000.0)
            alone.append(min(ts))
    la, ln = np.log(alone), np.log(sizes_ref)

    def t_alone(n):
        return float(np.exp(np.interp(np.log(n), ln, la)))

    def replay(rate, count, seed):
        t_arr, sizes = I.poisson_trace(count, rate_hz=rate, seed_offset=4 + seed)
        reqs = [I.uniform_pm1(int(n), w.box, seed_offset=5000 + seed * 1000 + i) for i, n in enumerate(sizes)]
        with hsma.Server(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32_tc", lanes=lanes,
                         max_batch=max_batch, express_lanes=express_lanes, express_max_n=express_max_n,
                         mid_lanes=mid_lanes, mid_max_n=mid_max_n) as srv:
            # warm the lanes (plans, workspaces): a small and a large request each
            for _ in range(lanes):
                for r in (reqs[int(np.argmin(sizes))], reqs[int(np.argmax(sizes))]):
                    tk = srv.submit(*r)
                    srv.result(tk, forces=False)
            tickets = [None] * count
            t0 = time.perf_counter()

            def feeder():
                for i in range(count):
                    delay = t0 + t_arr[i] - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                    tickets[i] = srv.submit(*reqs[i])
            th = threading.Thread(target=feeder)
            th.start()
            lat, batch, slow, nn = [], [], [], []
            th.join()
            for i in range(count):
                code, e, _, info = srv.result(tickets[i], forces=False)
                if code == 0:
                    lat.append(info["latency_ms"])
                    batch.append(info["batch_size"])
                    slow.append(info["latency_ms"] / t_alone(len(reqs[i][1])))
                    nn.append(len(reqs[i][1]))
            wall = time.perf_counter() - t0
            st = srv.stats()
        lat, slow, nn = np.array(lat), np.array(slow), np.array(nn)
        small = nn <= express_max_n
        pct = lambda a, p: float(np.percentile(a, p)) if len(a) else None  # noqa: E731
        by_size = {}
        for name, lo, hi in (("le20k", 0, 20000), ("20k_60k", 20000, 60000), ("gt60k", 60000, np.inf)):
            m = (nn > lo) & (nn <= hi)
            by_size[name] = {"count": int(m.sum()), "p99_ms": pct(lat[m], 99), "slowdown_p50": pct(slow[m], 50),
                             "slowdown_p99": pct(slow[m], 99)}
        return {"rate_hz": rate, "requests": count, "completed": int(len(lat)),
                "systems_per_s": len(lat) / wall, "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
                "slowdown_p50": pct(slow, 50), "slowdown_p99": pct(slow, 99),
                "small": {"count": int(small.sum()), "p50_ms": pct(lat[small], 50), "p99_ms": pct(lat[small], 99)},
                "large": {"count": int((~small).sum()), "p50_ms": pct(lat[~small], 50),
                          "p99_ms": pct(lat[~small], 99)},
                "by_size": by_size,
                "mean_batch": float(np.mean(batch)), "wall_s": wall, "hbm_budget_bytes": int(st["hbm_budget_bytes"])}

    main = replay(rate_hz, n_requests, 0)
    out = {"workload": "serving-periodic-p10 (Poisson arrivals, N log-uniform in [1000, 200000], +-1)",
           "lanes": lanes, "express_lanes": express_lanes, "express_max_n": express_max_n, "mid_lanes": mid_lanes,
           "mid_max_n": mid_max_n, "max_batch": max_batch,
           "alone_ms": dict(zip(map(str, sizes_ref), alone)), "offered": main}
    if sweep:
        cap = main["systems_per_s"]
        out["sweep"] = [replay(f * cap, max(20, int(n_requests * 0.3)), k + 1)
                        for k, f in enumerate((0.25, 0.5, 0.9))]
        out["capacity_systems_per_s"] = cap
    return out


def dist_env():
    """RANK, WORLD_SIZE and LOCAL_RANK from the environment (torchrun), defaults for one process."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks, power and throttle reasons during the timed region."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.path = None
        self.proc = None

    def start(self, gpu_index: int):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    @staticmethod
    def _stamp(field: str):
        """nvidia-smi's local-time timestamp as seconds since the epoch, or None."""
        import datetime
        try:
            return datetime.datetime.strptime(field.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self, window=None) -> dict:
        """Summary of the samples; window = (t0, t1) host times (time.time())
        keeps the samples taken inside the timed region, when the rows carry
        timestamps and some fall inside it."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows, stamps = [], []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            t = self._stamp(parts[0]) if parts else None
            if t is not None:
                parts = parts[1:]
            if len(parts) >= 9:
                rows.append(parts)
                stamps.append(t)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        in_window = False
        if window is not None:
            keep = [r for r, t in zip(rows, stamps) if t is not None and window[0] <= t <= window[1]]
            if keep:
                rows, in_window = keep, True
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        pw = [float(r[3]) for r in rows if r[3].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(rows), "reasons": reasons,
                "samples_in_timed_region": in_window}


# -------------------------------------------------------------- CPU oracle
def cpu_oracle_setup(xyz, q, w, threads: int | None = None):
    """The oracle's plan (preparation step) for the workload, built outside
    any timed region, and the thread count its sums use."""
    from oracle import hsma as oh
    threads = threads or os.cpu_count() or 1
    F2, _ = oh.fib_from_points(w.Q)
    return oh.make_plan(w.box, w.bc, w.p, w.R, w.Kmon, F2), threads


def cpu_oracle_step(xyz, q, plan, threads: int):
    """One complete FP64 update step of the oracle (as it stands: in-set,
    near-field sums at every particle and monitoring point, least squares,
    surface images, energy and forces), timed on the host clock."""
    from oracle import hsma as oh
    t0 = time.perf_counter()
    out = oh.energy_forces(xyz, q, plan, nthreads=threads)
    return time.perf_counter() - t0, out


def reference_arm(args, rank, world, budget_s: float = 150.0):
    """--impl reference: the FP64 CPU oracle on the host cores, complete
    update steps of the same workload.  A step takes tens of seconds, so at
    most as many of the requested steps are timed as fit in budget_s (at
    least one); the line says how many.  Warm-up: the oracle's plan and one
    call on 16 sampled particles (the W requested steps would each be a
    full step)."""
    if rank != 0:
        return 0
    from oracle import hsma as oh
    from paper_1806_04801_gb300 import inputs as I
    w = I.LARGE_PERIODIC
    xyz, q = I.large_periodic(args.n)
    plan, threads = cpu_oracle_setup(xyz, q, w)
    oh.energy_forces(xyz, q, plan, nthreads=threads, sample=np.arange(16))
    times = []
    t_start = time.perf_counter()
    while len(times) < args.steps:
        dt, out = cpu_oracle_step(xyz, q, plan, threads)
        times.append(dt)
        if time.perf_counter() - t_start + dt > budget_s:
            break
    total = sum(times)
    v = len(times) / total
    sample = (f"{len(times)} complete FP64 update steps of the N={args.n} workload (all particles, all "
              f"monitoring points, fit, surface images), plan built outside the timed region")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "systems/s", "n_gpus": 0,
            "steps": len(times), "steps_requested": args.steps, "warmup": args.warmup,
            "warmup_note": "oracle plan + one call on 16 sampled particles",
            "ms_per_step": 1000.0 * total / len(times), "step_s": times, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "N": args.n, "p": w.p, "Kmon": w.Kmon, "Q": w.Q, "Rs": w.R},
            "energy": out["energy"], "n_inset": int(out["n_inset"]),
            "cpu_baseline": {"value": v, "unit": "systems/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "systems/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ ours
def main():
    """The benchmark: one JSON line on rank 0."""
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_1806_04801_gb300 import build as B
    B.build()
    from paper_1806_04801_gb300 import hsma
    from paper_1806_04801_gb300 import inputs as I

    if args.workload != "periodic":
        # one of the other workloads on its own (rank 0, one GPU)
        if rank == 0:
            if args.workload == "batched":
                wb = I.BATCH_PERIODIC
                fl = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
                with hsma.Plan(wb.box, wb.bc, wb.p, wb.R, wb.Q, wb.Kmon, precision=args.precision) as pb32, \
                        hsma.Plan(wb.box, wb.bc, wb.p, wb.R, wb.Q, wb.Kmon, precision="fp64") as pb64:
                    r = run_batched(pb32, pb64, args.steps, args.warmup, fl, fixed=fixed_tuning(args))
                line = {"metric": METRIC, "value": r["systems_per_s"], "unit": "systems/s", "n_gpus": 1,
                        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_batch"],
                        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                        "data": "synthetic", "config": {"workload": r["workload"]}, "detail": r}
            elif args.workload == "basis":
                r = run_basis(args.steps, args.warmup, n=args.basis_points)
                line = {"metric": "harmonic basis evaluations/s (Eq. harmonic) and HBM GB/s written",
                        "value": r["points_per_s"], "unit": "points/s", "n_gpus": 1, "steps": args.steps,
                        "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True,
                        "scaling": "weak", "vs_baseline": None, "dtype": "f32x2 (double-float)",
                        "data": "synthetic", "config": {"workload": r["workload"]}, "roofline": r["roofline"],
                        "detail": r}
            elif args.workload == "paper":
                r = run_paper_config(args.steps, args.warmup, args.precision)
                line = {"metric": METRIC, "value": r["systems_per_s"], "unit": "systems/s", "n_gpus": 1,
                        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
                        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                        "data": "synthetic", "config": {"workload": r["workload"]}, "detail": r}
            elif args.workload == "md":
                r = run_md(max(args.steps, 10))
                big = r["rows"][-1]
                line = {"metric": "ms per MD step (in-set reuse vs rebuild)", "value": 1000.0 / big["reuse_ms"],
                        "unit": "systems/s", "n_gpus": 1, "steps": args.steps, "warmup": 2,
                        "ms_per_step": big["reuse_ms"], "higher_is_better": True, "scaling": "weak",
                        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                        "config": {"workload": r["workload"]}, "detail": r}
            elif args.workload == "grounded":
                r = run_grounded(args.steps, args.warmup)
                line = {"metric": METRIC, "value": r["systems_per_s"], "unit": "systems/s", "n_gpus": 1,
                        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
                        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                        "data": "synthetic", "config": {"workload": r["workload"]}, "detail": r}
            else:
                r = run_serving(args.requests)
                line = {"metric": METRIC, "value": r["offered"]["systems_per_s"], "unit": "systems/s",
                        "n_gpus": 1, "steps": args.requests, "warmup": 0, "higher_is_better": True,
                        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                        "latency_ms": {"p50": r["offered"]["p50_ms"], "p99": r["offered"]["p99_ms"]},
                        "config": {"workload": r["workload"]}, "detail": r}
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return 0

    w = I.LARGE_PERIODIC
    xyz, q = I.uniform_gauss(args.n, w.box, seed_offset=1 + 1000 * rank) if rank else I.large_periodic(args.n)
    dev = torch.device("cuda", local)
    dx = torch.as_tensor(xyz).to(dev)
    dq = torch.as_tensor(q).to(dev)
    plan = hsma.Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=args.precision, profile=True)
    info = plan.info()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    if args.tuning:
        v, i = fixed_tuning(args)
        plan.set_tuning(v, i)
        tuning = {"pair_variant": v, "items_per_slot": i, "ms": None, "fixed": True}
    else:
        tuning = plan.autotune(dx, dq)
    for _ in range(args.warmup):
        plan.energy_forces(dx, dq)
    torch.cuda.synchronize()

    # measured FP32 throughput of this device, beside the count-based peak
    fp32_meas = hsma.fp32_peak() if args.precision != "fp64" else None
    clocks = ClockSampler()
    if rank == 0:
        clocks.start(local)
        time.sleep(0.4)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, pair_ms, launches0 = [], [], hsma.kernel_launches()
    n_inset = None
    wall0 = time.perf_counter()
    epoch0 = time.time()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        U, F, _, n_inset = plan.energy_forces(dx, dq)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        phases = plan.last_timings()
        pair_ms.append(phases[1])
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = hsma.kernel_launches() - launches0
    if dist:
        dist.barrier()
    clk = clocks.stop(window=(epoch0, time.time())) if rank == 0 else None

    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    systems_per_s = world * args.steps / (total_ms / 1000.0)
    n = args.n
    nmon = info["n_mon_targets"]
    pairs_pf = n * (n_inset - 1)
    pairs_p = nmon * n_inset
    pairs_surf = n * 2 * (info["F2"] - 1)
    pairs_total = pairs_pf + pairs_p + pairs_surf
    pair_avg_ms = sum(pair_ms) / len(pair_ms)
    ops = OPS_POT_FIELD * pairs_pf + OPS_POT * pairs_p
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    # the lane peak at the SM clock sampled during the timed region (its
    # median), else at the part's maximum clock
    sm_mhz = (clk or {}).get("sm_mhz") or RECIPE_MAX_SM_MHZ
    peak_ops = sms * FP32_LANES_PER_SM * sm_mhz * 1e6
    achieved = ops / (pair_avg_ms / 1000.0)

    # end to end through the public API with host buffers (pinned)
    hx = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
    hq = torch.empty((n,), dtype=torch.float64, pin_memory=True)
    hx.copy_(torch.as_tensor(xyz))
    hq.copy_(torch.as_tensor(q))
    hxn, hqn = hx.numpy(), hq.numpy()
    plan.energy_forces(hxn, hqn)
    e2e_ms = []
    for _ in range(max(3, min(args.steps, 5))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.energy_forces(hxn, hqn)
        e2e_ms.append((time.perf_counter() - t0) * 1000.0)
    e2e_step = statistics.median(e2e_ms)
    if dist:
        # whole-job figure like `value`: every rank's system, the slowest rank's time
        t = torch.tensor([e2e_step], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_step = float(t.item())

    def side(fn):
        """A secondary figure: its result, or the error it raised (the
        headline figures above do not depend on it and are printed anyway)."""
        try:
            return fn()
        except Exception as e:  # reported in the JSON line, not swallowed
            return {"error": f"{type(e).__name__}: {e}"[:500]}

    accuracy = None
    if not args.no_check and rank == 0:
        def check():
            with hsma.Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp64") as p64:
                U64, F64, _, _ = p64.energy_forces(dx, dq)
            Uc, Fc, _, _ = plan.energy_forces(dx, dq)
            dF = (Fc - F64).double()
            return {"reference": "FP64 GPU path (same inputs)",
                    "rel_energy_err": abs(Uc - U64) / abs(U64),
                    "rms_force_err_rel": float(dF.pow(2).mean().sqrt() / F64.pow(2).mean().sqrt()),
                    "energy": Uc, "energy_fp64": U64}
        accuracy = side(check)

    extras = None
    if rank == 0 and world == 1 and not args.no_extras:
        wb = I.BATCH_PERIODIC

        def batched():
            with hsma.Plan(wb.box, wb.bc, wb.p, wb.R, wb.Q, wb.Kmon, precision=args.precision) as pb32, \
                    hsma.Plan(wb.box, wb.bc, wb.p, wb.R, wb.Q, wb.Kmon, precision="fp64") as pb64:
                return run_batched(pb32, pb64, max(3, min(args.steps, 5)), 2, flush)
        extras = {"batched": side(batched)}
        extras["serving"] = side(lambda: run_serving(args.requests))
        extras["paper_config"] = side(lambda: run_paper_config(max(3, min(args.steps, 5)), 2, args.precision))
        extras["md"] = side(lambda: run_md(10))
        extras["series_far_field"] = side(lambda: run_series_far_field(
            dx, dq, w, args.precision, tuning, phases[5], float(plan.energy_forces(dx, dq)[0])))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:  # the CPU baseline is an N = 1 figure
        def cpu_baseline():
            cplan, threads = cpu_oracle_setup(xyz, q, w)
            dt, out = cpu_oracle_step(xyz, q, cplan, threads)
            return {"value": 1.0 / dt, "unit": "systems/s", "cores": threads, "kind": "oracle",
                    "sample": (f"one complete FP64 update step of the N={n} workload (all {n} particles, "
                               f"{nmon} monitoring targets, fit, surface images), plan built outside the timed "
                               f"region"),
                    "step_s": dt, "n_inset": int(out["n_inset"]),
                    "pairs_per_s": (n * (out["n_inset"] - 1) + nmon * out["n_inset"]) / dt}
        cpu = side(cpu_baseline)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    step_sorted = sorted(step_ms)
    line = {
        "metric": METRIC, "value": systems_per_s, "unit": "systems/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision != "fp64" else "f64", "data": "synthetic",
        "pair_interactions_per_s": world * pairs_total * args.steps / (total_ms / 1000.0),
        "latency_ms": {"p50": float(np.percentile(step_sorted, 50)), "p99": float(np.percentile(step_sorted, 99))},
        "config": {"workload": w.name, "N": n, "p": w.p, "Kmon": w.Kmon, "Q": w.Q, "F2": info["F2"],
                   "N_o": info["n_images"], "Rs": w.R, "N_s": int(n_inset), "precision": args.precision,
                   "autotuned": tuning,
                   "pairs_per_step": {"pot_field": pairs_pf, "pot_only_monitor": pairs_p, "surface": pairs_surf},
                   "l2": "flushed between timed steps (256 MB write, outside the step events)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "kernel": "pair_fp32_kernel" if args.precision != "fp64" else "pair_fp64_kernel",
                     "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                     "unit": "T FP32 lane-instructions/s", "frac": achieved / peak_ops,
                     "traffic": (PAIR_FP32_TRAFFIC_BYTES.get((n, tuning["pair_variant"], tuning["items_per_slot"]))
                                 if args.precision != "fp64" else None),
                     "pairs_per_s": (pairs_pf + pairs_p) / (pair_avg_ms / 1000.0),
                     "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_mhz:.0f} MHz (median SM clock "
                                   f"sampled in the timed region); "
                                   f"{OPS_POT_FIELD} ops per potential+field pair, {OPS_POT} per potential pair",
                     "kernel_ms": pair_avg_ms, "share_of_step": pair_avg_ms / ms_per_step,
                     "measured_fp32": ({"scalar_fma": fp32_meas[0] / 1e12, "packed_fma": fp32_meas[1] / 1e12,
                                        "frac_of_scalar_fma": achieved / fp32_meas[0],
                                        "how": "hsma_fp32_peak: register-only FMA chains, 16 CTAs/SM"}
                                       if fp32_meas else None)},
        "roofline_surface": {"bound": "alu", "kernel": "surface_pairs_fp32_kernel",
                             "achieved": OPS_SURFACE * pairs_surf / (phases[5] / 1000.0) / 1e12,
                             "peak": peak_ops / 1e12, "unit": "T FP32 lane-instructions/s",
                             "frac": OPS_SURFACE * pairs_surf / (phases[5] / 1000.0) / peak_ops,
                             "kernel_ms": phases[5]},
        "e2e": {"value": world * 1000.0 / e2e_step, "unit": "systems/s", "ms_per_step": e2e_step,
                "h2d_bytes_per_step": n * 32, "d2h_bytes_per_step": n * 24 + 8},
        "gpu_launches": int(launches),
        "clocks": clk,
        "phases_ms": dict(zip(["inset", "near_field", "chunk_reduce", "fit", "surface_charges", "surface_pairs",
                               "finalize", "total"], phases)),
        "accuracy": accuracy,
        "workloads": extras,
        "cpu_baseline": cpu,
        "wall_s_timed_region": wall,
    }
    print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
