"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Sizes are chosen so the oracle finishes in seconds while the GPU work still
spans many target blocks and source tiles with ragged tails; the large
periodic workload is checked on sampled particles at full size, in the same
launch configuration the benchmark times.
"""
import numpy as np
import pytest

from gpu_common import TOL, assert_within, errors, rel_energy_err, rms, to_dev
from paper_1806_04801_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the -m gpu tests need a CUDA device"
    from paper_1806_04801_gb300 import build
    build.build()


def hs():
    from paper_1806_04801_gb300 import hsma
    return hsma


def oracle_run(xyz, q, w, sample=None, nthreads=8, F2=None):
    from oracle import hsma as oh
    F2 = F2 or oh.fib_from_points(w.Q)[0]
    plan = oh.make_plan(w.box, w.bc, w.p, w.R, w.Kmon, F2)
    return oh.energy_forces(xyz, q, plan, nthreads=nthreads, sample=sample), plan


PREC = ["fp64", "fp32", "fp32_tc"]


@pytest.fixture(scope="module")
def small_periodic():
    xyz, q = I.small_periodic()
    ref, oplan = oracle_run(xyz, q, I.SMALL_PERIODIC)
    return xyz, q, ref, oplan


@pytest.mark.parametrize("prec", PREC)
def test_small_periodic_energy_forces(small_periodic, prec):
    xyz, q, ref, _ = small_periodic
    w = I.SMALL_PERIODIC
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec) as plan:
        dx, dq = to_dev(xyz, q)
        U, F, pot, ns = plan.energy_forces(dx, dq, forces=True, potentials=True)
        assert ns == ref["n_inset"]
        e = errors(F.cpu().numpy(), ref["forces"], U, ref["energy"], pot.cpu().numpy(), ref["pot"])
        assert_within(e, prec, "small periodic")
        # intermediates: the fitted far field at the particles and the rhs.
        # FP64: the literal dipole layer (charges +-p/dr, dr = 1e-5 Rs) cancels
        # ~5 digits in both implementations, so Phi_out agrees to ~1e-10, not
        # 1e-15.  FP32: b = Phi(x~) - Phi(x) cancels the monitoring potentials
        # by a factor ~rms(Phi_mon)/rms(b), so its relative error is that factor
        # times the ~1e-7 of the pair sums.
        phi_out = plan.last_get(4, len(q))
        tol = 1e-9 if prec == "fp64" else 1e-5
        assert rms(phi_out - ref["phi_out"]) <= tol * rms(ref["phi_out"])
        b = plan.last_get(1, w.Kmon)
        phi_mon = plan.last_get(2, 2 * w.Kmon)
        assert rms(phi_mon - np.concatenate([ref["phi_mon"], ref["phi_mon_partner"]])) <= \
            (1e-13 if prec == "fp64" else 1e-6) * rms(ref["phi_mon"])
        assert rms(b - ref["b"]) <= (1e-11 if prec == "fp64" else 1e-5) * rms(ref["b"])


def test_host_and_device_inputs_agree(small_periodic):
    xyz, q, ref, _ = small_periodic
    w = I.SMALL_PERIODIC
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32") as plan:
        U1, F1, _, _ = plan.energy_forces(np.ascontiguousarray(xyz), np.ascontiguousarray(q))
        dx, dq = to_dev(xyz, q)
        U2, F2, _, _ = plan.energy_forces(dx, dq)
        assert U1 == U2
        assert np.array_equal(F1, F2.cpu().numpy())
        # deterministic across calls
        U3, F3, _, _ = plan.energy_forces(dx, dq)
        assert U3 == U2 and np.array_equal(F3.cpu().numpy(), F1)


def test_plan_matrices_match_oracle(small_periodic):
    import oracle
    from oracle import hsma as oh
    _, _, _, oplan = small_periodic
    w = I.SMALL_PERIODIC
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp64") as plan:
        info = plan.info()
        assert info["F2"] == oplan.F2 and info["F1"] == oplan.F1 and info["n_images"] == 6 * (oplan.F2 + 1)
        mon = plan.get_matrix(0)
        np.testing.assert_allclose(mon[:w.Kmon], oplan.x_mon, rtol=0, atol=1e-14)
        np.testing.assert_allclose(mon[w.Kmon:], oplan.x_mon_partner, rtol=0, atol=1e-14)
        dirs = plan.get_matrix(3)
        wts = plan.get_matrix(4)
        np.testing.assert_allclose(dirs, oplan.dirs, rtol=0, atol=1e-12)
        np.testing.assert_allclose(wts, oplan.weights, rtol=1e-13, atol=1e-15)
        # pseudo-inverse: M+ M = I on the GPU's own fitting matrix
        M = plan.get_matrix(1)
        Mp = plan.get_matrix(2)
        np.testing.assert_allclose(Mp @ M, np.eye(M.shape[1]), atol=1e-9)
        # its least-squares solution agrees with the oracle's solver
        g = np.random.default_rng(0)
        b = g.standard_normal(M.shape[0])
        x_ref, _ = oracle.lstsq(M, b)
        np.testing.assert_allclose(Mp @ b, x_ref, rtol=1e-8, atol=1e-10 * np.abs(x_ref).max())
        # basis at the integration points = oracle basis up to the known column normalisation
        Bq = plan.get_matrix(5)
        Bo = oracle.basis(oplan.Rs * oplan.dirs, w.p, oplan.Rs)
        scale = np.array([np.dot(Bq[:, k], Bo[:, k]) / np.dot(Bo[:, k], Bo[:, k]) for k in range(Bq.shape[1])])
        np.testing.assert_allclose(Bq, Bo * scale, rtol=0, atol=1e-12 * np.abs(Bq).max())
        assert np.all(scale > 0)


def _basis_points():
    """777 normal points (several warps' groups of 32 and a ragged tail) and
    the special rows: the origin, points on the z axis, in the x = 0 and y = 0
    planes, 1e-20 Rs and 1e-30 Rs from the origin (values below FP64's range
    at high degree; the double-float form takes its range-checked path for
    the warp holding them) and 66 Rs out."""
    g = np.random.default_rng(3)
    special = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.8], [0.0, 0.0, -1.1], [0.0, 0.4, -0.3], [0.7, 0.0, 0.2],
                        [3e-21, -5e-21, 2e-21], [50.0, -100.0, 25.0], [1.7, 0.0, 0.0], [1e-30, 2e-30, -1e-30]])
    return np.concatenate([g.standard_normal((777, 3)), special])


def _basis_reference(pts, P, Rs):
    """Oracle basis times the orthonormalisation sqrt((2 - d_m0)(2n + 1)/(4 pi) (n-|m|)!/(n+|m|)!),
    and the row scale sqrt(2 (2n + 1)/(4 pi)) (|x|/Rs)^n that bounds each value."""
    import math
    import oracle
    Bo = oracle.basis(pts, P, Rs)
    rho = np.linalg.norm(pts, axis=1) / Rs
    scale = np.empty_like(Bo)
    for n in range(P + 1):
        for m in range(-n, n + 1):
            k = n * n + n + m
            am = abs(m)
            Bo[:, k] *= math.sqrt((2 if m else 1) * (2 * n + 1) / (4 * math.pi)
                                  * math.factorial(n - am) / math.factorial(n + am))
            with np.errstate(under="ignore"):
                scale[:, k] = math.sqrt(2 * (2 * n + 1) / (4 * math.pi)) * rho ** n
    return Bo, scale


# Basis error bound relative to the row scale: FP64 recurrence a few ulps per
# degree; double-float ~2^-46 per operation over up to 3 operations per degree
BASIS_TOL = {"fp64": 5e-14, "fp32": 5e-12}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("P", [0, 1, 12, 25, 40])
def test_basis_entry_point(precision, P):
    pts = _basis_points()
    Rs = 1.7
    (dp,) = to_dev(pts)
    allocs = hs().allocation_calls()
    B = hs().basis(dp, P, Rs, precision=precision).cpu().numpy()
    assert hs().allocation_calls() == allocs  # both forms take their tables by value: no device buffer
    ref, scale = _basis_reference(pts, P, Rs)
    assert np.all(np.isfinite(B))
    err = np.abs(B - ref)
    bound = BASIS_TOL[precision] * scale + 1e-300
    assert np.all(err <= bound), (precision, P, float(np.max(err / (scale + 1e-300))))
    # the origin: Y_00 only, every other value exactly zero
    assert B[777, 0] == pytest.approx(1.0 / np.sqrt(4 * np.pi), rel=1e-15) and np.all(B[777, 1:] == 0.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_basis_of_a_non_finite_point_is_nan(precision):
    """A point with NaN coordinates between finite ones: Y_00 (which does not
    depend on the point) and NaN everywhere else in its row, the other rows
    as for finite input."""
    pts = _basis_points()[:100].copy()
    pts[37] = np.nan
    (dp,) = to_dev(pts)
    P, Rs = 12, 1.7
    B = hs().basis(dp, P, Rs, precision=precision).cpu().numpy()
    assert B[37, 0] == pytest.approx(1.0 / np.sqrt(4 * np.pi), rel=1e-15)
    assert np.all(np.isnan(B[37, 1:]))
    rows = np.delete(np.arange(100), 37)
    ref, scale = _basis_reference(pts[rows], P, Rs)
    assert np.all(np.abs(B[rows] - ref) <= BASIS_TOL[precision] * scale + 1e-300)


@pytest.mark.parametrize("P,n", [(12, 200_003), (40, 40_001)])
def test_basis_double_float_and_fp64_agree_at_scale(P, n):
    """The two forms at many points spread over the Rs ball (the plan's use:
    monitoring points and directions inside or on the sphere); every warp
    takes several groups of 32 points, and at P = 40 one block fills an SM's
    shared memory."""
    g = np.random.default_rng(31 + P)
    pts = g.standard_normal((n, 3))
    pts *= (g.random(len(pts)) ** (1 / 3) * 1.5 / np.linalg.norm(pts, axis=1))[:, None]
    (dp,) = to_dev(pts)
    Rs = 1.5
    B64 = hs().basis(dp, P, Rs, precision="fp64")
    Bdf = hs().basis(dp, P, Rs, precision="fp32")
    rho = np.linalg.norm(pts, axis=1) / Rs
    n_of_k = np.repeat(np.arange(P + 1), 2 * np.arange(P + 1) + 1)
    scale = np.sqrt(2 * (2 * n_of_k + 1) / (4 * np.pi))[None, :] * rho[:, None] ** n_of_k[None, :]
    err = np.abs((Bdf - B64).cpu().numpy())
    assert np.all(err <= BASIS_TOL["fp32"] * scale + 1e-300)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("ns,nt", [(1, 1), (511, 513), (5000, 1037), (40000, 700)])
def test_coulomb_sum_entry_point(prec, ns, nt):
    import oracle
    g = np.random.default_rng(ns + nt)
    src = np.concatenate([g.random((ns, 3)) * 2 - 1, g.standard_normal((ns, 1))], axis=1)
    tgt = g.random((nt, 3)) * 2 - 1
    tgt[: min(nt, ns) // 3] = src[: min(nt, ns) // 3, :3]  # some targets sit on sources: skipped
    ds, dt = to_dev(src, tgt)
    pot, fld = hs().coulomb_sum(ds, dt, field=True, precision=prec)
    pr, fr = oracle.coulomb(src[:, :3], src[:, 3], tgt, field=True)
    # the oracle skips nothing by distance: recompute with zero-distance pairs removed
    for t in range(min(nt, ns) // 3):
        keep = np.any(src[:, :3] != tgt[t], axis=1)
        pr[t], fr[t] = [v[0] for v in oracle.coulomb(src[keep, :3], src[keep, 3], tgt[t:t + 1], field=True)]
    tol = 1e-12 if prec == "fp64" else 2e-6
    assert rms(pot.cpu().numpy() - pr) <= tol * max(rms(pr), 1e-30)
    assert rms(fld.cpu().numpy() - fr) <= tol * 10 * max(rms(fr), 1e-30)


@pytest.fixture(scope="module")
def grounded_small():
    w = I.Workload("grounded-small", (1.0, 1.0, 2.0), I.GROUNDED, 10, I.GROUNDED_CAVITY.R, 6000, 1500)
    xyz, q = I.uniform_pm1(1500, w.box, seed_offset=20, margin=0.05)
    ref, _ = oracle_run(xyz, q, w)
    return w, xyz, q, ref


@pytest.mark.parametrize("prec", PREC)
def test_grounded_cavity_small(grounded_small, prec):
    w, xyz, q, ref = grounded_small
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec) as plan:
        dx, dq = to_dev(xyz, q)
        U, F, pot, ns = plan.energy_forces(dx, dq, potentials=True)
        assert ns == ref["n_inset"]
        e = errors(F.cpu().numpy(), ref["forces"], U, ref["energy"], pot.cpu().numpy(), ref["pot"])
        assert_within(e, prec, "grounded")


@pytest.mark.parametrize("n", [2, 3, 511, 512, 513, 4097])
def test_ragged_sizes_fp64(n):
    w = I.Workload("tiny", (1.0, 1.0, 1.0), I.PERIODIC, 6, 1.5, 600, 200)
    xyz, q = I.random_neutral(n + (n % 2), w.box, seed_offset=30 + n)
    ref, _ = oracle_run(xyz, q, w)
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp64") as plan:
        dx, dq = to_dev(xyz, q)
        U, F, _, ns = plan.energy_forces(dx, dq)
        assert ns == ref["n_inset"]
        assert_within(errors(F.cpu().numpy(), ref["forces"], U, ref["energy"]), "fp64", f"n={n}")
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32") as plan:
        U, F, _, _ = plan.energy_forces(dx, dq)
        assert_within(errors(F.cpu().numpy(), ref["forces"], U, ref["energy"]), "fp32", f"n={n}")


def test_tensor_core_fit_matches_fp64_fit(small_periodic, grounded_small):
    """The fit on the tensor cores (split-BF16 products, FP32 accumulation in
    tensor memory, one refinement with a compensated residual) against the FP64 fit of the
    same monitoring potentials: the FP32 and tensor-core forms share the pair
    kernel, so b is identical and A differs only by the fit's arithmetic.
    Each operand is held to ~1e-5 relative by its two BF16 words; the
    refinement removes that error from the fitted part of b but not from the
    least-squares residual e = b - M A*, so the coefficients agree to about
    1e-5 |e| / |b| (~2e-7 here).  A product term left out (lo.hi or hi.lo)
    would leave >= 4e-5, a wrong operand layout O(1)."""
    cases = [(small_periodic[0], small_periodic[1], I.SMALL_PERIODIC),
             (grounded_small[1], grounded_small[2], grounded_small[0])]
    for xyz, q, w in cases:
        res = {}
        for prec in ("fp32", "fp32_tc"):
            with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec) as plan:
                plan.energy_forces(*to_dev(xyz, q))
                nb = (w.p + 1) ** 2
                res[prec] = (plan.last_get(1, w.Kmon), plan.last_get(0, nb))
        b32, A32 = res["fp32"]
        btc, Atc = res["fp32_tc"]
        assert np.array_equal(b32, btc)
        assert rms(Atc - A32) <= 2e-6 * rms(A32), (w.name, rms(Atc - A32) / rms(A32))
    # a batch: the tensor-core product spans several systems (MMA N)
    systems = [I.uniform_pm1(int(n), (1.0, 1.0, 1.0), seed_offset=700 + i) for i, n in enumerate([300, 1200, 50, 2000, 800])]
    xyz = np.concatenate([a for a, _ in systems])
    q = np.concatenate([b for _, b in systems])
    off = np.concatenate([[0], np.cumsum([len(b) for _, b in systems])])
    w = I.SMALL_PERIODIC
    E = {}
    for prec in ("fp32", "fp32_tc"):
        with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec) as plan:
            E[prec], _, _, st = plan.energy_forces_batched(*to_dev(xyz, q), off)
            assert np.all(st == 0)
    for i in range(len(systems)):
        assert rel_energy_err(E["fp32_tc"][i], E["fp32"][i], systems[i][1]) <= 5e-7, i


def _tc_batch_against_fp64_fit(w, sizes, seed):
    """Energies of a batch with the tensor-core fit against the same batch
    with the FP64 fit (same pair sums, so only the fit differs)."""
    systems = [I.uniform_pm1(int(n), w.box, seed_offset=seed + i) for i, n in enumerate(sizes)]
    xyz = np.concatenate([a for a, _ in systems])
    q = np.concatenate([b for _, b in systems])
    off = np.concatenate([[0], np.cumsum([len(b) for _, b in systems])])
    E = {}
    for prec in ("fp32", "fp32_tc"):
        with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec) as plan:
            E[prec], _, _, st = plan.energy_forces_batched(*to_dev(xyz, q), off)
            assert np.all(st == 0)
    return [rel_energy_err(E["fp32_tc"][i], E["fp32"][i], systems[i][1]) for i in range(len(systems))]


def test_tensor_core_fit_many_systems():
    """More than eight systems: the refinement residual takes its
    many-systems form (a lane per system, blocks of 32 systems); 40 systems
    span two such blocks."""
    errs = _tc_batch_against_fp64_fit(I.SMALL_PERIODIC, [150 + 37 * i for i in range(40)], 720)
    assert max(errs) <= 5e-7, errs


def test_tensor_core_fit_above_the_shared_memory_form():
    """At p = 34 (1224 fitted columns) the residual's operands no longer fit
    in shared memory and are read from global memory instead; both the
    few-systems (3 systems) and the many-systems (12) forms.  alpha = 1.5:
    at alpha = 2 and this order the reduced-precision path as a whole (FP32
    pair sums with an FP64 fit) already leaves ~4e-5 of the FP64 energy,
    because the fit maps rounding in b onto the high-order coefficients
    amplified by about alpha^P (Sec. II.A error estimate)."""
    P = 34
    w = I.Workload("periodic-p34", (1.0, 1.0, 1.0), I.PERIODIC, P, 1.5 * 0.5 * 3.0 ** 0.5, 6000, 1400)
    for sizes in ([300, 500, 400], [200 + 20 * i for i in range(12)]):
        errs = _tc_batch_against_fp64_fit(w, sizes, 760)
        assert max(errs) <= 1e-6, errs


def test_tensor_core_fit_high_order():
    """The tensor-core fit at the paper's largest order (P = 25: M+ is
    675 x 1250, six M tiles of the tcgen05 product, K split over 20 CTAs) on a
    random-sign lattice, against the same plan with the FP64 fit."""
    xyz, q = I.lattice_random_sign(10, 1.0, seed_offset=510)
    P = 25
    w = I.Workload("lattice-p25", (1.0, 1.0, 1.0), I.PERIODIC, P, 2.0 * 0.5 * 3.0 ** 0.5, 6000, 2 * P * P)
    dx, dq = to_dev(xyz, q)
    res = {}
    for prec in ("fp32", "fp32_tc"):
        with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec) as plan:
            U, F, _, _ = plan.energy_forces(dx, dq)
            res[prec] = (U, F.cpu().numpy(), plan.last_get(0, (P + 1) ** 2))
    (U32, F32, A32), (Utc, Ftc, Atc) = res["fp32"], res["fp32_tc"]
    assert np.all(np.isfinite(Atc))
    assert rel_energy_err(Utc, U32, q) <= 1e-6, (Utc, U32)
    assert rms(Ftc - F32) <= 1e-5 * rms(F32)


# every blocking of the FP32 pair kernel the autotuner may pick
PAIR_VARIANTS = [4, 5, 2, 12, 13, 14, 15, 16, 17]


@pytest.mark.parametrize("variant", PAIR_VARIANTS)
def test_pair_variants_against_oracle(small_periodic, grounded_small, variant):
    """Each FP32 pair-kernel variant (scalar and packed, two and four targets
    per thread) at a fine and a coarse work split, periodic and grounded,
    against the oracle; plus a ragged size whose last tile and block are
    partial."""
    xyz, q, ref, _ = small_periodic
    w = I.SMALL_PERIODIC
    for ips in (8, 48):
        with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32") as plan:
            plan.set_tuning(variant, ips)
            U, F, pot, ns = plan.energy_forces(*to_dev(xyz, q), potentials=True)
            assert ns == ref["n_inset"]
            e = errors(F.cpu().numpy(), ref["forces"], U, ref["energy"], pot.cpu().numpy(), ref["pot"])
            assert_within(e, "fp32", f"periodic variant {variant} items {ips}")
    wg, xg, qg, refg = grounded_small
    with hs().Plan(wg.box, wg.bc, wg.p, wg.R, wg.Q, wg.Kmon, precision="fp32") as plan:
        plan.set_tuning(variant, 16)
        U, F, pot, ns = plan.energy_forces(*to_dev(xg, qg), potentials=True)
        assert ns == refg["n_inset"]
        e = errors(F.cpu().numpy(), refg["forces"], U, refg["energy"], pot.cpu().numpy(), refg["pot"])
        assert_within(e, "fp32", f"grounded variant {variant}")
    wt = I.Workload("tiny", (1.0, 1.0, 1.0), I.PERIODIC, 6, 1.5, 600, 200)
    xt, qt = I.random_neutral(514, wt.box, seed_offset=30 + 513)
    reft, _ = oracle_run(xt, qt, wt)
    with hs().Plan(wt.box, wt.bc, wt.p, wt.R, wt.Q, wt.Kmon, precision="fp32") as plan:
        plan.set_tuning(variant, 24)
        U, F, _, _ = plan.energy_forces(*to_dev(xt, qt))
        assert_within(errors(F.cpu().numpy(), reft["forces"], U, reft["energy"]), "fp32", f"n=514 variant {variant}")


def test_noncubic_periodic_box_and_wrapping():
    """A periodic box with unequal sides (1.0 x 1.3 x 0.8, Rs = sqrt(3) R0:
    two image shells along z, 75 shifts) against the oracle in FP64 and FP32;
    and periodic input outside [0, L) (whole periods added and subtracted)
    gives the result of the wrapped input."""
    box = (1.0, 1.3, 0.8)
    from oracle import hsma as oh
    Rs = oh.alpha_to_rs(box, 3.0 ** 0.5)
    w = I.Workload("noncubic", box, I.PERIODIC, 8, Rs, 2000, 600)
    xyz, q = I.uniform_pm1(800, box, seed_offset=90)
    ref, _ = oracle_run(xyz, q, w)
    shifted = xyz + np.asarray(box) * np.random.default_rng(91).integers(-2, 3, size=xyz.shape)
    for prec in ("fp64", "fp32"):
        with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec) as plan:
            assert plan.info()["n_shifts"] == 75
            U, F, pot, ns = plan.energy_forces(*to_dev(xyz, q), potentials=True)
            assert ns == ref["n_inset"]
            e = errors(F.cpu().numpy(), ref["forces"], U, ref["energy"], pot.cpu().numpy(), ref["pot"])
            assert_within(e, prec, f"non-cubic {prec}")
            Us, Fs, _, ns2 = plan.energy_forces(*to_dev(shifted, q))
            assert ns2 == ns
            assert abs(Us - U) <= (1e-12 if prec == "fp64" else 1e-7) * abs(U)
            assert rms(Fs.cpu().numpy() - F.cpu().numpy()) <= (1e-10 if prec == "fp64" else 1e-6) * rms(F.cpu().numpy())


def test_error_codes():
    hsma = hs()
    w = I.SMALL_PERIODIC
    with hsma.Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon) as plan:
        xyz, q = I.small_periodic()
        q2 = q.copy()
        q2[0] += 0.5
        with pytest.raises(hsma.HsmaError) as ei:
            plan.energy_forces(*to_dev(xyz, q2))
        assert ei.value.code == -2
        xyz2 = xyz.copy()
        xyz2[5] = xyz2[17]
        with pytest.raises(hsma.HsmaError) as ei:
            plan.energy_forces(*to_dev(xyz2, q))
        assert ei.value.code == -4
        xyz3 = xyz.copy()
        xyz3[3, 1] = np.nan
        with pytest.raises(hsma.HsmaError) as ei:
            plan.energy_forces(*to_dev(xyz3, q))
        assert ei.value.code == -3
        # the plan stays usable after errors
        U, F, _, _ = plan.energy_forces(*to_dev(xyz, q))
        assert np.isfinite(U)
    g = I.GROUNDED_CAVITY
    with hsma.Plan(g.box, g.bc, 6, g.R, 600, 200) as plan:
        xyz, q = I.uniform_pm1(100, g.box, seed_offset=40, margin=0.05)
        xyz[7, 2] = 2.5
        with pytest.raises(hsma.HsmaError) as ei:
            plan.energy_forces(*to_dev(xyz, q))
        assert ei.value.code == -3
    with pytest.raises(hsma.HsmaError):
        hsma.Plan((1, 1, 1), 0, 8, 0.5, 2000, 600)  # sphere inside the box
    with pytest.raises(hsma.HsmaError):
        hsma.Plan((1, 1, 1), 0, 8, 1.5, 2000, 10)  # fewer monitoring points than columns


def _near_sphere_sources(box, Rs, bc, deltas, seed):
    """Sources (box frame) each with one image at |r| = Rs (1 + delta): the
    image direction is a shift whose box lies about Rs away, tilted at
    random, and the source is solved from image = S c + s L (S flips the odd
    axes of a grounded shift), kept well inside the box."""
    import itertools
    rng = np.random.default_rng(seed)
    L = np.asarray(box, dtype=np.float64)
    cands = [np.array(s) for s in itertools.product(range(-3, 4), repeat=3)
             if any(s) and abs(np.linalg.norm(np.array(s) * L) - Rs) < 0.3 * L.min()]
    pts, want = [], []
    for d in deltas:
        while True:
            s = cands[rng.integers(len(cands))]
            u = s * L + rng.normal(scale=0.05, size=3)
            r = Rs * (1.0 + d) * u / np.linalg.norm(u)
            S = np.where((s % 2 == 1) & (bc == I.GROUNDED), -1.0, 1.0)
            c = S * (r - s * L)
            if np.all(np.abs(c) < 0.45 * L):
                break
        pts.append(c + 0.5 * L)
        want.append((S * c + s * L, d < 0))
    return np.array(pts), want


@pytest.mark.parametrize("bc", [I.PERIODIC, I.GROUNDED])
def test_inset_membership_at_the_sphere(bc):
    """Images within 1e-9 .. 1e-2 (relative) of the sphere |r| = Rs, on both
    sides, inside and outside the band where the in-set test falls back from
    FP32 to FP64: the in-set size and Phi_in at every particle (which moves
    by O(1) if one image changes side) match the oracle."""
    import oracle
    box = (1.0, 1.0, 1.0)
    w = I.Workload("near-sphere", box, bc, 8, 1.5, 2000, 600)
    mags = [1e-2, 1e-3, 2e-4, 1e-4, 1e-5, 1e-6, 1e-7, 1e-9]
    deltas = [sg * m for m in mags for sg in (1.0, -1.0)] * 2
    xyz, want = _near_sphere_sources(box, w.R, bc, deltas, seed=1806)
    n = len(xyz)
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    # the construction: each planned image sits on the side its delta says
    c = xyz - 0.5 * np.asarray(box)
    sx, _, _, _ = oracle.inset(c, q, np.asarray(box), bc, w.R)
    for img, inside in want:
        hit = np.any(np.all(np.abs(sx[n:] - img) <= 1e-12, axis=1))
        assert hit == inside, (img, inside)
    ref, _ = oracle_run(xyz, q, w)
    for prec in PREC:
        with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec) as plan:
            U, F, pot, ns = plan.energy_forces(*to_dev(xyz, q), potentials=True)
            assert ns == ref["n_inset"], prec
            phi_in = plan.last_get(3, n)
            tol = 1e-12 if prec == "fp64" else 1e-6
            assert rms(phi_in - ref["phi_in"]) <= tol * rms(ref["phi_in"]), prec


@pytest.mark.parametrize("scale", [7.3, 1000.0])
def test_scale_invariance(scale):
    """Gaussian units have no length scale: a box, sphere and positions all
    scaled by s give U / s and F / s^2 (potentials / s).  Every plan length
    (monitoring points, Rs, Delta r, images) scales with the box, so the two
    runs differ by rounding only; at s = 1000 the FP32 path also shows that
    its split (hi + lo) positions keep FP32 differences exact relative to
    the box, not to the origin."""
    w = I.SMALL_PERIODIC
    xyz, q = I.small_periodic()
    big = tuple(scale * b for b in w.box)
    # two runs, each within the parity tolerance of the oracle
    for prec, tol, ftol in (("fp64", 1e-11, 1e-11), ("fp32", 2e-6, 2e-5)):
        with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec) as p1, \
                hs().Plan(big, w.bc, w.p, scale * w.R, w.Q, w.Kmon, precision=prec) as ps:
            U1, F1, pot1, n1 = p1.energy_forces(*to_dev(xyz, q), potentials=True)
            Us, Fs, pots, ns = ps.energy_forces(*to_dev(scale * xyz, q), potentials=True)
            assert ns == n1
            assert abs(Us * scale - U1) <= tol * abs(U1), (prec, Us * scale, U1)
            F1 = F1.cpu().numpy()
            assert rms(Fs.cpu().numpy() * scale ** 2 - F1) <= ftol * rms(F1), prec
            pot1 = pot1.cpu().numpy()
            assert rms(pots.cpu().numpy() * scale - pot1) <= tol * rms(pot1), prec


def test_empty_input_and_single_grounded_charge():
    """Degenerate inputs: an empty system is an argument error (alone or
    inside a batch) and leaves the plan usable; one charge in a grounded box,
    whose only partners are its own images, matches the oracle and the exact
    doubled-cell lattice."""
    from oracle import checks
    hsma = hs()
    w = I.SMALL_PERIODIC
    xyz, q = I.small_periodic()
    with hsma.Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32") as plan:
        with pytest.raises(hsma.HsmaError) as ei:
            plan.energy_forces(np.zeros((0, 3)), np.zeros(0))
        assert ei.value.code == -1
        both_x = np.concatenate([xyz, xyz])
        both_q = np.concatenate([q, q])
        with pytest.raises(hsma.HsmaError) as ei:
            plan.energy_forces_batched(*to_dev(both_x, both_q), [0, len(q), len(q), 2 * len(q)])
        assert ei.value.code == -1
        U, _, _, _ = plan.energy_forces(*to_dev(xyz, q))
        assert np.isfinite(U)
    g = I.Workload("grounded-one", (1.0, 1.0, 1.0), I.GROUNDED, 12, 1.5, 6000, 1500)
    x1 = np.array([[0.31, 0.62, 0.45]])
    q1 = np.array([1.0])
    ref, _ = oracle_run(x1, q1, g)
    _, fld, U_exact = checks.grounded_box_exact(x1, q1, np.array(g.box))
    for prec in ("fp64", "fp32"):
        with hsma.Plan(g.box, g.bc, g.p, g.R, g.Q, g.Kmon, precision=prec) as plan:
            U, F, pot, ns = plan.energy_forces(*to_dev(x1, q1), potentials=True)
            assert ns == ref["n_inset"]
            e = errors(F.cpu().numpy(), ref["forces"], U, ref["energy"], pot.cpu().numpy(), ref["pot"])
            assert_within(e, prec, f"one grounded charge {prec}")
            # the method's own accuracy against the exact image lattice
            assert abs(U - U_exact) <= 1e-6 * abs(U_exact), (prec, U, U_exact)
            assert np.abs(F.cpu().numpy()[0] - q1[0] * fld[0]).max() <= 1e-4 * np.abs(fld[0]).max()


def test_batched_matches_single_and_oracle():
    w = I.BATCH_PERIODIC
    sizes = [600, 1000, 1500, 2048, 333 * 2]
    systems = [I.uniform_pm1(n, w.box, seed_offset=50 + i) for i, n in enumerate(sizes)]
    xyz = np.concatenate([s[0] for s in systems])
    q = np.concatenate([s[1] for s in systems])
    off = np.concatenate([[0], np.cumsum([len(s[1]) for s in systems])])
    for prec in ("fp64", "fp32"):
        with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec) as plan:
            dx, dq = to_dev(xyz, q)
            E, F, _, st = plan.energy_forces_batched(dx, dq, off)
            F = F.cpu().numpy()
            assert np.all(st == 0)
            for i, (sx, sq) in enumerate(systems):
                U1, F1, _, _ = plan.energy_forces(*to_dev(sx, sq))
                sl = slice(off[i], off[i + 1])
                assert abs(E[i] - U1) <= TOL[prec]["energy"] * abs(U1)
                assert rms(F[sl] - F1.cpu().numpy()) <= TOL[prec]["force_rms"] * rms(F1.cpu().numpy())
                if i in (0, 3):
                    ref, _ = oracle_run(sx, sq, w)
                    assert_within(errors(F[sl], ref["forces"], E[i], ref["energy"]), prec, f"batched sys {i}")


def test_batched_grounded_and_per_system_errors():
    """Grounded cavities of ragged sizes in one batched call match the same
    systems one by one (all three precisions) and the oracle (FP64); a batch
    with one non-neutral periodic system fails with that system's code in
    its slot and zeros elsewhere, and the plan serves the next batch."""
    hsma = hs()
    g = I.Workload("grounded-batch", (1.0, 1.0, 2.0), I.GROUNDED, 8, I.GROUNDED_CAVITY.R, 2000, 600)
    sizes = [700, 1300, 257, 1024]
    systems = [I.uniform_pm1(n, g.box, seed_offset=70 + i, margin=0.01) for i, n in enumerate(sizes)]
    xyz = np.concatenate([s[0] for s in systems])
    q = np.concatenate([s[1] for s in systems])
    off = np.concatenate([[0], np.cumsum([len(s[1]) for s in systems])])  # sizes rounded to even
    ref, _ = oracle_run(*systems[2], g)
    for prec in PREC:
        with hsma.Plan(g.box, g.bc, g.p, g.R, g.Q, g.Kmon, precision=prec) as plan:
            E, F, _, st = plan.energy_forces_batched(*to_dev(xyz, q), off)
            F = F.cpu().numpy()
            assert np.all(st == 0)
            for i, (sx, sq) in enumerate(systems):
                U1, F1, _, _ = plan.energy_forces(*to_dev(sx, sq))
                F1 = F1.cpu().numpy()
                sl = slice(off[i], off[i + 1])
                assert abs(E[i] - U1) <= TOL[prec]["energy"] * abs(U1), (prec, i)
                assert rms(F[sl] - F1) <= TOL[prec]["force_rms"] * rms(F1), (prec, i)
            sl = slice(off[2], off[3])
            assert_within(errors(F[sl], ref["forces"], E[2], ref["energy"]), prec, f"grounded batch {prec}")
    w = I.SMALL_PERIODIC
    per = [I.uniform_pm1(n, w.box, seed_offset=80 + i) for i, n in enumerate([500, 800, 600])]
    bad_q = per[1][1].copy()
    bad_q[0] += 1.0
    xyz = np.concatenate([s[0] for s in per])
    qb = np.concatenate([per[0][1], bad_q, per[2][1]])
    qg = np.concatenate([s[1] for s in per])
    off = np.concatenate([[0], np.cumsum([len(s[1]) for s in per])])
    with hsma.Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32") as plan:
        with pytest.raises(hsma.HsmaError) as ei:
            plan.energy_forces_batched(*to_dev(xyz, qb), off)
        assert ei.value.code == -2
        assert list(ei.value.status) == [0, -2, 0]
        E, _, _, st = plan.energy_forces_batched(*to_dev(xyz, qg), off)
        assert np.all(st == 0) and np.all(np.isfinite(E))


@pytest.mark.slow
def test_large_periodic_sampled_full_size():
    """The benchmarked workload at full size (100000 charges, p = 12): FP32 and
    FP64 GPU results on sampled particles against the oracle, and the FP32
    energy against the FP64 GPU energy."""
    w = I.LARGE_PERIODIC
    xyz, q = I.large_periodic()
    sample = np.linspace(0, len(q) - 1, 48).astype(np.int64)
    ref, _ = oracle_run(xyz, q, w, sample=sample, nthreads=16)
    dx, dq = to_dev(xyz, q)
    res = {}
    # FP64 and every FP32 pair-kernel variant (the benchmark times the one the
    # autotuner picks, with 48 items per slot)
    runs = [("fp64", None)] + [("fp32", v) for v in PAIR_VARIANTS]
    for prec, variant in runs:
        with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec) as plan:
            if variant is not None:
                plan.set_tuning(variant, 48)
            U, F, pot, ns = plan.energy_forces(dx, dq, potentials=True)
            assert ns == ref["n_inset"]
            res[(prec, variant)] = (U, F.cpu().numpy(), pot.cpu().numpy())
            r = res[(prec, variant)]
            e = errors(r[1][sample], ref["forces"], None, None, r[2][sample], ref["pot"])
            tol = TOL[prec]
            assert e["force_rms"] <= tol["force_rms"] and e["pot_rms"] <= tol["pot_rms"], (prec, variant, e)
    U64, F64 = res[("fp64", None)][0], res[("fp64", None)][1]
    for v in PAIR_VARIANTS:
        U32, F32 = res[("fp32", v)][0], res[("fp32", v)][1]
        assert abs(U32 - U64) <= 1e-6 * abs(U64), v
        assert rms(F32 - F64) <= 1e-5 * rms(F64), v


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp32_tc", "fp64"])
def test_grounded_cavity_full_size(prec):
    """The 1x1x2 conducting cavity at full size (20000 charges, p = 10,
    Kmon = 1500, Q = 6000): energy against the oracle's full energy, forces on
    sampled particles."""
    w = I.GROUNDED_CAVITY
    xyz, q = I.grounded_cavity()
    from oracle import hsma as oh
    F2, _ = oh.fib_from_points(w.Q)
    oplan = oh.make_plan(w.box, w.bc, w.p, w.R, w.Kmon, F2)
    ref = oh.energy_forces(xyz, q, oplan, nthreads=16)
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec) as plan:
        U, F, pot, ns = plan.energy_forces(*to_dev(xyz, q), potentials=True)
        assert ns == ref["n_inset"]
        e = errors(F.cpu().numpy(), ref["forces"], U, ref["energy"], pot.cpu().numpy(), ref["pot"])
        assert_within(e, prec, "grounded full size")


@pytest.mark.slow
def test_large_periodic_fp64_full_energy():
    """The benchmarked periodic workload (100000 charges): the FP64 GPU energy
    against the oracle's full FP64 energy (1.4e11 pairs on the host cores)."""
    import os
    w = I.LARGE_PERIODIC
    xyz, q = I.large_periodic()
    from oracle import hsma as oh
    F2, _ = oh.fib_from_points(w.Q)
    oplan = oh.make_plan(w.box, w.bc, w.p, w.R, w.Kmon, F2)
    ref = oh.energy_forces(xyz, q, oplan, nthreads=os.cpu_count() or 16)
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp64") as plan:
        U, F, _, _ = plan.energy_forces(*to_dev(xyz, q))
    assert_within(errors(F.cpu().numpy(), ref["forces"], U, ref["energy"]), "fp64", "periodic 1e5 full")
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32") as plan:
        U32, F32, _, _ = plan.energy_forces(*to_dev(xyz, q))
    assert_within(errors(F32.cpu().numpy(), ref["forces"], U32, ref["energy"]), "fp32", "periodic 1e5 full")


@pytest.mark.parametrize("bc", ["periodic", "grounded"])
def test_series_far_field(bc):
    """Far field by the fitted series at each particle (far_field = series):
    against the oracle's series evaluation (its field by central differences,
    accurate to ~1e-9) and against the GPU's own surface-image path."""
    from oracle import hsma as oh
    if bc == "periodic":
        w = I.SMALL_PERIODIC
        xyz, q = I.small_periodic()
    else:
        w = I.Workload("grounded-small", (1.0, 1.0, 2.0), I.GROUNDED, 10, I.GROUNDED_CAVITY.R, 6000, 1500)
        xyz, q = I.uniform_pm1(1500, w.box, seed_offset=20, margin=0.05)
    F2, _ = oh.fib_from_points(w.Q)
    oplan = oh.make_plan(w.box, w.bc, w.p, w.R, w.Kmon, F2)
    ref = oh.energy_forces_series(xyz, q, oplan, nthreads=8)
    dx, dq = to_dev(xyz, q)
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp64", far_field="series") as plan:
        U, F, pot, _ = plan.energy_forces(dx, dq, potentials=True)
        e = errors(F.cpu().numpy(), ref["forces"], U, ref["energy"], pot.cpu().numpy(), ref["pot"])
        assert e["energy"] <= 1e-10 and e["pot_rms"] <= 1e-10 and e["force_rms"] <= 1e-8, e
        phi_out = plan.last_get(4, len(q))
        assert rms(phi_out - ref["phi_out"]) <= 1e-10 * rms(ref["phi_out"])
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp32", far_field="series") as plan:
        U32, F32, _, _ = plan.energy_forces(dx, dq)
        assert_within(errors(F32.cpu().numpy(), ref["forces"], U32, ref["energy"]), "fp32", "series fp32")
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision="fp64") as plan:
        Ui, Fi, _, _ = plan.energy_forces(dx, dq)
    # mapping accuracy of the surface images (quadrature + O(dr^2))
    assert abs(Ui - U) <= 1e-7 * abs(U)


@pytest.mark.parametrize("P", [25, 30, 40])
def test_series_far_field_high_order(P):
    """The series far field at high harmonic order: the FP32 kernel runs the
    fully normalised recurrence, whose values stay of order (r/Rs)^n, so it
    serves every order up to the largest (the unnormalised (2m - 1)!! would
    leave the FP32 range near m = 29); it agrees with the FP64 path's series
    and, up to P = 30, with the surface images of the same plan."""
    w = I.Workload(f"series-p{P}", (1.0, 1.0, 1.0), I.PERIODIC, P, 2.0 * 0.5 * 3.0 ** 0.5, 6000, 2 * (P + 1) ** 2)
    xyz, q = I.random_neutral(256, w.box, seed_offset=60 + P)
    dx, dq = to_dev(xyz, q)
    out = {}
    for prec, far in (("fp64", "series"), ("fp32", "series"), ("fp32", "images")):
        with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec, far_field=far) as plan:
            U, F, _, _ = plan.energy_forces(dx, dq)
            F = F.cpu().numpy()
            assert np.isfinite(U) and np.all(np.isfinite(F)), (prec, far)
            out[(prec, far)] = (U, F)
    U64, F64 = out[("fp64", "series")]
    # the FP32 series against the FP64 series: the reduced-form bar
    Us, Fs = out[("fp32", "series")]
    assert rel_energy_err(Us, U64, q) <= 1e-6, (Us, U64)
    assert rms(Fs - F64) <= 1e-5 * rms(F64)
    # the surface images add the quadrature's error for harmonics up to
    # degree P (N_o = 5928 directions): a looser, method-level bound
    if P > 30:
        return
    Ui, Fi = out[("fp32", "images")]
    assert rel_energy_err(Ui, U64, q) <= 1e-5, (Ui, U64)
    assert rms(Fi - F64) <= 1e-4 * rms(F64)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("bc", ["periodic", "grounded"])
def test_target_sharded_stages(prec, bc):
    """hsma_shard_near / hsma_shard_far for every part of a split step (all
    parts on this one GPU, exchanges as plain sums) reproduce
    hsma_energy_forces."""
    from paper_1806_04801_gb300 import sharded
    if bc == "periodic":
        w = I.SMALL_PERIODIC
        xyz, q = I.uniform_pm1(5000, w.box, seed_offset=402)
    else:
        w = I.Workload("grounded-small", (1.0, 1.0, 2.0), I.GROUNDED, 10, I.GROUNDED_CAVITY.R, 6000, 1500)
        xyz, q = I.uniform_pm1(3000, w.box, seed_offset=403, margin=0.05)
    dx, dq = to_dev(xyz, q)
    with hs().Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon, precision=prec) as plan:
        U0, F0, P0, _ = plan.energy_forces(dx, dq, potentials=True)
        F0 = F0.cpu().numpy()
        for nparts in (1, 2, 3, 8):
            U, F, pot = sharded.shard_update_local(sharded.GpuBackend(plan), dx, dq, nparts)
            tol = 1e-12 if prec == "fp64" else 1e-7
            assert abs(U - U0) <= tol * abs(U0), (nparts, U, U0)
            assert rms(F - F0) <= tol * 10 * rms(F0), nparts
        # host inputs give the same split
        U_h, F_h, _ = sharded.shard_update_local(sharded.GpuBackend(plan), xyz, q, 2)
        assert abs(U_h - U0) <= (1e-12 if prec == "fp64" else 1e-7) * abs(U0)
