"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/hsma.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hsma.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hsma_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1806_04801_gb300 import build
    build.build()
    from paper_1806_04801_gb300 import hsma
    return hsma.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("hsma_plan", "hsma_energy_forces", "hsma_energy_forces_batched", "hsma_plan_destroy",
                 "hsma_strerror", "hsma_plan_footprint"):
        assert must in names


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_1806_04801_gb300 import hsma
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in hsma.SIGNATURES, f"{name} has no ctypes signature in the binding"


def test_host_only_calls(lib):
    from paper_1806_04801_gb300 import hsma
    assert "sm_103a" in hsma.version()
    assert hsma.strerror(0) == "ok"
    assert "neutral" in hsma.strerror(-2)
    o = hsma.hsma_opts()
    assert lib.hsma_opts_default(ctypes.byref(o)) == 0
    assert o.precision == hsma.FP32_ACC64 and o.use_graphs == 1
    assert lib.hsma_opts_default(None) == -1
    assert hsma.kernel_launches() >= 0


def test_library_is_built_for_sm_103a_only():
    import subprocess
    from paper_1806_04801_gb300 import build
    src = open(os.path.join(ROOT, "paper_1806_04801_gb300", "build.py")).read()
    assert "arch=compute_103a,code=sm_103a" in src
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    from paper_1806_04801_gb300 import hsma
    monkeypatch.setattr(hsma, "_LIB", None)
    monkeypatch.setattr(hsma, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        hsma.lib()


def test_argument_errors_are_caught_before_any_device_work(lib):
    """Every entry point validates its arguments on the host and returns
    HSMA_E_ARG (or HSMA_E_CAPACITY for a direct sum beyond the static array)
    before it touches the device, so these calls run without a GPU."""
    from paper_1806_04801_gb300 import hsma
    ARG, CAP = -1, -11
    D3 = ctypes.c_double * 3
    out = ctypes.c_void_p()
    unit = D3(1.0, 1.0, 1.0)

    def plan(box=unit, bc=0, p=8, R=1.5, Q=2000, K=600, **opt):
        o = hsma.hsma_opts()
        lib.hsma_opts_default(ctypes.byref(o))
        for k, v in opt.items():
            setattr(o, k, v)
        return lib.hsma_plan(ctypes.byref(out), box, bc, p, R, Q, K, ctypes.byref(o))

    assert lib.hsma_plan(None, unit, 0, 8, 1.5, 2000, 600, None) == ARG
    assert lib.hsma_plan(ctypes.byref(out), None, 0, 8, 1.5, 2000, 600, None) == ARG
    assert plan(box=D3(1.0, 0.0, 1.0)) == ARG             # empty box
    assert plan(box=D3(1.0, -1.0, 1.0)) == ARG
    assert plan(bc=2) == ARG                               # neither periodic nor grounded
    assert plan(p=0) == ARG and plan(p=41) == ARG          # harmonic order out of range
    assert plan(R=0.5 * 3 ** 0.5) == ARG                   # sphere must enclose the box
    assert plan(R=float("nan")) == ARG and plan(R=float("inf")) == ARG
    assert plan(K=79) == ARG                               # periodic p = 8: 80 fitted columns
    assert plan(bc=1, K=80) == ARG                         # grounded p = 8: 81 columns
    assert plan(K=16385) == ARG
    assert plan(Q=11) == ARG                               # fewer surface points than the smallest rule
    assert plan(fib_F2=100) == ARG                         # not a Fibonacci number
    assert plan(precision=3) == ARG and plan(precision=-1) == ARG
    assert plan(far_field=2) == ARG
    # a sphere many box lengths across: more image shifts than a launch grid holds
    assert plan(box=D3(1e-4, 1.0, 1.0), R=1.0) == ARG      # 20001 x 3 x 3 shifts
    assert plan(box=D3(1e-12, 1.0, 1.0), R=1.0) == ARG
    assert out.value is None                               # no plan handed out

    # update, sharding, tuning and inspection calls without a plan
    parts = hsma.hsma_particles(0, None, None, 0)
    res = hsma.hsma_out()
    assert lib.hsma_energy_forces(None, ctypes.byref(parts), ctypes.byref(res)) == ARG
    e = (ctypes.c_double * 2)()
    off = (ctypes.c_int64 * 3)(0, 5, 9)
    assert lib.hsma_energy_forces_batched(None, 2, off, ctypes.byref(parts), e, None, None, None) == ARG
    cnt = ctypes.c_int64()
    assert lib.hsma_shard_near(None, ctypes.byref(parts), 0, 1, None, None, None, ctypes.byref(cnt), None) == ARG
    assert lib.hsma_shard_far(None, ctypes.byref(parts), None, None, None, 0, 0, 1, None, None, None, ctypes.byref(cnt),
                              None) == ARG
    tun = hsma.hsma_tuning(14, 48, 0.0)
    assert lib.hsma_plan_set_tuning(None, ctypes.byref(tun)) == ARG
    assert lib.hsma_plan_get_tuning(None, 2, off, ctypes.byref(tun)) == ARG
    assert lib.hsma_autotune(None, 2, off, ctypes.byref(parts), None, ctypes.byref(tun)) == ARG
    assert lib.hsma_plan_load_tuning(None, b"/nonexistent") == ARG
    sz = ctypes.c_size_t()
    assert lib.hsma_plan_footprint(None, 10, ctypes.byref(sz)) == ARG
    info = hsma.hsma_plan_info_t()
    assert lib.hsma_plan_get_info(None, ctypes.byref(info)) == ARG
    assert lib.hsma_plan_set_precision(None, 0) == ARG
    assert lib.hsma_plan_set_inset_skin(None, ctypes.c_double(0.05)) == ARG
    assert lib.hsma_plan_inset_stats(None, None, None, None) == ARG
    assert lib.hsma_plan_set_preemptible(None, 1) == ARG
    buf = (ctypes.c_double * 8)()
    assert lib.hsma_plan_get_matrix(None, 0, buf, 8) == ARG
    assert lib.hsma_last_timings(None, buf, 8) == ARG
    assert lib.hsma_last_get(None, 0, buf, 8) == ARG
    lib.hsma_plan_destroy(None)                            # a no-op

    # direct sums and the basis: sizes, precision, alignment
    src = (ctypes.c_double * 8)()
    tgt = (ctypes.c_double * 6)()
    pot = (ctypes.c_double * 2)()
    for fn in (lib.hsma_coulomb_sum, lib.hsma_coulomb_sum_static):
        assert fn(0, src, 2, tgt, pot, None, 1, None) == ARG
        assert fn(2, src, 0, tgt, pot, None, 1, None) == ARG
        assert fn(2, None, 2, tgt, pot, None, 1, None) == ARG
        assert fn(2, src, 2, tgt, None, None, 1, None) == ARG
        assert fn(2, src, 2, tgt, pot, None, 2, None) == ARG     # only FP64 or FP32 pair sums
        misaligned = ctypes.c_void_p(ctypes.addressof(src) + 4)
        assert fn(2, misaligned, 2, tgt, pot, None, 1, None) == ARG
    assert lib.hsma_coulomb_sum(1 << 32, src, 2, tgt, pot, None, 1, None) == ARG
    assert lib.hsma_coulomb_sum_static(1 << 32, src, 2, tgt, pot, None, 1, None) == CAP
    for prec in (0, 1):
        assert lib.hsma_basis(-1, 1.0, 2, tgt, buf, prec, None) == ARG
        assert lib.hsma_basis(41, 1.0, 2, tgt, buf, prec, None) == ARG
        assert lib.hsma_basis(4, 0.0, 2, tgt, buf, prec, None) == ARG
        assert lib.hsma_basis(4, 1.0, 0, tgt, buf, prec, None) == ARG
    assert lib.hsma_basis(4, 1.0, 2, tgt, buf, 2, None) == ARG        # FP64 or double-float only
    assert lib.hsma_fp32_peak(None, None) == ARG

    # serving: options and handles
    so = hsma.hsma_server_opts()
    assert lib.hsma_server_opts_default(ctypes.byref(so)) == 0
    assert so.max_batch == 64 and so.lanes == 2 and so.precision == hsma.FP32_ACC64
    srv = ctypes.c_void_p()
    assert so.mid_lanes == 0 and so.mid_max_n >= so.express_max_n
    for changes in ({"lanes": 0}, {"lanes": 17}, {"max_batch": 0}, {"max_batch": 65529}, {"mid_lanes": -1},
                    {"lanes": 2, "express_lanes": 1, "mid_lanes": 1},     # no bulk lane left
                    {"lanes": 3, "mid_lanes": 1, "mid_max_n": 1000}):     # medium below small
        o2 = hsma.hsma_server_opts()
        lib.hsma_server_opts_default(ctypes.byref(o2))
        for field, bad in changes.items():
            setattr(o2, field, bad)
        assert lib.hsma_server_create(ctypes.byref(srv), unit, 0, 8, 1.5, 2000, 600, ctypes.byref(o2)) == ARG
    assert srv.value is None
    t = ctypes.c_int64()
    assert lib.hsma_server_submit(None, 2, src, pot, ctypes.byref(t)) == ARG
    assert lib.hsma_server_cancel(None, 1) == ARG
    assert lib.hsma_server_stats(None, None) == ARG


def test_every_error_code_has_its_own_message(lib):
    from paper_1806_04801_gb300 import hsma
    msgs = [hsma.strerror(c) for c in range(-12, 1)]
    assert len(set(msgs)) == len(msgs)
    assert all(m != "unknown error" for m in msgs)
    assert hsma.strerror(-13) == "unknown error" and hsma.strerror(7) == "unknown error"
    assert "static scratch" in hsma.strerror(-11) and "memory budget" in hsma.strerror(-11)


def test_binding_checks_shapes_before_calling_the_library(lib):
    """The Python binding passes sizes to the C ABI that it derives from the
    arrays, so it checks them first: a mismatch raises ValueError before any
    library call (here on a plan object that holds no library handle)."""
    import torch
    from paper_1806_04801_gb300 import hsma
    plan = hsma.Plan.__new__(hsma.Plan)
    plan._h = None
    x5, q5 = np.zeros((5, 3)), np.zeros(5)
    with pytest.raises(ValueError, match="shape"):
        plan.energy_forces(np.zeros((4, 3)), q5)
    with pytest.raises(ValueError, match="shape"):
        plan.energy_forces(np.zeros((5, 2)), q5)
    with pytest.raises(ValueError, match="float64"):
        plan.energy_forces(x5.astype(np.float32), q5)
    with pytest.raises(ValueError, match="float64"):
        plan.energy_forces(torch.zeros((5, 3), dtype=torch.int64), torch.zeros(5, dtype=torch.int64))
    with pytest.raises(ValueError, match="contiguous"):
        plan.energy_forces(np.zeros((3, 5)).T, q5)
    # batched: the offsets must end where the arrays end
    with pytest.raises(ValueError, match=r"shape \(7, 3\)"):
        plan.energy_forces_batched(x5, q5, [0, 2, 7])
    with pytest.raises(ValueError, match="shape"):
        plan.energy_forces_batched(x5, np.zeros(4), [0, 2, 5])
    with pytest.raises(ValueError, match="entries"):
        plan.energy_forces_batched(x5, q5, [5])
    with pytest.raises(ValueError, match="offsets end at 4"):
        plan.autotune(x5, q5, [0, 4])
    with pytest.raises(ValueError, match="shape"):
        plan.shard_near(np.zeros((6, 3)), q5, 0, 2)
    # direct sums and the basis take (ns, 4) sources, (nt, 3) targets and points
    with pytest.raises(ValueError):
        hsma.coulomb_sum(np.zeros((4, 4)), np.zeros((2, 3)))        # host arrays
    del plan


def test_plan_dims_follow_the_readings_of_the_paper(lib):
    """hsma_plan_dims (host only) against the oracle's own, independently
    written rules: F2 from Q (the Fibonacci number whose N_o = 6(F2 + 1) is
    nearest to Q, ties to the larger; Sec. II.B), the image shells per axis
    (the smallest K with (K + 1/2) L_a >= Rs; Sec. II.A), the fitted columns
    and monitoring targets (periodic: n = 0 column dropped, points paired with
    their wrapped partners; Sec. II.A), and Delta r (Sec. III)."""
    import math
    import oracle
    from oracle import hsma as oh
    from paper_1806_04801_gb300 import hsma
    unit = (1.0, 1.0, 1.0)
    for Q in list(range(12, 400)) + [1000, 2000, 2268, 3600, 5928, 6000, 8000, 9588, 20000, 123456]:
        d = hsma.plan_dims(unit, hsma.PERIODIC, 8, 1.5, Q, 600)
        F2, F1 = oh.fib_from_points(Q)
        assert (d["F2"], d["F1"], d["n_images"]) == (F2, F1, 6 * (F2 + 1)), Q
    # the workloads' surface-point counts (reading of Q) and the paper's N_o = 5928
    assert [hsma.plan_dims(unit, 0, 8, 1.5, Q, 600)["F2"] for Q in (2000, 8000, 6000)] == [377, 1597, 987]
    assert hsma.plan_dims(unit, 0, 8, 1.5, 0, 600, fib_F2=987)["n_images"] == 5928
    with pytest.raises(hsma.HsmaError):
        hsma.plan_dims(unit, 0, 8, 1.5, 0, 600, fib_F2=988)
    for box, R in ((unit, 1.5), (unit, 2.0 * 0.5 * math.sqrt(3.0)), ((1.0, 1.3, 0.8), None), ((1.0, 1.0, 2.0), None),
                   ((2.0, 2.0, 2.0), 2.0 * math.sqrt(3.0)), (unit, 10.0)):
        R0 = 0.5 * math.sqrt(sum(b * b for b in box))
        R = math.sqrt(3.0) * R0 if R is None else R
        for bc in (hsma.PERIODIC, hsma.GROUNDED):
            d = hsma.plan_dims(box, bc, 10, R, 6000, 1500)
            shifts = 1
            for La in box:
                shifts *= 2 * oracle.num_shells(R, La) + 1
            assert d["n_shifts"] == shifts, (box, R)
            assert d["n_basis"] == 121 and d["n_cols"] == (120 if bc == hsma.PERIODIC else 121)
            assert d["n_mon_targets"] == (3000 if bc == hsma.PERIODIC else 1500) and d["Kmon"] == 1500
            assert d["dr"] == pytest.approx((1e-5 if bc == hsma.PERIODIC else 1e-4) * R, rel=1e-15)
            assert d["R0"] == pytest.approx(R0, rel=1e-15) and d["alpha"] == pytest.approx(R / R0, rel=1e-15)
            assert d["cond_estimate"] == 0.0
    assert hsma.plan_dims(unit, 0, 8, 1.5, 2000, 600)["n_shifts"] == 27      # 3 x 3 x 3 copies at Rs = 1.5 L
    assert hsma.plan_dims(unit, 0, 8, 1.5, 2000, 600, dr_rel=3e-6)["dr"] == pytest.approx(4.5e-6, rel=1e-15)
    assert hsma.plan_dims(unit, 0, 8, 1.5, 2000, 600, precision="fp32_tc")["precision"] == hsma.FP32_TC_FIT
    # the same argument checks as hsma_plan
    for args in (((1.0, 0.0, 1.0), 0, 8, 1.5, 2000, 600), (unit, 2, 8, 1.5, 2000, 600), (unit, 0, 41, 1.5, 2000, 600),
                 (unit, 0, 8, 0.8, 2000, 600), (unit, 0, 8, 1.5, 2000, 79), (unit, 0, 8, 1.5, 11, 600)):
        with pytest.raises(hsma.HsmaError):
            hsma.plan_dims(*args)


def test_binding_precision_names(lib):
    from paper_1806_04801_gb300 import hsma
    assert hsma.plan_dims((1.0, 1.0, 1.0), 0, 8, 1.5, 2000, 600, precision="fp64")["precision"] == hsma.FP64
    assert hsma.plan_dims((1.0, 1.0, 1.0), 0, 8, 1.5, 2000, 600, precision=2)["precision"] == hsma.FP32_TC_FIT
    with pytest.raises(ValueError, match="precision must be one of"):
        hsma.plan_dims((1.0, 1.0, 1.0), 0, 8, 1.5, 2000, 600, precision="fp16")


C_CLIENT = r"""
#include <stdio.h>
#include "hsma.h"
int main(void)
{
    hsma_opts o;
    double box[3] = {1.0, 1.0, 1.0};
    hsma_plan_info_t info;
    if (hsma_opts_default(&o) != HSMA_OK) return 1;
    if (hsma_plan_dims(box, HSMA_BC_PERIODIC, 12, 1.5, 8000, 2000, &o, &info) != HSMA_OK) return 2;
    if (hsma_plan(NULL, box, HSMA_BC_PERIODIC, 12, 1.5, 8000, 2000, &o) != HSMA_E_ARG) return 3;
    printf("%s|%d|%d|%d|%d|%s\n", hsma_version(), info.F2, info.n_images, info.n_shifts, info.n_cols,
           hsma_strerror(HSMA_E_NONNEUTRAL));
    return 0;
}
"""


@pytest.mark.parametrize("lang", ["c99", "c++17"])
def test_header_serves_plain_c_and_cpp_clients(lib, tmp_path, lang):
    """include/hsma.h compiles as pedantic C99 and as C++17 without warnings,
    and a client built from it links against libhsma.so and calls the
    host-only entry points (no device needed)."""
    import shutil
    import subprocess
    from paper_1806_04801_gb300 import hsma
    cc = shutil.which("gcc" if lang == "c99" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / ("client.c" if lang == "c99" else "client.cpp")
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(hsma.LIB_PATH)
    r = subprocess.run([cc, f"-std={lang}", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                        os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", libdir, "-lhsma",
                        f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stderr)
    version, F2, n_images, n_shifts, n_cols, msg = out.stdout.strip().split("|")
    assert "sm_103a" in version and (F2, n_images, n_shifts, n_cols) == ("1597", "9588", "27", "168")
    assert msg == "periodic system is not charge neutral"
