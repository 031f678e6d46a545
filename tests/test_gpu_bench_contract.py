"""bench.py keeps its output contract: one JSON line with the required keys,
a roofline object, the end-to-end figure, clock samples and the CPU
baseline -- checked on a short run of a reduced size."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_bench_json_line():
    r = _run("--n", "20000", "--steps", "3", "--warmup", "3", "--no-extras")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in r, k
    assert r["n_gpus"] == 1 and r["steps"] == 3 and r["warmup"] == 3 and r["higher_is_better"] is True
    assert r["value"] > 0 and abs(r["value"] - 1000.0 / r["ms_per_step"]) <= 1e-6 * r["value"]
    rf = r["roofline"]
    assert rf["bound"] == "alu" and 0 < rf["frac"] < 1.2 and abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-9
    assert r["e2e"]["h2d_bytes_per_step"] == 20000 * 32 and r["e2e"]["value"] > 0
    assert r["cpu_baseline"]["kind"] == "oracle" and r["cpu_baseline"]["cores"] >= 1
    assert r["gpu_launches"] >= 3 * 10
    assert r["accuracy"]["rel_energy_err"] <= 1e-6
    assert "workload" in r["config"]
    m = rf["measured_fp32"]
    assert m and 0 < m["packed_fma"] and 0 < m["scalar_fma"] <= 1.05 * rf["peak"]
    assert abs(m["frac_of_scalar_fma"] - rf["achieved"] / m["scalar_fma"]) < 1e-9


def test_fp32_peak_probe():
    """The measured FP32 FMA throughput lies between half and all of the
    count-based lane peak (SMs x 128 lanes x 2070 MHz): no probe can beat the
    lane count, and independent chains at 16 CTAs/SM cannot fall far short."""
    import torch
    from paper_1806_04801_gb300 import build, hsma
    build.build()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 128 * 2070e6
    sc, pk = hsma.fp32_peak()
    assert 0.5 * nominal < sc <= 1.02 * nominal, (sc, nominal)
    assert 0.5 * nominal < pk <= 1.02 * nominal, (pk, nominal)


def test_reference_arm_json_line():
    r = _run("--impl", "reference", "--steps", "1", "--warmup", "0")
    assert r["impl"] == "reference" and r["value"] > 0 and r["cpu_baseline"]["kind"] == "oracle"
    assert r["e2e"]["h2d_bytes_per_step"] == 0
