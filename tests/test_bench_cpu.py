"""bench.py's reference arm (the FP64 oracle on the host cores) launched the
way a multi-GPU job launches the benchmark: torchrun with two ranks on
127.0.0.1.  Rank 0 alone runs and prints one JSON line; the other rank exits
0 without work."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_under_torchrun_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "0", "--particles", "3000"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    r = json.loads(lines[0])
    assert r["impl"] == "reference" and r["value"] > 0 and r["unit"] == "systems/s"
    assert r["cpu_baseline"]["kind"] == "oracle" and r["e2e"]["h2d_bytes_per_step"] == 0
    assert r["config"]["N"] == 3000
    # complete oracle steps, each timed (as many of the requested as fit the time budget)
    assert 1 <= r["steps"] <= 2 and len(r["step_s"]) == r["steps"] and r["steps_requested"] == 2
    assert abs(r["ms_per_step"] - 1000.0 * sum(r["step_s"]) / r["steps"]) < 1e-6


def test_clock_sampler_reads_clocks_and_throttle_reasons(tmp_path):
    """bench.py's clock record: median SM clock under load, the maximum, and
    the throttle reasons seen, parsed from nvidia-smi's noheader/nounits CSV
    rows (as sampled during the timed region)."""
    sys.path.insert(0, ROOT)
    import bench

    class _Done:  # stands in for the finished nvidia-smi process
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    rows = [
        "0, 2070, 2070, 812.40, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.02, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1201.75, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler()
    cs.path, cs.proc = str(path), _Done()
    r = cs.stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["power_w_max"] == 1390.02
    assert r["reasons"] == ["sw_power_cap"]
    assert not path.exists()  # the temporary record is removed
    path.write_text("0, 1400, 2070, 700.0, 0x0000000000000040, Not Active, Active, Not Active, Not Active\n")
    cs.path, cs.proc = str(path), _Done()
    assert cs.stop()["reasons"] == ["hw_thermal_slowdown"]
    assert bench.ClockSampler().stop()["reasons"] == ["nvidia-smi unavailable"]


def test_profile_commands_parse_with_the_current_bench(monkeypatch):
    """Every bench.py command quoted in profiles/ (the commands the ncu
    summaries were made with) still parses with bench.py's options, and
    names only files that are in the repository."""
    import glob
    import re
    import shlex
    sys.path.insert(0, ROOT)
    import bench
    cmds = []
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read().replace("\\\n", " ")
        for m in re.finditer(r"python (bench\.py[^\n]*)", text):
            cmds.append((os.path.basename(path), shlex.split(m.group(1))))
    assert len(cmds) >= 6
    for name, argv in cmds:
        assert os.path.exists(os.path.join(ROOT, argv[0])), (name, argv[0])
        monkeypatch.setattr(sys, "argv", argv)
        args = bench.parse()  # exits (SystemExit) on an unknown option
        if args.tuning:
            v, i = bench.fixed_tuning(args)
            assert v in (2, 4, 5, 12, 13, 14, 15, 16, 17) and i >= 1, (name, args.tuning)


def test_clock_sampler_keeps_the_timed_region(tmp_path):
    """With nvidia-smi's timestamp column, only samples inside the timed
    region's host-time window enter the median."""
    import datetime
    sys.path.insert(0, ROOT)
    import bench

    class _Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    t0 = 1_800_000_000.0
    stamp = lambda t: datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]  # noqa: E731
    rows = [f"{stamp(t0 - 1.0)}, 0, 1200, 2070, 200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            f"{stamp(t0 + 0.2)}, 0, 1965, 2070, 1300.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            f"{stamp(t0 + 0.4)}, 0, 1980, 2070, 1310.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            f"{stamp(t0 + 5.0)}, 0, 1100, 2070, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler()
    cs.path, cs.proc = str(path), _Done()
    r = cs.stop(window=(t0, t0 + 1.0))
    assert r["samples"] == 2 and r["samples_in_timed_region"] and r["sm_mhz"] == 1972.5
