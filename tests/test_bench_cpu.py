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
           "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    r = json.loads(lines[0])
    assert r["impl"] == "reference" and r["value"] > 0 and r["unit"] == "systems/s"
    assert r["cpu_baseline"]["kind"] == "oracle" and r["e2e"]["h2d_bytes_per_step"] == 0
    assert r["config"]["N"] == 100_000
