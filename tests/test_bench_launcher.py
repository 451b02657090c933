"""bench.py's multi-rank launch on CPU (gloo): with --gpus N and no torchrun
environment it starts N ranks of itself under torch.distributed.run; every
rank joins the barrier and the max-over-ranks reduction, and rank 0 prints
one line with the world size.  --gpus 1 runs in the calling process."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*argv):
    env = {k: v for k, v in os.environ.items()
           if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *argv], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=240)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("n", [1, 2, 3])
def test_launcher_starts_n_ranks_and_reduces_the_max(n):
    out = _run("--gpus", str(n), "--check-launcher")
    assert out["n_gpus"] == n
    assert out["max_ms"] == float(n)   # rank r reports 1 + r


def test_gpus_must_agree_with_a_torchrun_environment():
    env = dict(os.environ, WORLD_SIZE="2", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "4",
                        "--check-launcher"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode != 0 and "disagrees" in (r.stderr + r.stdout)


def test_reference_arm_prints_its_line():
    """bench.py --impl reference times the oracle on the host cores and
    prints the reference line (no GPU needed)."""
    out = _run("--impl", "reference", "--steps", "1", "--warmup", "0")
    assert out["impl"] == "reference" and out["value"] > 0
    assert out["unit"] == "Gvoxel-angle/s" and out["higher_is_better"] is True
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["cores"] >= 1
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["value"] == out["value"]


def test_roofline_traffic_comes_from_the_committed_profiles():
    """The DRAM bytes per launch that the benchmark line reports beside its
    roofline are the ncu figures recorded in profiles/traffic.txt: the
    z-first polarisation + z-FFT launch at 1024 x 1024 x 128 (its dominant
    kernel), and nothing for a kernel whose capture is no longer current."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench._traffic_from_profiles("p1-1024", "zfirst-pol_fftx", 32) == 29215200000.0
    assert bench._traffic_from_profiles("p1-1024", "zfirst-fftx", 32) is None
    assert bench._traffic_from_profiles("p1-1024", "zfirst-pol_fftx", 64) is None
