"""The benchmark's JSON line: the reference arm (the CPU oracle; no GPU
needed) and, on a GPU, a short device-only run carry the keys the
measurement contract asks for."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COMMON = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
          "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def _line(args, timeout):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                       timeout=timeout, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _line(["--impl", "reference", "--steps", "1", "--warmup", "1"], 600)
    assert COMMON <= set(d), COMMON - set(d)
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


@pytest.mark.gpu
def test_device_run_line():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = _line(["--device-only", "--steps", "3", "--warmup", "3", "--no-cpu-baseline"], 900)
    assert {"roofline", "gpu_launches", "clocks", "tuning", "chain"} <= set(d)
    rf = d["roofline"]
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= set(rf)
    assert 0 < rf["frac"] < 2 and rf["unit"] == "GB/s"
    assert d["gpu_launches"] == 3 * 6
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["scaling"] == "weak"
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
