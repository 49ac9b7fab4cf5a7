"""bench.py on the host: the reference arm's JSON line (the FP64 oracle, the
one arm that runs without a GPU) and the product arm's refusal to run without
one (no CPU fallback)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, timeout=300):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_json_line():
    p = _bench("--impl", "reference", "--m", "600", "--n", "500", "--steps", "1", "--warmup", "1")
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["metric"] == "time-to-tolerance per CUR"
    assert out["unit"] == "ms" and out["value"] > 0 and out["higher_is_better"] is False
    assert out["steps"] == 1 and out["warmup"] == 1 and out["n_gpus"] == 1
    assert "600x500" in out["config"]["workload"]
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == out["value"] and cb["sample"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["h2d_bytes_per_step"] == 0
    assert e2e["d2h_bytes_per_step"] == 0


def test_product_arm_needs_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = _bench("--m", "64", "--n", "64", "--steps", "1", "--warmup", "1", timeout=120)
    assert p.returncode != 0
    assert not any(ln.startswith("{") for ln in p.stdout.splitlines())
