"""bench.py on a host without a GPU: the reference arm (the oracle timed on
the host cores) prints its JSON line with the contract's keys, and the fused
arm refuses to run instead of falling back to the CPU."""
import json
import os
import subprocess
import sys

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, timeout=300):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                          text=True, timeout=timeout)


def test_reference_arm_prints_contract_line():
    r = run_bench("--impl", "reference", "--steps", "1", "--warmup", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU refusal")
def test_fused_arm_refuses_without_a_gpu():
    r = run_bench("--steps", "1", "--warmup", "3", timeout=120)
    assert r.returncode != 0
    assert "GPU" in (r.stderr + r.stdout)


def test_cpu_baseline_reports_cores_and_single_thread():
    """The oracle baseline that the fused lines carry: its thread count, a
    bounded sample, and the one-thread rate beside it."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2603_02804_gb300 import workloads
    r = bench.cpu_baseline(workloads.WORKLOADS["hea12"], 2.0, 2)
    assert r["kind"] == "oracle" and r["cores"] == 2 and r["value"] > 0 and r["unit"] == "samples/s"
    assert "of the 256 samples of the hea12 workload" in r["sample"]
    st = r["single_thread"]
    assert st["value"] > 0 and st["unit"] == "samples/s" and "one thread" in st["sample"]
    assert abs(st["speedup_on_cores"] - r["value"] / st["value"]) < 1e-12
