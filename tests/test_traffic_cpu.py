"""Host-side pieces of the measurement: the planner places a multi-pass
plan's checkpoints at pass outputs (so the adjoint re-anchors without a
load), the benchmark's algorithmic byte count per adjoint launch follows the
exported plan, and a recorded DRAM-traffic figure is parsed from an ncu CSV
and reported only for the kernel sources it was captured on. No GPU."""
import importlib.util
import json
import os

import pytest

from paper_2603_02804_gb300 import build as qbuild
from paper_2603_02804_gb300 import qfuse
from paper_2603_02804_gb300 import record_traffic as rt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    qbuild.build()
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def plan(n, d, c, B=4):
    h = qfuse.qf_hea_create(n, d)
    qfuse.qf_plan(h, B, ckpt_layers=c, host_only=True)
    return h


def headers(h, direction):
    w = [int(v) for v in qfuse.qf_plan_export(h, direction)]
    n_pass, i = w[2], 3
    heads = []
    for _ in range(n_pass):
        heads.append(dict(zip(("op_begin", "op_end", "psi_src", "psi_dst", "lam_src", "lam_dst"), w[i:i + 6])))
        i += 11 + 32
    n_ops = w[i]
    codes = [w[i + 1 + 2 * k] & 15 for k in range(n_ops)]
    return heads, codes


@pytest.mark.parametrize("n,d,c,none_mid", [(20, 40, 4, True), (20, 12, 2, True), (16, 100, 10, True),
                                              (16, 30, 4, False), (14, 20, 3, False)])
def test_multi_pass_checkpoints_are_pass_outputs(n, d, c, none_mid):
    """A checkpoint boundary that falls inside a pass (not the last) moves to
    that pass's output; only a pass that crosses several boundaries keeps the
    earlier ones after their steps, and the last pass keeps its own (its
    output is psi_M). Plans whose passes span less than c layers (the large
    workload's family) have no mid-pass checkpoint and no re-anchor load."""
    h = plan(n, d, c)
    try:
        info = qfuse.qf_plan_info(h)
        assert info["n_passes"] > 1 and info["n_ckpt"] > 2
        fwd, fcodes = headers(h, 0)
        bwd, bcodes = headers(h, 1)
        for pi, f in enumerate(fwd[:-1]):
            if 6 in fcodes[f["op_begin"]:f["op_end"]]:
                assert f["psi_dst"] >= 0, pi   # crossed several boundaries: the last is the output
        if none_mid:
            assert 6 not in fcodes and 7 not in bcodes
            assert len([p for p in fwd[:-1] if p["psi_dst"] >= 0]) == info["n_ckpt"] - 1
        # adjoint passes that start from a stored state write no psi back
        for b, f in zip(bwd, reversed(fwd)):
            assert b["psi_src"] == (f["psi_dst"] if f["psi_dst"] >= 0 else -2)
            if f["psi_src"] >= 0:
                assert b["psi_dst"] == -3
    finally:
        qfuse.qf_circuit_destroy(h)


def test_single_pass_plan_keeps_step_checkpoints():
    h = plan(12, 20, 10)
    try:
        assert qfuse.qf_plan_info(h)["n_passes"] == 1
        _, fcodes = headers(h, 0)
        _, bcodes = headers(h, 1)
        assert fcodes.count(6) == 1 and bcodes.count(7) == 1
    finally:
        qfuse.qf_circuit_destroy(h)


def test_adjoint_bytes_follow_the_plan(bench):
    h = plan(12, 20, 10)
    try:
        # one pass: psi_M in, lambda seeded from it, nothing written, one re-anchor
        assert bench.adjoint_bytes_per_amp(h) == (16.0, 1)
    finally:
        qfuse.qf_circuit_destroy(h)
    h = plan(20, 40, 4)
    try:
        bpa, passes = bench.adjoint_bytes_per_amp(h)
        bwd, _ = headers(h, 1)
        n_from_slot = sum(1 for p in bwd if p["psi_dst"] == -3) - 1  # the last pass writes nothing either
        expect = (8 * passes                 # psi in
                  + 8 * (passes - 1)         # lambda in (the first pass seeds it)
                  + 8 * (passes - 1 - n_from_slot)   # psi out
                  + 8 * (passes - 1)) / passes       # lambda out
        assert passes == 21 and abs(bpa - expect) < 1e-12
        assert 24 < bpa < 32
    finally:
        qfuse.qf_circuit_destroy(h)


def _csv(path, rows):
    hdr = '"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n'
    with open(path, "w") as f:
        f.write("==PROF== noise line\n")
        f.write(hdr)
        for r in rows:
            f.write(",".join('"%s"' % v for v in r) + "\n")


def test_launch_bytes_parse_units(tmp_path):
    p = str(tmp_path / "t.csv")
    _csv(p, [(0, "k", "dram__bytes_read.sum", "byte", "1,000"), (0, "k", "dram__bytes_write.sum", "Kbyte", "2"),
             (0, "k", "gpu__time_duration.sum", "usecond", "5"),
             (1, "k", "dram__bytes_read.sum", "Mbyte", "1.5"), (1, "k", "dram__bytes_write.sum", "byte", "0")])
    assert rt.launch_bytes(p) == [3000.0, 1.5e6]


def test_measured_traffic_is_gated_by_the_sources_hash(bench, tmp_path, monkeypatch):
    table = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(table))
    assert bench.measured_traffic("hea20", 100)[0] is None
    table.write_text(json.dumps({"hea20": {"bytes_per_amp": 26.5, "case": "c", "sources_sha": rt.sources_sha()}}))
    assert bench.measured_traffic("hea20", 100) == (2650.0, "c")
    assert bench.measured_traffic("hea12", 100)[0] is None
    table.write_text(json.dumps({"hea20": {"bytes_per_amp": 26.5, "case": "c", "sources_sha": "stale"}}))
    v, note = bench.measured_traffic("hea20", 100)
    assert v is None and "changed" in note
