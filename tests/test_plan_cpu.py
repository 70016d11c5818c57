"""Host-side checks of the library: exported symbols, argument checking and
the fusion planner (via a complex128 interpreter of the exported programs,
compared with the oracle). No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2603_02804_gb300 import build as qbuild
from paper_2603_02804_gb300 import qfuse
from tests import plan_interp as pi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    qbuild.build()
    return qfuse.load()


def header_symbols():
    src = open(os.path.join(ROOT, "include", "qfuse.h")).read()
    return sorted(set(re.findall(r"^\s*(?:qf_status|const char\*|int32_t|double)\s+(qf_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol(lib):
    syms = header_symbols()
    assert len(syms) >= 14
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(qfuse.SIGNATURES), "binding and header must declare the same entry points"


def test_version_and_error_string(lib):
    assert qfuse.qf_version() >= 100
    with pytest.raises(qfuse.QFError) as e:
        qfuse.qf_hea_create(0, 3)
    assert e.value.status == qfuse.QF_ERR_INVALID_ARG
    assert "n_qubits" in qfuse.qf_last_error()


@pytest.mark.parametrize("bad", [
    dict(n=31, d=2), dict(n=4, d=-1),
])
def test_hea_create_rejects(bad):
    with pytest.raises(qfuse.QFError):
        qfuse.qf_hea_create(bad["n"], bad["d"])


def test_circuit_create_rejects_bad_gates():
    with pytest.raises(qfuse.QFError):
        qfuse.qf_circuit_create(3, [(qfuse.QF_GATE_RY, 3, -1, 0)], 1)   # qubit out of range
    with pytest.raises(qfuse.QFError):
        qfuse.qf_circuit_create(3, [(qfuse.QF_GATE_RY, 0, -1, 5)], 1)   # param out of range
    with pytest.raises(qfuse.QFError):
        qfuse.qf_circuit_create(3, [(qfuse.QF_GATE_CZ, 1, 1, -1)], 0)   # CZ on one qubit
    with pytest.raises(qfuse.QFError):
        qfuse.qf_circuit_create(3, [(7, 0, -1, 0)], 1)                   # unknown kind


def test_plan_rejects_bad_options():
    h = qfuse.qf_hea_create(5, 2)
    try:
        for kw in (dict(tile_bits=3), dict(tile_bits=13), dict(path=5), dict(ckpt_layers=-1)):
            with pytest.raises(qfuse.QFError):
                qfuse.qf_plan(h, 4, host_only=True, **kw)
        with pytest.raises(qfuse.QFError):
            qfuse.qf_plan(h, -1, host_only=True)
    finally:
        qfuse.qf_circuit_destroy(h)


def test_host_only_plan_refuses_device_calls():
    h = qfuse.qf_hea_create(5, 2)
    try:
        ws = qfuse.qf_plan(h, 4, host_only=True)
        assert ws > 0
        with pytest.raises(qfuse.QFError) as e:
            qfuse.qf_forward(h, 0, 0, 4, qfuse.pauli("Z", 5), 0, 0, ws)
        assert e.value.status in (qfuse.QF_ERR_WORKSPACE, qfuse.QF_ERR_INVALID_ARG)
    finally:
        qfuse.qf_circuit_destroy(h)


def interp_check(handle, n, theta, x, obs, slot_param, slot_kind, tol=1e-10, oracle_circ=None, kernel_order=False):
    info = qfuse.qf_plan_info(handle)
    n_eff = info["n_eff"]
    fwd = pi.parse(qfuse.qf_plan_export(handle, 0))
    bwd = pi.parse(qfuse.qf_plan_export(handle, 1))
    # every rotation gate appears exactly once in the fused forward entries
    entries = sorted((k, p) for run in fwd.fused for (k, p, _) in run)
    expect = sorted(zip(slot_kind, slot_param))
    assert entries == expect
    # and exactly once in the gradient terms
    assert sorted(p for _, ps in bwd.terms for p in ps) == sorted(slot_param)
    pq = qfuse.pauli(obs, n)
    gp, Ep = orc.gradient(oracle_circ, theta, x, obs, per_sample=True)
    for b in range(len(x)):
        E, slots = pi.run_forward(fwd, n, n_eff, theta, x[b], pq.x_mask, pq.z_mask, kernel_order)
        assert abs(E - Ep[b]) < tol
        g = pi.run_backward(bwd, n_eff, theta, slots, pq.x_mask, pq.z_mask, 1.0, len(theta), kernel_order)
        assert np.max(np.abs(g - gp[b])) < tol
    return info, fwd.rounds_mode


@pytest.mark.parametrize("program", [0, 1])
@pytest.mark.parametrize("n,d,K,ck", [
    (1, 2, 0, 0), (3, 3, 0, 0), (4, 2, 0, 0), (5, 3, 0, 1), (6, 4, 0, 2), (7, 3, 0, 1), (8, 3, 0, 0),
    (10, 3, 0, 1), (12, 2, 0, 1), (13, 2, 0, 1), (14, 3, 8, 1), (9, 4, 6, 2), (11, 2, 5, 0),
    (15, 4, 7, 1), (17, 3, 0, 1),
])
def test_fused_plan_matches_oracle_hea(n, d, K, ck, program):
    rng = np.random.default_rng(1000 + 37 * n + d)
    h = qfuse.qf_hea_create(n, d)
    try:
        qfuse.qf_plan(h, 2, tile_bits=K, ckpt_layers=ck, host_only=True, program=program)
        theta = rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32).astype(np.float64)
        x = rng.uniform(0, np.pi, (2, n)).astype(np.float32).astype(np.float64)
        c = orc.hea(n, d)
        obs = "Z" if n < 3 else "ZXY"[: min(3, n)]
        P = 3 * n * d
        slot_param = list(range(P))
        slot_kind = [orc.RY if (p % 3) == 1 else orc.RZ for p in range(P)]
        info, rounds = interp_check(h, n, theta, x, obs, slot_param, slot_kind, oracle_circ=c)
        if n <= 12 and K == 0:
            assert info["n_passes"] == 1
        assert rounds == (program == 0 and info["tile_bits"] >= 7)
    finally:
        qfuse.qf_circuit_destroy(h)


@pytest.mark.parametrize("seed", range(4))
def test_fused_plan_matches_oracle_random_gate_list(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 9))
    rows, kinds = [], [orc.RX, orc.RY, orc.RZ, orc.CZ]
    n_params = 7
    for _ in range(40):
        k = int(rng.choice(kinds))
        if k == orc.CZ:
            a, b = rng.choice(n, 2, replace=False)
            rows.append((k, int(a), int(b), -1))
        else:
            rows.append((k, int(rng.integers(n)), -1, int(rng.integers(n_params))))
    h = qfuse.qf_circuit_create(n, rows, n_params)
    try:
        qfuse.qf_plan(h, 3, tile_bits=int(rng.choice([0, 4, 5])), ckpt_layers=1, host_only=True)
        theta = rng.uniform(0, 2 * np.pi, n_params).astype(np.float32).astype(np.float64)
        x = rng.uniform(0, np.pi, (3, n)).astype(np.float32).astype(np.float64)
        c = orc.Circuit(n=n, gates=np.array(rows, np.int32), n_params=n_params)
        slot_param = [r[3] for r in rows if r[0] != orc.CZ]
        slot_kind = [r[0] for r in rows if r[0] != orc.CZ]
        obs = "".join(rng.choice(list("IZ"), size=n))
        interp_check(h, n, theta, x, obs, slot_param, slot_kind, oracle_circ=c)
    finally:
        qfuse.qf_circuit_destroy(h)


def test_plan_statistics_for_benchmark_shapes():
    """Planner shape on the benchmark circuits: n = 12 is one pass (whole state
    in one CTA); n = 16 and n = 20 stream tiles with a few passes per layer."""
    out = {}
    for n, d in ((12, 20), (16, 100), (20, 50)):
        h = qfuse.qf_hea_create(n, d)
        try:
            qfuse.qf_plan(h, 1, ckpt_layers=10, host_only=True)
            out[n] = qfuse.qf_plan_info(h)
        finally:
            qfuse.qf_circuit_destroy(h)
    assert out[12]["n_passes"] == 1
    # about one fused 2x2 per qubit and layer (RZ RY RZ -> one op)
    assert 12 * 20 <= out[12]["n_fused_ops"] <= 12 * 22
    assert out[12]["n_steps"] <= 2 * 20
    # round programs: group-level light-cone staircases, so a pass over HBM
    # covers about 2 layers at n = 16 and 1 layer at n = 20 with full rounds
    assert out[16]["n_passes"] <= 0.6 * 100
    assert out[20]["n_passes"] <= 1.1 * 50
    for n, d in ((12, 20), (16, 100), (20, 50)):
        h = qfuse.qf_hea_create(n, d)
        try:
            qfuse.qf_plan(h, 1, ckpt_layers=10, host_only=True)
            prog = pi.parse(qfuse.qf_plan_export(h, 0))
            assert prog.rounds_mode
            words = prog.round_words
            W = pi.FWD_ROUND_WORDS
            pads = sum(1 for k in range(len(words) // W) for r in range(4) if words[W * k + r] == 0)
            assert pads == 0, (n, pads)
        finally:
            qfuse.qf_circuit_destroy(h)


# Memory-saving mode: each stored pass output is rounded once to bfloat16
# (relative 2^-9 per component); a gradient term sees one such rounding of
# psi. Measured ~1e-4 on these shapes; the bound leaves 20x room.
BF16_GRAD_TOL = 2e-3


@pytest.mark.parametrize("mem_save", [False, True])
@pytest.mark.parametrize("program", [0, 1])
@pytest.mark.parametrize("n,d,K,ck", [
    (6, 4, 0, 1), (12, 4, 0, 1), (12, 3, 0, 2), (13, 3, 0, 1), (14, 3, 8, 1), (17, 3, 0, 1), (9, 4, 6, 2),
    (11, 2, 5, 0),
])
def test_mode_a_schedule_matches_oracle(n, d, K, ck, program, mem_save):
    """Checkpoint mode A (per-block forward re-run storing pass outputs, each
    adjoint pass starting from the stored output of the forward pass it
    undoes): the exported launch list, executed on whole complex128 vectors,
    gives the oracle's gradient; every gradient term is visited once."""
    rng = np.random.default_rng(7000 + 37 * n + d)
    h = qfuse.qf_hea_create(n, d)
    try:
        qfuse.qf_plan(h, 2, tile_bits=K, ckpt_layers=ck, host_only=True, program=program, ckpt_mode=1,
                      mem_save=mem_save)
        info = qfuse.qf_plan_info(h)
        assert info["ckpt_mode"] == 1 and info["mem_save"] == int(mem_save)
        n_eff = info["n_eff"]
        fwd = pi.parse(qfuse.qf_plan_export(h, 0))
        bwd = pi.parse(qfuse.qf_plan_export(h, 1))
        sched = pi.parse_schedule(qfuse.qf_plan_export(h, 2))
        assert info["launches_bwd"] == len(sched) + 2
        # no adjoint launch writes psi back; pass-output slots stay within the plan's count
        for s in sched:
            if s["dir"] == 1:
                assert s["psi_dst"] == pi.BUF_NONE
            h_dst = s["flags"] & pi.PF_DST_H
            if s["dir"] == 0:
                idx = s["psi_dst"] if h_dst else s["psi_dst"] - info["n_ckpt"]
                assert 0 <= idx < info["n_pass_slots"]
        theta = rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32).astype(np.float64)
        x = rng.uniform(0, np.pi, (2, n)).astype(np.float32).astype(np.float64)
        obs = "Z" if n < 3 else "ZXY"[: min(3, n)]
        pq = qfuse.pauli(obs, n)
        gp, Ep = orc.gradient(orc.hea(n, d), theta, x, obs, per_sample=True)
        tol = BF16_GRAD_TOL if mem_save else 1e-10
        for b in range(len(x)):
            E, slots = pi.run_forward(fwd, n, n_eff, theta, x[b], pq.x_mask, pq.z_mask)
            assert abs(E - Ep[b]) < 1e-10
            g = pi.run_backward_mode_a(fwd, bwd, sched, n, n_eff, theta, x[b], slots, pq.x_mask, pq.z_mask,
                                       1.0, len(theta))
            assert np.max(np.abs(g - gp[b])) < tol
            if mem_save and info["n_pass_slots"] > 0 and info["n_passes"] > 1:
                assert np.max(np.abs(g - gp[b])) > 1e-9  # the rounding is really there
    finally:
        qfuse.qf_circuit_destroy(h)


def test_mode_a_memory_and_options():
    """Mode A stores p*c pass outputs of one block on top of the checkpoints;
    the memory-saving mode stores them at half the bytes; mem_save without
    mode A and mode A on the per-gate path are refused."""
    n, d, B = 16, 40, 4
    h = qfuse.qf_hea_create(n, d)
    try:
        ws_b = qfuse.qf_plan(h, B, ckpt_layers=10, host_only=True)
        ws_a = qfuse.qf_plan(h, B, ckpt_layers=10, host_only=True, ckpt_mode=1)
        ia = qfuse.qf_plan_info(h)
        ws_h = qfuse.qf_plan(h, B, ckpt_layers=10, host_only=True, ckpt_mode=1, mem_save=True)
        ih = qfuse.qf_plan_info(h)
        st = ia["state_bytes"]
        assert ia["n_pass_slots"] >= 1 and ih["n_pass_slots"] == ia["n_pass_slots"]
        assert ws_a - ws_b == ia["n_pass_slots"] * st
        assert ws_h - ws_b == ia["n_pass_slots"] * st // 2
        with pytest.raises(qfuse.QFError):
            qfuse.qf_plan(h, B, host_only=True, mem_save=True)
        with pytest.raises(qfuse.QFError):
            qfuse.qf_plan(h, B, host_only=True, ckpt_mode=2)
        with pytest.raises(qfuse.QFError):
            qfuse.qf_plan(h, B, host_only=True, path=qfuse.QF_PATH_PER_GATE, ckpt_mode=1)
        with pytest.raises(qfuse.QFError):
            qfuse.qf_plan_export(h, 3)
        qfuse.qf_plan(h, B, ckpt_layers=10, host_only=True)
        with pytest.raises(qfuse.QFError):
            qfuse.qf_plan_export(h, 2)
    finally:
        qfuse.qf_circuit_destroy(h)


def test_mode_a_fit_minimises_the_workspace():
    """qf_plan_fit in mode A takes the checkpoint interval with the smallest
    workspace (about sqrt(d / p) layers, Eq. 8), not the smallest interval."""
    n, d, B = 16, 64, 2
    h = qfuse.qf_hea_create(n, d)
    try:
        c, ws = qfuse.qf_plan_fit(h, B, 1 << 40, host_only=True, ckpt_mode=1)
        sizes = {cl: qfuse.qf_plan(h, B, ckpt_layers=cl, host_only=True, ckpt_mode=1) for cl in range(1, d + 1)}
        assert ws == sizes[c] == min(sizes.values())
        assert 1 < c < d
        with pytest.raises(qfuse.QFError):
            qfuse.qf_plan_fit(h, B, min(sizes.values()) - 1, host_only=True, ckpt_mode=1)
    finally:
        qfuse.qf_circuit_destroy(h)


def test_tc_path_options():
    """The tensor-core path needs round programs on 12-qubit tiles."""
    h = qfuse.qf_hea_create(8, 3)
    try:
        with pytest.raises(qfuse.QFError) as e:
            qfuse.qf_plan(h, 2, host_only=True, tc_path=True)
        assert e.value.status == qfuse.QF_ERR_UNSUPPORTED
    finally:
        qfuse.qf_circuit_destroy(h)
    h = qfuse.qf_hea_create(12, 3)
    try:
        ws0 = qfuse.qf_plan(h, 2, host_only=True)
        ws1 = qfuse.qf_plan(h, 2, host_only=True, tc_path=True)
        info = qfuse.qf_plan_info(h)
        assert info["tc_path"] == 1 and ws1 > ws0
        assert info["launches_fwd"] == info["n_passes"] + 3
        with pytest.raises(qfuse.QFError):
            qfuse.qf_plan(h, 2, host_only=True, tc_path=True, program=1)
        with pytest.raises(qfuse.QFError):
            qfuse.qf_plan(h, 2, host_only=True, tc_path=True, path=qfuse.QF_PATH_PER_GATE)
    finally:
        qfuse.qf_circuit_destroy(h)


def test_encoding_argument_and_input_sizes():
    """QF_ENC_STATE_IN takes complex64 [B][2^n] states: the host-buffer staging
    grows accordingly; unknown encodings are refused."""
    h0 = qfuse.qf_hea_create(10, 2)
    h1 = qfuse.qf_hea_create(10, 2, qfuse.QF_ENT_CHAIN, qfuse.QF_ENC_STATE_IN)
    try:
        ws0 = qfuse.qf_plan(h0, 4, host_only=True)
        ws1 = qfuse.qf_plan(h1, 4, host_only=True)
        assert ws1 - ws0 >= 4 * (1 << 10) * 8 - 4 * 10 * 4 - 256
        with pytest.raises(qfuse.QFError):
            qfuse.qf_hea_create(10, 2, qfuse.QF_ENT_CHAIN, 7)
        with pytest.raises(qfuse.QFError):
            qfuse.qf_circuit_create(3, [(qfuse.QF_GATE_RY, 0, -1, 0)], 1, 5)
    finally:
        qfuse.qf_circuit_destroy(h0)
        qfuse.qf_circuit_destroy(h1)


def test_xyz_ring_ansatz_rows():
    from paper_2603_02804_gb300 import workloads
    rows = workloads.xyz_ring_gates(5, 2)
    assert len(rows) == 2 * (15 + 5)
    assert rows[:3] == [(0, 0, -1, 0), (1, 0, -1, 1), (2, 0, -1, 2)]
    assert rows[15:20] == [(3, 0, 1, -1), (3, 1, 2, -1), (3, 2, 3, -1), (3, 3, 4, -1), (3, 4, 0, -1)]
    assert workloads.ixyz(6) == "IXYZIX"


@pytest.mark.parametrize("program", [0, 1])
@pytest.mark.parametrize("n,d,K,ck", [(5, 2, 0, 0), (7, 3, 0, 1), (9, 2, 0, 0), (13, 2, 0, 1), (14, 2, 8, 1),
                                      (17, 2, 0, 0)])
def test_xyz_ring_ansatz_plans_match_oracle(n, d, K, ck, program):
    """The paper's Rx, Ry, Rz + CZ-ring ansatz: round programs (RX items, the
    ring's CZ(n-1, 0) as link n-1) and generic programs both give the
    oracle's expectations and gradients."""
    from paper_2603_02804_gb300 import workloads
    rng = np.random.default_rng(900 + 7 * n + d)
    rows = workloads.xyz_ring_gates(n, d)
    P = 3 * n * d
    h = qfuse.qf_circuit_create(n, rows, P)
    try:
        qfuse.qf_plan(h, 2, tile_bits=K, ckpt_layers=ck, host_only=True, program=program)
        theta = rng.uniform(0, 2 * np.pi, P).astype(np.float32).astype(np.float64)
        x = rng.uniform(0, np.pi, (2, n)).astype(np.float32).astype(np.float64)
        c = orc.Circuit(n=n, gates=np.array(rows, np.int32), n_params=P)
        slot_param = [r[3] for r in rows if r[0] != orc.CZ]
        slot_kind = [r[0] for r in rows if r[0] != orc.CZ]
        info, rounds = interp_check(h, n, theta, x, "ZXY"[: min(3, n)], slot_param, slot_kind, oracle_circ=c)
        assert rounds == (program == 0 and info["tile_bits"] >= 7)
    finally:
        qfuse.qf_circuit_destroy(h)


@pytest.mark.parametrize("kind,n,d,K,ck", [
    ("hea", 7, 3, 0, 1), ("hea", 9, 4, 0, 2), ("hea", 12, 3, 0, 1), ("hea", 13, 3, 0, 1), ("hea", 15, 3, 7, 1),
    ("hea", 17, 2, 0, 0), ("ring", 9, 2, 0, 0), ("ring", 14, 2, 8, 1), ("sweep", 9, 5, 0, 0),
    ("sweep", 13, 4, 0, 1),
])
def test_round_programs_in_kernel_order_match_oracle(kind, n, d, K, ck):
    """Round programs executed the way the round kernels execute them (the
    interpreter's kernel order): per round the rotations from the rotation
    terms, then one diagonal built from the RZ-run terms' summed angles per
    register index with the register-register CZ signs, then the other links;
    the adjoint takes the four RZ-run terms at the diagonal from
    Im(conj(lambda) psi) before any rotation of the round. Expectations and
    gradients must equal the oracle's, which pins the merged diagonal's
    algebra (signs, direction, the links it absorbs) without a GPU."""
    from paper_2603_02804_gb300 import workloads
    rng = np.random.default_rng(1300 + 11 * n + d)
    if kind == "hea":
        rows = None
        h = qfuse.qf_hea_create(n, d)
        P = 3 * n * d
        c = orc.hea(n, d)
        slot_param = list(range(P))
        slot_kind = [orc.RY if (p % 3) == 1 else orc.RZ for p in range(P)]
    else:
        # the Rx,Ry,Rz + CZ ring ansatz, or the fusion-depth circuit (d consecutive
        # Rx,Ry,Rz gates per qubit, no entangler)
        rows = workloads.xyz_ring_gates(n, d) if kind == "ring" else workloads.consecutive_gates(n, d)
        P = 3 * n * d if kind == "ring" else n * d
        h = qfuse.qf_circuit_create(n, rows, P)
        c = orc.Circuit(n=n, gates=np.array(rows, np.int32), n_params=P)
        slot_param = [r[3] for r in rows if r[0] != orc.CZ]
        slot_kind = [r[0] for r in rows if r[0] != orc.CZ]
    try:
        qfuse.qf_plan(h, 2, tile_bits=K, ckpt_layers=ck, host_only=True, program=0)
        theta = rng.uniform(0, 2 * np.pi, P).astype(np.float32).astype(np.float64)
        x = rng.uniform(0, np.pi, (2, n)).astype(np.float32).astype(np.float64)
        info, rounds = interp_check(h, n, theta, x, "ZXY"[: min(3, n)], slot_param, slot_kind, oracle_circ=c,
                                    kernel_order=True)
        assert rounds
        if kind == "hea":
            # some round of the plan carries register-register CZ signs in its diagonal
            fwd = pi.parse(qfuse.qf_plan_export(h, 0))
            W = pi.FWD_ROUND_WORDS
            assert any(fwd.round_words[W * k + 5] for k in range(len(fwd.round_words) // W))
    finally:
        qfuse.qf_circuit_destroy(h)


def test_consecutive_gates_rows():
    from paper_2603_02804_gb300 import workloads
    rows = workloads.consecutive_gates(3, 4)
    assert rows[:5] == [(0, 0, -1, 0), (1, 0, -1, 1), (2, 0, -1, 2), (0, 0, -1, 3), (0, 1, -1, 4)]
    assert len(rows) == 12 and sorted(r[3] for r in rows) == list(range(12))


@pytest.mark.parametrize("seed", range(6))
def test_cnot_gate_lists_match_oracle(seed):
    """Random gate lists with CNOTs (control inside or outside the target's
    register group, inside or outside the tile) on generic programs."""
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(3, 15))
    n_params = 9
    rows = []
    for _ in range(50):
        k = int(rng.choice([orc.RX, orc.RY, orc.RZ, orc.CZ, orc.CNOT]))
        if k in (orc.CZ, orc.CNOT):
            a, b = rng.choice(n, 2, replace=False)
            rows.append((k, int(a), int(b), -1))
        else:
            rows.append((k, int(rng.integers(n)), -1, int(rng.integers(n_params))))
    h = qfuse.qf_circuit_create(n, rows, n_params)
    try:
        qfuse.qf_plan(h, 2, tile_bits=int(rng.choice([0, 5, 6])), ckpt_layers=1, host_only=True)
        theta = rng.uniform(0, 2 * np.pi, n_params).astype(np.float32).astype(np.float64)
        x = rng.uniform(0, np.pi, (2, n)).astype(np.float32).astype(np.float64)
        c = orc.Circuit(n=n, gates=np.array(rows, np.int32), n_params=n_params)
        slot_param = [r[3] for r in rows if r[0] not in (orc.CZ, orc.CNOT)]
        slot_kind = [r[0] for r in rows if r[0] not in (orc.CZ, orc.CNOT)]
        obs = "".join(rng.choice(list("IZ"), size=n))
        info, rounds = interp_check(h, n, theta, x, obs, slot_param, slot_kind, oracle_circ=c)
        assert not rounds
    finally:
        qfuse.qf_circuit_destroy(h)


@pytest.mark.parametrize("rule", [1, 2])
@pytest.mark.parametrize("n,d,K,ck", [(13, 3, 0, 1), (15, 3, 7, 1), (17, 2, 10, 0), (14, 4, 9, 2)])
def test_forced_catch_up_rules_match_oracle(rule, n, d, K, ck):
    """Both catch-up rules (strict, rising) that the autotuner may force give
    programs whose expectations and gradients equal the oracle's."""
    rng = np.random.default_rng(1500 + 7 * n + d + rule)
    h = qfuse.qf_hea_create(n, d)
    try:
        qfuse.qf_plan(h, 2, tile_bits=K, ckpt_layers=ck, host_only=True, catch_up=rule)
        info = qfuse.qf_plan_info(h)
        assert info["catch_up"] == rule
        P = 3 * n * d
        theta = rng.uniform(0, 2 * np.pi, P).astype(np.float32).astype(np.float64)
        x = rng.uniform(0, np.pi, (2, n)).astype(np.float32).astype(np.float64)
        slot_kind = [orc.RY if (p % 3) == 1 else orc.RZ for p in range(P)]
        interp_check(h, n, theta, x, "ZXY", list(range(P)), slot_kind, oracle_circ=orc.hea(n, d),
                     kernel_order=True)
    finally:
        qfuse.qf_circuit_destroy(h)


def test_tuning_options_are_validated_and_reported():
    h = qfuse.qf_hea_create(14, 3)
    try:
        for kw in (dict(catch_up=3), dict(catch_up=-1), dict(fwd_ctas=1), dict(fwd_ctas=4)):
            with pytest.raises(qfuse.QFError) as e:
                qfuse.qf_plan(h, 4, host_only=True, **kw)
            assert e.value.status == qfuse.QF_ERR_INVALID_ARG
        qfuse.qf_plan(h, 4, host_only=True, fwd_ctas=3)
        info = qfuse.qf_plan_info(h)
        assert info["fwd_ctas"] == 3 and info["catch_up"] in (1, 2)
        # the planner's choice is one of the two rules; forcing it reports it
        for rule in (1, 2):
            qfuse.qf_plan(h, 4, host_only=True, catch_up=rule)
            assert qfuse.qf_plan_info(h)["catch_up"] == rule
        # a single-tile circuit has no catch-up rounds
        h2 = qfuse.qf_hea_create(10, 3)
        try:
            qfuse.qf_plan(h2, 4, host_only=True, catch_up=1)
            assert qfuse.qf_plan_info(h2)["catch_up"] == 0
        finally:
            qfuse.qf_circuit_destroy(h2)
    finally:
        qfuse.qf_circuit_destroy(h)
