"""Host-side checks of complex128 plans (precision QF_PREC_C128): option
checking, plan summary and workspace, the exported program (interpreted in
complex128 against the oracle), and the precision check of every entry
point. No GPU needed."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2603_02804_gb300 import build as qbuild
from paper_2603_02804_gb300 import qfuse
from tests import plan_interp as pi


@pytest.fixture(scope="module", autouse=True)
def lib():
    qbuild.build()
    return qfuse.load()


@pytest.fixture
def hea12():
    h = qfuse.qf_hea_create(12, 3)
    yield h
    qfuse.qf_circuit_destroy(h)


def test_plan_info_and_workspace(hea12):
    B = 8
    ws32 = qfuse.qf_plan(hea12, B, host_only=True)
    i32 = qfuse.qf_plan_info(hea12)
    ws64 = qfuse.qf_plan(hea12, B, host_only=True, precision=qfuse.QF_PREC_C128)
    i64 = qfuse.qf_plan_info(hea12)
    assert i32["precision"] == qfuse.QF_PREC_C64 and i64["precision"] == qfuse.QF_PREC_C128
    assert i32["state_bytes"] == 8 * B * 4096 and i64["state_bytes"] == 16 * B * 4096
    # states dominate the workspace: work, lambda and the checkpoints double
    states = (2 + i64["n_ckpt"]) * i64["state_bytes"]
    assert ws64 - ws32 >= states // 2
    assert ws64 < 2 * ws32 + (1 << 20)


def test_complex128_plans_share_the_programs(hea12):
    """complex128 plans get the same programs as complex64 ones: round
    programs for the RZ,RY,RZ + chain circuit, generic steps on request."""
    qfuse.qf_plan(hea12, 2, host_only=True)
    p32 = qfuse.qf_plan_export(hea12, 0)
    qfuse.qf_plan(hea12, 2, host_only=True, precision=qfuse.QF_PREC_C128)
    p64 = qfuse.qf_plan_export(hea12, 0)
    assert p64[0] == 1 and np.array_equal(p32, p64)
    qfuse.qf_plan(hea12, 2, host_only=True, precision=qfuse.QF_PREC_C128, program=1)
    assert qfuse.qf_plan_export(hea12, 0)[0] == 0


@pytest.mark.parametrize("kw,status", [
    (dict(precision=2), qfuse.QF_ERR_INVALID_ARG),
    (dict(precision=-1), qfuse.QF_ERR_INVALID_ARG),
    (dict(precision=1, path=qfuse.QF_PATH_PER_GATE), qfuse.QF_ERR_UNSUPPORTED),
    (dict(precision=1, tc_path=True), qfuse.QF_ERR_UNSUPPORTED),
])
def test_plan_rejects(hea12, kw, status):
    with pytest.raises(qfuse.QFError) as e:
        qfuse.qf_plan(hea12, 4, host_only=True, **kw)
    assert e.value.status == status


def test_mode_a_mem_save_stores_complex64():
    """With ckpt_mode 1 and mem_save, the pass outputs of a complex128 plan
    are complex64: 8 bytes per stored amplitude instead of 16."""
    n, B = 14, 4
    h = qfuse.qf_hea_create(n, 4)
    sizes = {}
    try:
        for ms in (False, True):
            sizes[ms] = qfuse.qf_plan(h, B, ckpt_layers=2, ckpt_mode=1, mem_save=ms, host_only=True,
                                      precision=qfuse.QF_PREC_C128)
            info = qfuse.qf_plan_info(h)
            assert info["mem_save"] == int(ms)
    finally:
        qfuse.qf_circuit_destroy(h)
    slots = info["n_pass_slots"]
    assert slots >= 1
    saved = sizes[False] - sizes[True]
    assert abs(saved - slots * B * (1 << n) * 8) < 4096


@pytest.mark.parametrize("program", [0, 1])
@pytest.mark.parametrize("n,d,K,ck", [(5, 3, 0, 1), (9, 3, 6, 1), (13, 2, 0, 1)])
def test_exported_program_matches_oracle(n, d, K, ck, program):
    """The complex128 plan's forward and backward programs, interpreted in
    complex128 on the host, give the oracle's E and gradients."""
    rng = np.random.default_rng(4000 + n)
    h = qfuse.qf_hea_create(n, d)
    try:
        qfuse.qf_plan(h, 2, tile_bits=K, ckpt_layers=ck, host_only=True, precision=qfuse.QF_PREC_C128,
                      program=program)
        info = qfuse.qf_plan_info(h)
        theta = rng.uniform(0, 2 * np.pi, 3 * n * d)
        x = rng.uniform(0, np.pi, (2, n))
        fwd = pi.parse(qfuse.qf_plan_export(h, 0))
        bwd = pi.parse(qfuse.qf_plan_export(h, 1))
        assert fwd.rounds_mode == (program == 0 and info["tile_bits"] >= 7)
        pq = qfuse.pauli("XZ", n)
        gr, Er = orc.gradient(orc.hea(n, d), theta, x, "XZ", per_sample=True)
        for b in range(2):
            E, slots = pi.run_forward(fwd, n, info["n_eff"], theta, x[b], pq.x_mask, pq.z_mask)
            assert abs(E - Er[b]) < 1e-10
            g = pi.run_backward(bwd, info["n_eff"], theta, slots, pq.x_mask, pq.z_mask, 1.0, len(theta))
            assert np.max(np.abs(g - gr[b])) < 1e-10
    finally:
        qfuse.qf_circuit_destroy(h)


def test_entry_points_check_precision():
    n, B = 5, 4
    h = qfuse.qf_hea_create(n, 2)
    obs = qfuse.pauli("Z", n)
    try:
        ws = qfuse.qf_plan(h, B, host_only=True, precision=qfuse.QF_PREC_C128)
        for call in (lambda: qfuse.qf_forward(h, 0, 0, B, obs, 0, 0, ws),
                     lambda: qfuse.qf_backward(h, 0, 0, B, obs, 0, 0, 0, 0, ws),
                     lambda: qfuse.qf_train_step(h, 0, 0, 0, B, 0, obs, 0, 0, 0, 0, ws),
                     lambda: qfuse.qf_train_step_host(h, 0, 0, 0, B, 0, obs, 0, 0, 0, 0, ws),
                     lambda: qfuse.qf_train_step_noalloc(h, 0, 0, 0, B, 0, obs, 0, 0, 0)):
            with pytest.raises(qfuse.QFError) as e:
                call()
            assert e.value.status == qfuse.QF_ERR_INVALID_ARG
            assert "complex128" in qfuse.qf_last_error()
        # the *64 entry points accept the plan and stop at the missing device tables
        with pytest.raises(qfuse.QFError) as e:
            qfuse.qf_forward64(h, 0, 0, B, obs, 0, 256, ws)
        assert e.value.status == qfuse.QF_ERR_WORKSPACE
        qfuse.qf_plan(h, B, host_only=True)
        with pytest.raises(qfuse.QFError) as e:
            qfuse.qf_train_step64(h, 0, 0, 0, B, 0, obs, 0, 0, 0, 0, ws)
        assert e.value.status == qfuse.QF_ERR_INVALID_ARG
        assert "complex64" in qfuse.qf_last_error()
    finally:
        qfuse.qf_circuit_destroy(h)


def test_loss64_argument_checks():
    with pytest.raises(qfuse.QFError):
        qfuse.qf_loss64(7, 0, 0, 1, 0, 0)
    with pytest.raises(qfuse.QFError):
        qfuse.qf_loss64(qfuse.QF_LOSS_MSE, 0, None, 4, 0, 0)
