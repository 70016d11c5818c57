"""qf_train_step_noalloc: the training step for callers that cannot allocate
device memory.

Some callers live inside a host application that owns the whole device-memory
budget and forbids new allocations once it is running (a real-time loop, a
plugin inside another framework's memory pool). They cannot call cudaMalloc
or hand the library a workspace sized per call, so this entry point keeps its
buffers in one fixed 32 MiB block that the library reserves per GPU. The test
checks, through the C-ABI, that it returns what the regular workspace entry
point (qf_train_step) returns, on two calls in a row with another circuit's
call between them, and what the float64 oracle returns, and that requests
beyond the plan or the fixed block are refused with a clear error.
"""
import numpy as np
import pytest
import torch

from paper_2603_02804_gb300 import build as qbuild
from paper_2603_02804_gb300 import qfuse, workloads

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()


def _inputs(B):
    w = workloads.WORKLOADS["hea12"]
    theta, x, y = workloads.make_inputs(w, B=B)
    cuda = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return w, cuda(theta), cuda(x), cuda(y)


def _outputs(w, B):
    z = lambda *s: torch.zeros(*s, dtype=torch.float64, device="cuda")
    return z(1), z(B), z(w.n_params)


def _tiny_noalloc_call(stream):
    """A different circuit and batch through the shared block (4 qubits, B=8,
    L = sum E), so that the next hea12 call meets a block holding another
    call's contents."""
    w = workloads.WORKLOADS["tiny"]
    theta, x, _ = workloads.make_inputs(w)
    h = qfuse.qf_hea_create(w.n, w.d)
    qfuse.qf_plan(h, w.B, host_only=True)
    try:
        loss, E, g = _outputs(w, w.B)
        qfuse.qf_train_step_noalloc(h, torch.from_numpy(theta).cuda(), torch.from_numpy(x).cuda(), None, w.B,
                                    qfuse.QF_LOSS_SUM, qfuse.pauli("Z", w.n), loss, E, g, stream)
        torch.cuda.synchronize()
        assert abs(loss.item() - E.sum().item()) < TOL
    finally:
        qfuse.qf_circuit_destroy(h)


def test_noalloc_step_matches_workspace_step_twice():
    B = 64
    w, theta, x, y = _inputs(B)
    obs = qfuse.pauli("Z", w.n)
    stream = torch.cuda.current_stream()

    # regular entry point with a caller-allocated workspace
    ref_h = qfuse.qf_hea_create(w.n, w.d)
    ws_bytes = qfuse.qf_plan(ref_h, B)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    loss_r, E_r, g_r = _outputs(w, B)
    qfuse.qf_train_step(ref_h, theta, x, y, B, qfuse.QF_LOSS_MSE, obs, loss_r, E_r, g_r, ws, ws_bytes, stream)

    # no-allocation entry point on a host-only plan (no device tables either);
    # between the two compared calls another circuit and batch use the block
    h = qfuse.qf_hea_create(w.n, w.d)
    qfuse.qf_plan(h, B, host_only=True)
    try:
        for call in range(2):
            loss, E, g = _outputs(w, B)
            qfuse.qf_train_step_noalloc(h, theta, x, y, B, qfuse.QF_LOSS_MSE, obs, loss, E, g, stream)
            torch.cuda.synchronize()
            assert abs(loss.item() - loss_r.item()) < TOL, call
            assert torch.max(torch.abs(E - E_r)).item() < TOL, call
            assert torch.max(torch.abs(g - g_r)).item() < TOL, call
            if call == 0:
                _tiny_noalloc_call(stream)
        # and against the float64 oracle directly (MSE loss, its gradient)
        from oracle import oracle as orc
        th64, x64, y64 = (t.cpu().numpy().astype(np.float64) for t in (theta, x, y))
        E_o = orc.expectation(orc.hea(w.n, w.d), th64, x64, "Z")
        g_o, _ = orc.gradient(orc.hea(w.n, w.d), th64, x64, "Z", dLdE=orc.mse_dLdE(E_o, y64))
        assert abs(loss.item() - orc.mse_loss(E_o, y64)) < TOL
        assert np.max(np.abs(E.cpu().numpy() - E_o)) < TOL
        assert np.max(np.abs(g.cpu().numpy() - g_o)) < TOL
    finally:
        qfuse.qf_circuit_destroy(h)
        qfuse.qf_circuit_destroy(ref_h)


def test_noalloc_step_refuses_a_batch_beyond_the_plan():
    B = 8
    w, theta, x, y = _inputs(B)
    h = qfuse.qf_hea_create(w.n, w.d)
    qfuse.qf_plan(h, B, host_only=True)
    try:
        loss, E, g = _outputs(w, B)
        with pytest.raises(qfuse.QFError) as e:
            qfuse.qf_train_step_noalloc(h, theta, x, y, 1 << 40, qfuse.QF_LOSS_MSE, qfuse.pauli("Z", w.n),
                                        loss, E, g)
        assert e.value.status == qfuse.QF_ERR_INVALID_ARG
    finally:
        qfuse.qf_circuit_destroy(h)


def test_noalloc_step_refuses_batches_beyond_the_fixed_block():
    B = 256  # the hea12 step at full batch needs more than 32 MiB
    w, theta, x, y = _inputs(B)
    h = qfuse.qf_hea_create(w.n, w.d)
    qfuse.qf_plan(h, B, host_only=True)
    try:
        loss, E, g = _outputs(w, B)
        with pytest.raises(qfuse.QFError) as e:
            qfuse.qf_train_step_noalloc(h, theta, x, y, B, qfuse.QF_LOSS_MSE, qfuse.pauli("Z", w.n), loss, E, g)
        assert e.value.status == qfuse.QF_ERR_WORKSPACE
        assert "QF_NOALLOC_MAX_BYTES" in str(e.value)
    finally:
        qfuse.qf_circuit_destroy(h)
