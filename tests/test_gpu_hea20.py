"""GPU parity at the shape of the large workload (n = 20, d = 1000, 1000
samples in micro-batches of 100): the same planner, the same checkpoint
interval chosen from device memory for a micro-batch of 100, the same qubit
layout, many passes, checkpoint re-anchors, and, for mode A, the re-run
forward. Inputs: the workload's own theta (its first d layers) and x (its
first samples). Deep enough (d = 24 > n) that the light cone of Z_0 covers
every qubit, so every gradient is compared against the full 20-qubit oracle.

Tolerance: 1e-5 max absolute error on E and on every per-sample gradient
dE_b/dtheta, and on the whole-batch gradient of a train step.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2603_02804_gb300 import build as qbuild
from paper_2603_02804_gb300 import qfuse, workloads
from paper_2603_02804_gb300.torch_api import Simulator
from tests import oracle_proc

pytestmark = pytest.mark.gpu
TOL = 1e-5
N, D, B = 20, 24, 2
MICRO_BATCH = 100


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    orc.build()


@pytest.fixture(scope="module")
def inputs():
    w = workloads.WORKLOADS["hea20"]
    theta, x, _ = workloads.make_inputs(w, B=B)
    theta = np.ascontiguousarray(theta[:3 * N * D])
    return theta, np.ascontiguousarray(x)


@pytest.fixture(scope="module")
def reference(inputs):
    theta, x = inputs
    g, E = oracle_proc.call("gradient", orc.hea(N, D), theta.astype(np.float64), x.astype(np.float64), "Z",
                            per_sample=True)
    return E, g


def epoch_interval(ckpt_mode):
    """The checkpoint interval the benchmark's epoch plans for a micro-batch of
    100 samples from the free device memory (as bench.py chooses it)."""
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    h = qfuse.qf_hea_create(N, 1000)
    try:
        c, _ = qfuse.qf_plan_fit(h, MICRO_BATCH, int(0.8 * free), host_only=True, ckpt_mode=ckpt_mode)
        shift = qfuse.qf_plan_info(h)["qubit_shift"]
    finally:
        qfuse.qf_circuit_destroy(h)
    return c, shift


def run(theta, x, **kw):
    sim = Simulator(N, D, B, **kw)
    th = torch.from_numpy(theta).cuda()
    xd = torch.from_numpy(x).cuda()
    E = sim.forward(th, xd)
    g = sim.backward(th, xd, torch.ones(B, dtype=torch.float64), per_sample=True)
    loss, E2, g2 = sim.train_step(th, xd, loss="sum")
    torch.cuda.synchronize()
    return E.cpu().numpy(), g.cpu().numpy(), loss.item(), g2.cpu().numpy(), sim


@pytest.mark.parametrize("ckpt_mode", [0, 1])
def test_hea20_epoch_plan_against_full_oracle(inputs, reference, ckpt_mode):
    theta, x = inputs
    E_r, g_r = reference
    c, shift = epoch_interval(0)
    assert 1 <= c <= D // 3, c
    if ckpt_mode == 1:
        # mode A's interval from memory is about sqrt(d / passes per layer)
        # (40 at d = 1000), a single block at this depth: take 6 (4 blocks)
        c = 6
    E, g, loss, g_sum, sim = run(theta, x, ckpt_layers=c, ckpt_mode=ckpt_mode)
    info = sim.info()
    # the epoch's plan structure: the same qubit layout, many passes over
    # 12-qubit tiles, and several stored checkpoints
    assert info["qubit_shift"] == shift
    assert info["tile_bits"] == 12 and info["n_passes"] >= 8
    assert info["n_ckpt"] >= 3
    e_err = float(np.max(np.abs(E - E_r)))
    g_err = float(np.max(np.abs(g - g_r)))
    assert e_err < TOL, e_err
    assert g_err < TOL, g_err
    assert abs(loss - E_r.sum()) < TOL
    assert np.max(np.abs(g_sum - g_r.sum(0))) < TOL
    # no rotation is outside the light cone at this depth except the last RZ
    # on qubit 0 of the last layer, which commutes with Z_0
    gz = np.abs(g_r).reshape(B, D, N, 3)
    assert np.min(gz[:, :D - N, :, :].max(axis=0)) > 0


def test_hea20_tensor_core_forward_against_full_oracle(inputs, reference):
    theta, x = inputs
    E_r, g_r = reference
    c, _ = epoch_interval(0)
    E, g, _, _, sim = run(theta, x, ckpt_layers=c, tc_path=True)
    assert sim.info()["tc_path"] == 1
    assert qfuse.qf_device_status() == 0
    assert float(np.max(np.abs(E - E_r))) < TOL
    assert float(np.max(np.abs(g - g_r))) < TOL
