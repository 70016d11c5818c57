"""GPU parity of the complex128 path (precision QF_PREC_C128) against the
float64 oracle, through the C-ABI.

Both sides compute in float64, so only rounding separates them: a circuit of
M gates moves each amplitude by at most about 8 M 2^-53 relative (a complex
2x2 update is 8 floating-point operations per output), under 1e-12 for the
M <= 1000 gates used here, and the float64 reductions add less. The
tolerance is 1e-11 on E and on every per-sample gradient. The memory-saving
mode stores pass outputs as complex64 (relative rounding 2^-24 each), checked
at 1e-6. Parameters, angles and given states are drawn in float64 and used
unrounded on both sides.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2603_02804_gb300 import build as qbuild
from paper_2603_02804_gb300 import qfuse, workloads
from paper_2603_02804_gb300.torch_api import HEA, QFuseFn, Simulator

pytestmark = pytest.mark.gpu
TOL64 = 1e-11
TOL_SAVE = 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    orc.build()


def run64(n, d, theta, x, obs="Z", per_sample=True, dLdE=None, **kw):
    B = len(x)
    sim = Simulator(n, d, B, obs=obs, precision="complex128", **kw)
    th = torch.as_tensor(theta, dtype=torch.float64, device="cuda")
    xd = torch.as_tensor(np.ascontiguousarray(x), device="cuda")
    E = sim.forward(th, xd)
    w = torch.ones(B, dtype=torch.float64) if dLdE is None else torch.as_tensor(dLdE, dtype=torch.float64)
    g = sim.backward(th, xd, w, per_sample=per_sample)
    torch.cuda.synchronize()
    return E.cpu().numpy(), g.cpu().numpy(), sim


def draw(n_params, B, n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, 2 * np.pi, n_params), rng.uniform(0, np.pi, (B, n))


@pytest.mark.parametrize("program", [0, 1])
@pytest.mark.parametrize("n,d,K,ck,obs", [
    (1, 2, 0, 0, "X"), (3, 3, 0, 0, "XZ"), (4, 3, 0, 0, "ZX"), (6, 4, 0, 1, "XZ"), (9, 4, 6, 2, "ZZ"),
    (12, 6, 0, 2, "XYZ"), (13, 3, 5, 1, "Z"), (14, 4, 0, 1, "XZ"),
])
def test_hea_angles(n, d, K, ck, obs, program):
    """RY(x) encoding, RZ,RY,RZ + CZ chain: single tiles (n <= 12, including
    padded n < 4 and the one-thread tile n = 4), several passes per layer
    (tile_bits 5 and 6), checkpoints and re-anchoring, X/Y observables; round
    programs (program 0, tiles of >= 7 qubits) and generic steps."""
    B = 5
    theta, x = draw(3 * n * d, B, n, 500 + 31 * n + d)
    E, g, sim = run64(n, d, theta, x, obs=obs, tile_bits=K, ckpt_layers=ck, program=program)
    info = sim.info()
    assert info["precision"] == qfuse.QF_PREC_C128
    assert info["state_bytes"] == 16 * B * (1 << info["n_eff"])
    gr, Er = orc.gradient(orc.hea(n, d), theta, x, obs, per_sample=True)
    assert np.max(np.abs(E - Er)) < TOL64
    assert np.max(np.abs(g - gr)) < TOL64


def test_hea12_full_batch():
    """n = 12, d = 20, batch 256 (the benchmarked shape), every sample; plus
    the batch-summed gradient with random dL/dE."""
    n, d, B = 12, 20, 256
    theta, x = draw(3 * n * d, B, n, 1220)
    E, g, _ = run64(n, d, theta, x)
    gr, Er = orc.gradient(orc.hea(n, d), theta, x, "Z", per_sample=True)
    assert np.max(np.abs(E - Er)) < TOL64
    assert np.max(np.abs(g - gr)) < TOL64
    w = np.random.default_rng(1221).standard_normal(B)
    _, gs, _ = run64(n, d, theta, x, per_sample=False, dLdE=w)
    assert np.max(np.abs(gs - w @ gr)) < 1e-10 * max(1.0, np.max(np.abs(w @ gr)))


@pytest.mark.parametrize("seed", range(3))
def test_gate_lists_cnot_cz_rx(seed):
    """Random gate lists: RX/RY/RZ with shared parameters, CZ and CNOT on
    arbitrary qubit pairs (controls inside and outside the register group)."""
    rng = np.random.default_rng(580 + seed)
    n = [6, 11, 15][seed]
    n_params = 10
    rows = []
    for _ in range(70):
        k = int(rng.choice([orc.RX, orc.RY, orc.RZ, orc.CZ, orc.CNOT]))
        if k in (orc.CZ, orc.CNOT):
            a, b = rng.choice(n, 2, replace=False)
            rows.append((k, int(a), int(b), -1))
        else:
            rows.append((k, int(rng.integers(n)), -1, int(rng.integers(n_params))))
    theta, x = draw(n_params, 4, n, 590 + seed)
    c = orc.Circuit(n=n, gates=np.array(rows, np.int32), n_params=n_params)
    gr, Er = orc.gradient(c, theta, x, "ZX", per_sample=True)
    E, g, _ = run64(n, 0, theta, x, obs="ZX", gates=rows, n_params=n_params, ckpt_layers=1)
    assert np.max(np.abs(E - Er)) < TOL64
    assert np.max(np.abs(g - gr)) < TOL64


@pytest.mark.parametrize("n,d,ck,mode", [(3, 2, 0, 0), (8, 3, 0, 0), (14, 2, 1, 0), (14, 3, 1, 1), (16, 2, 1, 0)])
def test_given_states_ixyz(n, d, ck, mode):
    """The paper's measurement setting in complex128: given random states,
    Rx,Ry,Rz + CZ ring, O = IXYZ...; for n > 12 the X/Y qubits span more than
    one tile (expectation and adjoint seed as full passes)."""
    B = 3
    rows = workloads.xyz_ring_gates(n, d)
    P = 3 * n * d
    theta = np.random.default_rng(600 + n + d).uniform(0, 2 * np.pi, P)
    psi0 = workloads.draw_state(B, n, 601 + n, dtype=np.complex128)
    obs = workloads.ixyz(n)
    E, g, _ = run64(n, 0, theta, psi0, obs, encoding="state", gates=rows, n_params=P, ckpt_layers=ck,
                    ckpt_mode=mode)
    c = orc.Circuit(n=n, gates=np.array(rows, np.int32), n_params=P)
    gr, Er = orc.gradient(c, theta, None, obs, per_sample=True, init_states=psi0)
    assert np.max(np.abs(E - Er)) < TOL64
    assert np.max(np.abs(g - gr)) < TOL64


@pytest.mark.parametrize("program", [0, 1])
@pytest.mark.parametrize("mem_save", [False, True])
def test_mode_a_block_recompute(mem_save, program):
    """Checkpoint mode 1 (per-block forward re-run storing pass outputs); with
    mem_save the stored pass outputs are complex64."""
    n, d, B = 14, 6, 3
    theta, x = draw(3 * n * d, B, n, 1414)
    E, g, sim = run64(n, d, theta, x, obs="XZ", ckpt_layers=2, ckpt_mode=1, mem_save=mem_save, program=program)
    info = sim.info()
    assert info["ckpt_mode"] == 1 and info["n_pass_slots"] > 0 and info["mem_save"] == int(mem_save)
    gr, Er = orc.gradient(orc.hea(n, d), theta, x, "XZ", per_sample=True)
    assert np.max(np.abs(E - Er)) < TOL64  # the forward itself stores nothing at reduced precision
    tol = TOL_SAVE if mem_save else TOL64
    err = np.max(np.abs(g - gr))
    assert err < tol
    if mem_save:
        assert err > 1e-13  # the complex64 storage is really in the path


def test_train_step_mse_device_and_host():
    """qf_train_step64 (forward + MSE + adjoint) against the oracle, and
    qf_train_step_host64 returning the same numbers bit for bit."""
    n, d, B = 10, 5, 16
    theta, x = draw(3 * n * d, B, n, 1010)
    y = np.random.default_rng(1011).uniform(-1, 1, B)
    sim = Simulator(n, d, B, precision="complex128")
    dv = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    loss, E, g = sim.train_step(dv(theta), dv(x), dv(y), loss="mse")
    torch.cuda.synchronize()
    c = orc.hea(n, d)
    Er = orc.expectation(c, theta, x, "Z")
    gr, _ = orc.gradient(c, theta, x, "Z", dLdE=orc.mse_dLdE(Er, y))
    assert abs(loss.item() - orc.mse_loss(Er, y)) < TOL64
    assert np.max(np.abs(E.cpu().numpy() - Er)) < TOL64
    assert np.max(np.abs(g.cpu().numpy() - gr)) < TOL64
    pin = lambda a: torch.as_tensor(a, dtype=torch.float64).pin_memory()
    lh, Eh, gh = sim.train_step_host(pin(theta), pin(x), pin(y), loss="mse")
    assert lh.item() == loss.item()
    assert torch.equal(Eh, E.cpu()) and torch.equal(gh, g.cpu())


def test_autograd_gradcheck():
    """Finite differences of the GPU forward against the GPU adjoint (torch's
    gradcheck in float64): a check that needs neither the oracle nor the
    adjoint's algebra."""
    n, d, B = 5, 2, 3
    sim = Simulator(n, d, B, obs="XZY", precision="complex128")
    gen = torch.Generator().manual_seed(55)
    theta = (torch.rand(3 * n * d, generator=gen, dtype=torch.float64) * 6.283).cuda().requires_grad_()
    x = (torch.rand(B, n, generator=gen, dtype=torch.float64) * 3.1416).cuda()
    assert torch.autograd.gradcheck(lambda t: QFuseFn.apply(t, x, sim), (theta,), eps=1e-6, atol=1e-7, rtol=1e-5)


def test_hea_module_float64_parameters():
    model = HEA(6, 3, 8, precision="complex128")
    assert model.theta.dtype == torch.float64
    x = torch.rand(8, 6, dtype=torch.float64, device="cuda")
    model(x).sum().backward()
    theta = model.theta.detach().cpu().numpy()
    gr, _ = orc.gradient(orc.hea(6, 3), theta, x.cpu().numpy(), "Z")
    assert np.max(np.abs(model.theta.grad.cpu().numpy() - gr)) < TOL64


def test_precision_mismatch_and_repeatability():
    """complex64 entry points refuse a complex128 plan (and the reverse); two
    runs give bitwise equal results."""
    n, d, B = 7, 3, 4
    theta, x = draw(3 * n * d, B, n, 77)
    E1, g1, sim = run64(n, d, theta, x)
    E2, g2, _ = run64(n, d, theta, x)
    assert np.array_equal(E1, E2) and np.array_equal(g1, g2)
    th32 = torch.zeros(3 * n * d, device="cuda")
    x32 = torch.zeros(B, n, device="cuda")
    E = torch.empty(B, dtype=torch.float64, device="cuda")
    with pytest.raises(qfuse.QFError) as e:
        qfuse.qf_forward(sim.handle, th32, x32, B, sim.obs, E, sim.ws, sim.ws_bytes)
    assert e.value.status == qfuse.QF_ERR_INVALID_ARG
    s32 = Simulator(n, d, B)
    with pytest.raises(qfuse.QFError) as e:
        qfuse.qf_forward64(s32.handle, th32.double(), x32.double(), B, s32.obs, E, s32.ws, s32.ws_bytes)
    assert e.value.status == qfuse.QF_ERR_INVALID_ARG
