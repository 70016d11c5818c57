"""GPU parity for the paper's measurement setting (Sec. 4): given random
initial states instead of the RY(x) encoding, the Rx, Ry, Rz + CZ-ring ansatz,
and the (IXYZ)^(n/4) observable, including observables whose X/Y qubits lie
outside the last pass's tile (expectation and adjoint seed as their own full
passes). Tolerance 1e-5 against the oracle."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2603_02804_gb300 import build as qbuild
from paper_2603_02804_gb300 import qfuse, workloads
from paper_2603_02804_gb300.torch_api import Simulator

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    orc.build()


def run(n, d, theta, x, obs, **kw):
    B = len(x)
    sim = Simulator(n, d, B, obs=obs, **kw)
    th = torch.as_tensor(theta, dtype=torch.float32, device="cuda")
    xd = torch.as_tensor(x, device="cuda")
    E = sim.forward(th, xd)
    g = sim.backward(th, xd, torch.ones(B, dtype=torch.float64), per_sample=True)
    torch.cuda.synchronize()
    return E.cpu().numpy(), g.cpu().numpy(), sim


def f64(a):
    return np.asarray(a, np.float32).astype(np.float64)


def oracle_states(c, theta, psi0, obs):
    return orc.gradient(c, f64(theta), None, obs, per_sample=True, init_states=psi0.astype(np.complex128))


@pytest.mark.parametrize("path", ["fused", "per_gate"])
@pytest.mark.parametrize("n,d", [(3, 2), (12, 4)])
def test_given_states_hea(n, d, path):
    B = 5
    rng = np.random.default_rng(60 + n)
    theta = rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32)
    psi0 = workloads.draw_state(B, n, 61 + n)
    E, g, _ = run(n, d, theta, psi0, "Z" * min(n, 2), encoding="state", path=path)
    gr, Er = oracle_states(orc.hea(n, d), theta, psi0, "Z" * min(n, 2))
    assert np.max(np.abs(E - Er)) < TOL
    assert np.max(np.abs(g - gr)) < TOL


@pytest.mark.parametrize("n,d,ck,mode", [(8, 3, 0, 0), (14, 2, 1, 0), (14, 3, 1, 1), (16, 2, 1, 0)])
def test_paper_ansatz_random_states_ixyz(n, d, ck, mode):
    """Rx, Ry, Rz + CZ ring on random states with O = IXYZ...; for n > 12 the
    observable's X/Y qubits span more than one tile."""
    B = 3
    rows = workloads.xyz_ring_gates(n, d)
    P = 3 * n * d
    rng = np.random.default_rng(70 + n + d)
    theta = rng.uniform(0, 2 * np.pi, P).astype(np.float32)
    psi0 = workloads.draw_state(B, n, 71 + n)
    obs = workloads.ixyz(n)
    E, g, sim = run(n, 0, theta, psi0, obs, encoding="state", gates=rows, n_params=P, ckpt_layers=ck,
                    ckpt_mode=mode)
    c = orc.Circuit(n=n, gates=np.array(rows, np.int32), n_params=P)
    gr, Er = oracle_states(c, theta, psi0, obs)
    assert np.max(np.abs(E - Er)) < TOL
    assert np.max(np.abs(g - gr)) < TOL


@pytest.mark.parametrize("tc", [False, True])
def test_off_tile_observable_with_encoding(tc):
    """RY(x) encoding, RZ,RY,RZ + chain, n = 16: O = IXYZ IXYZ IXYZ IXYZ has X
    and Y factors on qubits 13 and 14, outside a 12-qubit tile of the last pass."""
    n, d, B = 16, 3, 4
    rng = np.random.default_rng(1616)
    theta = rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32)
    x = rng.uniform(0, np.pi, (B, n)).astype(np.float32)
    obs = workloads.ixyz(n)
    E, g, sim = run(n, d, theta, x, obs, tc_path=tc, ckpt_layers=1)
    gr, Er = orc.gradient(orc.hea(n, d), f64(theta), f64(x), obs, per_sample=True)
    assert np.max(np.abs(E - Er)) < TOL
    assert np.max(np.abs(g - gr)) < TOL


def test_n20_paper_ansatz_depth1():
    """The measured configuration's shape: n = 20, d = 1, random states, O = IXYZ..."""
    n, d, B = 20, 1, 2
    rows = workloads.xyz_ring_gates(n, d)
    P = 3 * n * d
    rng = np.random.default_rng(2020)
    theta = rng.uniform(0, 2 * np.pi, P).astype(np.float32)
    psi0 = workloads.draw_state(B, n, 2021)
    obs = workloads.ixyz(n)
    E, g, _ = run(n, 0, theta, psi0, obs, encoding="state", gates=rows, n_params=P)
    c = orc.Circuit(n=n, gates=np.array(rows, np.int32), n_params=P)
    gr, Er = oracle_states(c, theta, psi0, obs)
    assert np.max(np.abs(E - Er)) < TOL
    assert np.max(np.abs(g - gr)) < TOL


@pytest.mark.parametrize("m", [1, 9, 20])
def test_consecutive_gates_fusion_depth(m):
    """The fusion-depth circuit of Sec. 4.1 (m consecutive Rx, Ry, Rz gates on
    every qubit), n = 14 so that it takes two tiles."""
    n, B = 14, 3
    rows = workloads.consecutive_gates(n, m)
    P = n * m
    rng = np.random.default_rng(3000 + m)
    theta = rng.uniform(0, 2 * np.pi, P).astype(np.float32)
    psi0 = workloads.draw_state(B, n, 3001 + m)
    obs = workloads.ixyz(n)
    E, g, _ = run(n, 0, theta, psi0, obs, encoding="state", gates=rows, n_params=P)
    c = orc.Circuit(n=n, gates=np.array(rows, np.int32), n_params=P)
    gr, Er = oracle_states(c, theta, psi0, obs)
    assert np.max(np.abs(E - Er)) < TOL
    assert np.max(np.abs(g - gr)) < TOL
