"""GPU parity of the tensor-core block path: forward rounds applied as 32x32
real blocks with tcgen05 MMAs in split precision (3xTF32, float32
accumulation), the adjoint on the CUDA cores. Tolerance 1e-5 against the
oracle, like the CUDA-core path."""
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


def run(n, d, theta, x, obs="Z", **kw):
    B = len(x)
    sim = Simulator(n, d, B, obs=obs, **kw)
    th = torch.as_tensor(theta, dtype=torch.float32, device="cuda")
    xd = torch.as_tensor(x, dtype=torch.float32, device="cuda")
    E = sim.forward(th, xd)
    g = sim.backward(th, xd, torch.ones(B, dtype=torch.float64), per_sample=True)
    torch.cuda.synchronize()
    assert qfuse.qf_device_status() == 0
    return E.cpu().numpy(), g.cpu().numpy(), sim


def inputs(n, d, B, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32),
            rng.uniform(0, np.pi, (B, n)).astype(np.float32))


def f64(a):
    return np.asarray(a, np.float32).astype(np.float64)


def test_tc_single_layer():
    n, d, B = 12, 1, 2
    theta, x = inputs(n, d, B, 1201)
    E, g, sim = run(n, d, theta, x, tc_path=True)
    assert sim.info()["tc_path"] == 1
    gr, Er = orc.gradient(orc.hea(n, d), f64(theta), f64(x), "Z", per_sample=True)
    assert np.max(np.abs(E - Er)) < TOL
    assert np.max(np.abs(g - gr)) < TOL


def test_tc_hea12_full_batch():
    """The benchmarked shape (n = 12, d = 20, B = 256), every sample."""
    w = workloads.WORKLOADS["hea12"]
    theta, x, _ = workloads.make_inputs(w)
    E, g, _ = run(w.n, w.d, theta, x, tc_path=True, ckpt_layers=10)
    gr, Er = orc.gradient(orc.hea(w.n, w.d), f64(theta), f64(x), "Z", per_sample=True)
    assert np.max(np.abs(E - Er)) < TOL
    assert np.max(np.abs(g - gr)) < TOL
    E0, _, _ = run(w.n, w.d, theta, x, ckpt_layers=10)
    assert np.max(np.abs(E - E0)) < TOL


@pytest.mark.parametrize("n,d,ck,obs", [(13, 4, 1, "ZIX"), (16, 12, 4, "Z"), (14, 6, 2, "XY")])
def test_tc_multi_pass(n, d, ck, obs):
    theta, x = inputs(n, d, 3, 1300 + n)
    E, g, sim = run(n, d, theta, x, obs=obs, tc_path=True, ckpt_layers=ck)
    gr, Er = orc.gradient(orc.hea(n, d), f64(theta), f64(x), obs, per_sample=True)
    assert np.max(np.abs(E - Er)) < TOL
    assert np.max(np.abs(g - gr)) < TOL


def test_tc_mode_a_recompute():
    n, d = 15, 6
    theta, x = inputs(n, d, 2, 1515)
    E, g, sim = run(n, d, theta, x, tc_path=True, ckpt_layers=2, ckpt_mode=1)
    gr, Er = orc.gradient(orc.hea(n, d), f64(theta), f64(x), "Z", per_sample=True)
    assert np.max(np.abs(E - Er)) < TOL
    assert np.max(np.abs(g - gr)) < TOL


def test_tc_n20_light_cone():
    n, d, B = 20, 5, 4
    theta, x = inputs(n, d, B, 2025)
    E, g, _ = run(n, d, theta, x, tc_path=True, ckpt_layers=2)
    m = d
    tt = f64(theta).reshape(d, n, 3)[:, :m, :].reshape(-1)
    gr, Er = orc.gradient(orc.hea(m, d), tt, f64(x[:, :m]), "Z", per_sample=True)
    assert np.max(np.abs(E - Er)) < TOL
    gg = g.reshape(B, d, n, 3)
    assert np.max(np.abs(gg[:, :, :m, :].reshape(B, -1) - gr)) < TOL
    assert np.max(np.abs(gg[:, :, m:, :])) < TOL
