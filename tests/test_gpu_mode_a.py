"""GPU parity of checkpoint mode A (the paper's checkpointed scheme, Sec. 3.4:
per block the forward is re-run storing every pass output, and each adjoint
pass starts from the stored output of the forward pass it undoes) and of its
memory-saving variant (pass outputs stored as bfloat16, Sec. 3.2).

Mode A: 1e-5 max absolute error against the oracle, like mode B. Memory
saving: the bfloat16 rounding of the stored pass outputs (relative 2^-9)
bounds the error; the measured error is printed and must stay below 2e-3.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2603_02804_gb300 import build as qbuild
from paper_2603_02804_gb300.torch_api import Simulator

pytestmark = pytest.mark.gpu
TOL = 1e-5
BF16_TOL = 2e-3


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
    return E.cpu().numpy(), g.cpu().numpy(), sim


def inputs(n, d, B, seed):
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32)
    x = rng.uniform(0, np.pi, (B, n)).astype(np.float32)
    return theta, x


def f64(a):
    return np.asarray(a, np.float32).astype(np.float64)


@pytest.mark.parametrize("n,d,K,ck", [(12, 6, 0, 2), (13, 4, 0, 1), (14, 3, 8, 2), (15, 5, 5, 2), (17, 3, 0, 1),
                                      (16, 20, 0, 5)])
def test_mode_a_matches_oracle(n, d, K, ck):
    theta, x = inputs(n, d, 3, 300 + n + d)
    E, g, sim = run(n, d, theta, x, obs="ZIX", tile_bits=K, ckpt_layers=ck, ckpt_mode=1)
    info = sim.info()
    assert info["ckpt_mode"] == 1
    gr, Er = orc.gradient(orc.hea(n, d), f64(theta), f64(x), "ZIX", per_sample=True)
    assert np.max(np.abs(E - Er)) < TOL
    assert np.max(np.abs(g - gr)) < TOL
    assert sim.launches() > 0


def test_mode_a_equals_mode_b_n18():
    n, d, B = 18, 10, 2
    theta, x = inputs(n, d, B, 1818)
    Ea, ga, sa = run(n, d, theta, x, ckpt_layers=3, ckpt_mode=1)
    Eb, gb, sb = run(n, d, theta, x, ckpt_layers=3)
    assert sa.info()["n_pass_slots"] >= 1 and sa.info()["n_passes"] > 1
    gr, Er = orc.gradient(orc.hea(n, d), f64(theta), f64(x), "Z", per_sample=True)
    assert np.max(np.abs(Ea - Er)) < TOL and np.max(np.abs(Eb - Er)) < TOL
    assert np.max(np.abs(ga - gr)) < TOL and np.max(np.abs(gb - gr)) < TOL
    assert np.max(np.abs(ga - gb)) < TOL


@pytest.mark.parametrize("n,d,ck", [(14, 6, 2), (17, 4, 2), (20, 6, 3)])
def test_mem_save_error_bound(n, d, ck, capsys):
    B = 2
    theta, x = inputs(n, d, B, 500 + n)
    E, g, sim = run(n, d, theta, x, ckpt_layers=ck, ckpt_mode=1, mem_save=True)
    assert sim.info()["mem_save"] == 1
    if n <= 17:
        gr, Er = orc.gradient(orc.hea(n, d), f64(theta), f64(x), "Z", per_sample=True)
    else:
        # light cone of Z_0: the d-qubit truncation gives the exact values
        m = d
        tt = f64(theta).reshape(d, n, 3)[:, :m, :].reshape(-1)
        gt, Er = orc.gradient(orc.hea(m, d), tt, f64(x[:, :m]), "Z", per_sample=True)
        gr = np.zeros((B, d, n, 3))
        gr[:, :, :m, :] = gt.reshape(B, d, m, 3)
        gr = gr.reshape(B, -1)
    e_err = float(np.max(np.abs(E - Er)))
    g_err = float(np.max(np.abs(g - gr)))
    with capsys.disabled():
        print(f"\nmemory-saving mode n={n} d={d} c={ck}: E err {e_err:.2e}, grad err {g_err:.2e}")
    assert e_err < TOL  # the forward itself is float32 throughout
    assert g_err < BF16_TOL
