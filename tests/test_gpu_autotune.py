"""Autotuned plans on the GPU: the tuner times real configurations (tile
width, catch-up rule, forward instance) and the plans it picks are
oracle-exact, in a single-circuit step and in a persistent batch."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2603_02804_gb300 import build as qbuild
from paper_2603_02804_gb300.autotune import Autotuner
from paper_2603_02804_gb300.torch_api import Batch, Simulator

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    orc.build()


def f64(a):
    return np.asarray(a, np.float32).astype(np.float64)


def test_tuned_single_circuit_matches_oracle():
    n, d, B = 14, 6, 8
    tuner = Autotuner(path=None, max_depth=8, max_batch=8)
    cfg = tuner.choose(n, d, B)
    assert tuner.trials >= 8 and all(np.isfinite(v) for v in next(iter(tuner.timings.values())).values())
    rng = np.random.default_rng(140)
    theta = rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32)
    x = rng.uniform(0, np.pi, (B, n)).astype(np.float32)
    sim = Simulator(n, d, B, ckpt_layers=2, **cfg)
    info = sim.info()
    assert info["tile_bits"] == (cfg["tile_bits"] or 12) and info["fwd_ctas"] == cfg["fwd_ctas"]
    th, xd = torch.from_numpy(theta).cuda(), torch.from_numpy(x).cuda()
    E = sim.forward(th, xd)
    g = sim.backward(th, xd, torch.ones(B, dtype=torch.float64), per_sample=True)
    torch.cuda.synchronize()
    gr, Er = orc.gradient(orc.hea(n, d), f64(theta), f64(x), "Z", per_sample=True)
    assert np.max(np.abs(E.cpu().numpy() - Er)) < TOL
    assert np.max(np.abs(g.cpu().numpy() - gr)) < TOL


@pytest.mark.parametrize("rule,ctas", [(1, 2), (2, 3)])
def test_forced_options_match_oracle(rule, ctas):
    n, d, B = 15, 5, 40   # 40 samples x 8 tiles: a forward grid beyond two CTAs per SM
    rng = np.random.default_rng(150 + rule)
    theta = rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32)
    x = rng.uniform(0, np.pi, (B, n)).astype(np.float32)
    sim = Simulator(n, d, B, ckpt_layers=2, tile_bits=9, catch_up=rule, fwd_ctas=ctas)
    assert sim.info()["catch_up"] == rule
    th, xd = torch.from_numpy(theta).cuda(), torch.from_numpy(x).cuda()
    E = sim.forward(th, xd)
    g = sim.backward(th, xd, torch.ones(B, dtype=torch.float64), per_sample=True)
    torch.cuda.synchronize()
    gr, Er = orc.gradient(orc.hea(n, d), f64(theta), f64(x), "Z", per_sample=True)
    assert np.max(np.abs(E.cpu().numpy() - Er)) < TOL
    assert np.max(np.abs(g.cpu().numpy() - gr)) < TOL


def test_tuned_batch_matches_oracle():
    specs = [(13, 4, 3), (14, 3, 2), (10, 5, 4)]
    tuner = Autotuner(path=None, kind="batch", max_depth=4, max_batch=4)
    bt = Batch(specs, loss="sum", tile_bits=tuner)
    assert len(tuner.cache) == 2  # the two circuits wider than one tile
    rng = np.random.default_rng(13)
    thetas = [rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32) for n, d, _ in specs]
    xs = [rng.uniform(0, np.pi, (b, n)).astype(np.float32) for n, _, b in specs]
    cat = lambda a: torch.from_numpy(np.concatenate([v.reshape(-1) for v in a])).cuda()
    _, E, g = bt.train_step(cat(thetas), cat(xs))
    torch.cuda.synchronize()
    E, g = E.cpu().numpy(), g.cpu().numpy()
    for i, (n, d, b) in enumerate(specs):
        gr, Er = orc.gradient(orc.hea(n, d), f64(thetas[i]), f64(xs[i]), "Z")
        assert np.max(np.abs(E[bt.sample_off[i]:bt.sample_off[i + 1]] - Er)) < TOL
        assert np.max(np.abs(g[bt.theta_off[i]:bt.theta_off[i + 1]] - gr)) < TOL
