"""Batched persistent launch (many circuits, one kernel) against the oracle."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2603_02804_gb300 import build as qbuild
from paper_2603_02804_gb300 import workloads
from paper_2603_02804_gb300.torch_api import Batch
from tests import oracle_proc

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    orc.build()


def f64(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def make(specs, seed):
    rng = np.random.default_rng(seed)
    thetas = [rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32) for n, d, _ in specs]
    xs = [rng.uniform(0, np.pi, (B, n)).astype(np.float32) for n, _, B in specs]
    ys = [(2 * rng.integers(0, 2, B) - 1).astype(np.float32) for _, _, B in specs]
    return thetas, xs, ys


def cat(arrs):
    return torch.from_numpy(np.concatenate([a.reshape(-1) for a in arrs])).cuda()


SPECS = [(7, 3, 4), (8, 2, 5), (9, 4, 3), (12, 3, 6), (13, 2, 2), (14, 2, 3), (10, 5, 1), (11, 1, 7),
         (16, 2, 2)]


@pytest.mark.parametrize("loss", ["sum", "mse"])
def test_mixed_batch_matches_oracle(loss):
    thetas, xs, ys = make(SPECS, 5)
    bt = Batch(SPECS, loss=loss, ckpt_layers=1)
    lv, E, g = bt.train_step(cat(thetas), cat(xs), cat(ys) if loss == "mse" else None)
    torch.cuda.synchronize()
    E, g = E.cpu().numpy(), g.cpu().numpy()
    total = 0.0
    for i, (n, d, B) in enumerate(SPECS):
        c = orc.hea(n, d)
        Er = orc.expectation(c, f64(thetas[i]), f64(xs[i]), "Z")
        dLdE = orc.mse_dLdE(Er, ys[i]) if loss == "mse" else np.ones(B)
        gr, _ = orc.gradient(c, f64(thetas[i]), f64(xs[i]), "Z", dLdE=dLdE)
        s0, s1 = bt.sample_off[i], bt.sample_off[i + 1]
        t0, t1 = bt.theta_off[i], bt.theta_off[i + 1]
        assert np.max(np.abs(E[s0:s1] - Er)) < TOL, (i, n, d, B)
        assert np.max(np.abs(g[t0:t1] - gr)) < TOL, (i, n, d, B)
        total += orc.mse_loss(Er, ys[i]) if loss == "mse" else Er.sum()
    assert abs(lv.item() - total) < TOL * len(SPECS)


def test_batch_graph_replay_is_bitwise_equal():
    thetas, xs, ys = make(SPECS, 6)
    bt = Batch(SPECS, loss="mse")
    th, x, y = cat(thetas), cat(xs), cat(ys)
    ref = [t.clone() for t in bt.train_step(th, x, y)]
    out = bt.outputs()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        bt.capture(th, x, y, out, stream)
        for _ in range(3):
            bt.replay()
    stream.synchronize()
    for a, b in zip(ref, out):
        assert torch.equal(a, b)


def test_mixed512_full_launch_sampled():
    """The 512-circuit workload (n 8..18, d 10..200, B 1..64) in one launch;
    sampled circuits small enough for the oracle are checked exactly, every
    expectation is checked to lie in [-1, 1]."""
    circs = workloads.mixed_circuits(512)
    specs = [(c.n, c.d, c.B) for c in circs]
    bt = Batch(specs, loss="sum")
    lv, E, g = bt.train_step(cat([c.theta for c in circs]), cat([c.x for c in circs]))
    torch.cuda.synchronize()
    E, g = E.cpu().numpy(), g.cpu().numpy()
    assert np.all(np.abs(E) <= 1 + 1e-5)
    assert abs(lv.item() - E.sum()) < 1e-6 * max(1.0, abs(E.sum()))
    cheap = sorted(range(512), key=lambda i: (1 << circs[i].n) * circs[i].d * circs[i].B)[:6]
    for i in cheap:
        c = circs[i]
        oc = orc.hea(c.n, c.d)
        gr, Er = orc.gradient(oc, f64(c.theta), f64(c.x), "Z")
        s0, s1 = bt.sample_off[i], bt.sample_off[i + 1]
        t0, t1 = bt.theta_off[i], bt.theta_off[i + 1]
        assert np.max(np.abs(E[s0:s1] - Er)) < TOL, (i, c.n, c.d, c.B)
        assert np.max(np.abs(g[t0:t1] - gr)) < TOL, (i, c.n, c.d, c.B)


def test_mixed512_heaviest_circuits_against_oracle():
    """The most expensive circuits of the 512-circuit workload (n = 18, the
    largest depths; most of its flops are n >= 17 circuits), launched
    together as one persistent batch with the same plans and tile widths as
    the full launch, one sample each (their first), every expectation and
    gradient compared with the oracle."""
    circs = workloads.mixed_circuits(512)
    heavy = sorted(circs, key=lambda c: -(1 << c.n) * c.d * c.n)[:4]
    assert all(c.n == 18 for c in heavy) and min(c.d for c in heavy) >= 150
    specs = [(c.n, c.d, 1) for c in heavy]
    bt = Batch(specs, loss="sum")
    lv, E, g = bt.train_step(cat([c.theta for c in heavy]), cat([c.x[:1] for c in heavy]))
    torch.cuda.synchronize()
    E, g = E.cpu().numpy(), g.cpu().numpy()
    total = 0.0
    for i, c in enumerate(heavy):
        gr, Er = oracle_proc.call("gradient", orc.hea(c.n, c.d), f64(c.theta), f64(c.x[:1]), "Z")
        s0, s1 = bt.sample_off[i], bt.sample_off[i + 1]
        t0, t1 = bt.theta_off[i], bt.theta_off[i + 1]
        assert np.max(np.abs(E[s0:s1] - Er)) < TOL, (c.cid, c.n, c.d)
        assert np.max(np.abs(g[t0:t1] - gr)) < TOL, (c.cid, c.n, c.d)
        total += Er.sum()
    assert abs(lv.item() - total) < TOL * len(heavy)
