"""GPU parity: the CUDA path (through the C-ABI) against the oracle.

Tolerance: 1e-5 max absolute error on expectations and on per-sample
gradients dE_b/dtheta (mean-loss gradients for whole-batch checks).
"""
import multiprocessing as mp

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2603_02804_gb300 import build as qbuild
from paper_2603_02804_gb300 import qfuse, workloads
from paper_2603_02804_gb300.torch_api import HEA, QFuseFn, Simulator
from tests import oracle_proc

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    orc.build()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def gpu_run(n, d, theta, x, obs="Z", path="fused", per_sample=True, ckpt=0, tile_bits=0, dLdE=None,
            entangler="chain", gates=None, n_params=0):
    B = len(x)
    sim = Simulator(n, d, B, path=path, ckpt_layers=ckpt, tile_bits=tile_bits, obs=obs, entangler=entangler,
                    gates=gates, n_params=n_params)
    th, xd = dev(theta), dev(x)
    E = sim.forward(th, xd)
    g = sim.backward(th, xd, torch.ones(B, dtype=torch.float64) if dLdE is None else torch.as_tensor(dLdE),
                     per_sample=per_sample)
    torch.cuda.synchronize()
    return E.cpu().numpy(), g.cpu().numpy(), sim


def f64(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("path", ["fused", "per_gate"])
def test_tiny_workload(path):
    w = workloads.WORKLOADS["tiny"]
    theta, x, _ = workloads.make_inputs(w)
    E, g, _ = gpu_run(w.n, w.d, theta, x, path=path)
    gr, Er = orc.gradient(orc.hea(w.n, w.d), f64(theta), f64(x), "Z", per_sample=True)
    assert np.max(np.abs(E - Er)) < TOL
    assert np.max(np.abs(g - gr)) < TOL


@pytest.mark.parametrize("path", ["fused", "per_gate"])
def test_hea12_full_batch_per_sample(path):
    """The benchmarked launch: n=12, d=20, B=256, every sample compared."""
    w = workloads.WORKLOADS["hea12"]
    theta, x, y = workloads.make_inputs(w)
    E, g, _ = gpu_run(w.n, w.d, theta, x, path=path)
    gr, Er = orc.gradient(orc.hea(w.n, w.d), f64(theta), f64(x), "Z", per_sample=True)
    assert np.max(np.abs(E - Er)) < TOL
    assert np.max(np.abs(g - gr)) < TOL


def test_hea12_train_step_mse():
    """qf_train_step (forward + MSE loss + backward) against the oracle's
    gradient of L = mean (E - y)^2."""
    w = workloads.WORKLOADS["hea12"]
    theta, x, y = workloads.make_inputs(w)
    sim = Simulator(w.n, w.d, w.B)
    loss, E, g = sim.train_step(dev(theta), dev(x), dev(y), loss="mse")
    torch.cuda.synchronize()
    c = orc.hea(w.n, w.d)
    Er = orc.expectation(c, f64(theta), f64(x), "Z")
    gr, _ = orc.gradient(c, f64(theta), f64(x), "Z", dLdE=orc.mse_dLdE(Er, y))
    assert abs(loss.item() - orc.mse_loss(Er, y)) < TOL
    assert np.max(np.abs(g.cpu().numpy() - gr)) < TOL
    n_launch = sim.launches()
    # forward + backward with one shared parameter-table launch; E and the
    # loss are finished by the last CTA of the expectation pass, so the
    # forward's E-reduction launch is not needed either
    assert n_launch == sim.info()["launches_fwd"] + sim.info()["launches_bwd"] - 2


@pytest.mark.parametrize("n,d,B,kw", [(14, 3, 5, {}), (13, 4, 300, {}), (12, 3, 7, {"tc_path": True}),
                                       (10, 4, 9, {"tile_bits": 7})])
def test_train_step_loss_finished_in_pass(n, d, B, kw):
    """The train step's E, loss and dL/dE come from the last CTA of the
    expectation pass: several tiles per sample (n = 13, 14), more CTAs than
    SM slots (B = 300), the tensor-core forward, several samples per CTA
    (7-qubit tiles); against the oracle's MSE loss and its gradient."""
    rng = np.random.default_rng(40 + n + d + B)
    theta = rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32)
    x = rng.uniform(0, np.pi, (B, n)).astype(np.float32)
    y = rng.choice([-1.0, 1.0], B).astype(np.float32)
    sim = Simulator(n, d, B, **kw)
    loss, E, g = sim.train_step(dev(theta), dev(x), dev(y), loss="mse")
    torch.cuda.synchronize()
    c = orc.hea(n, d)
    Er = orc.expectation(c, f64(theta), f64(x), "Z")
    gr, _ = orc.gradient(c, f64(theta), f64(x), "Z", dLdE=orc.mse_dLdE(Er, f64(y)))
    assert np.max(np.abs(E.cpu().numpy() - Er)) < TOL
    assert abs(loss.item() - orc.mse_loss(Er, f64(y))) < TOL
    assert np.max(np.abs(g.cpu().numpy() - gr)) < TOL
    # a second step on the same buffers (replayed graph) gives the same numbers
    out = sim.device_outputs(B)
    r1 = [t.clone() for t in sim.train_step(dev(theta), dev(x), dev(y), loss="mse", out=out)]
    r2 = [t.clone() for t in sim.train_step(dev(theta), dev(x), dev(y), loss="mse", out=out)]
    assert all(torch.equal(a, b) for a, b in zip(r1, r2))
    assert torch.equal(r1[1], E) and torch.equal(r1[2], g)


def test_train_step_host_buffers():
    w = workloads.WORKLOADS["tiny"]
    theta, x, _ = workloads.make_inputs(w)
    sim = Simulator(w.n, w.d, w.B)
    loss, E, g = sim.train_step_host(torch.from_numpy(theta).pin_memory(), torch.from_numpy(x).pin_memory())
    gr, Er = orc.gradient(orc.hea(w.n, w.d), f64(theta), f64(x), "Z")
    assert abs(loss.item() - Er.sum()) < TOL
    assert np.max(np.abs(E.numpy() - Er)) < TOL
    assert np.max(np.abs(g.numpy() - gr)) < TOL


def test_hea16_full_batch():
    """n=16, d=100, B=128, checkpoint every 10 layers (multi-pass tiles):
    E and the per-sample gradients of all 128 samples against the oracle,
    and the MSE train step's whole-batch gradient against the oracle's."""
    w = workloads.WORKLOADS["hea16"]
    theta, x, y = workloads.make_inputs(w)
    E, g, sim = gpu_run(w.n, w.d, theta, x, ckpt=w.ckpt_layers)
    assert sim.info()["n_passes"] > 1
    gr, Er = oracle_proc.call("gradient", orc.hea(w.n, w.d), f64(theta), f64(x), "Z", per_sample=True)
    assert np.max(np.abs(E - Er)) < TOL
    assert np.max(np.abs(g - gr)) < TOL
    # the MSE loss's gradient is the dL/dE-weighted sum of the rows
    loss, E2, g2 = sim.train_step(dev(theta), dev(x), dev(y), loss="mse")
    torch.cuda.synchronize()
    dLdE = orc.mse_dLdE(Er, y)
    assert abs(loss.item() - orc.mse_loss(Er, y)) < TOL
    assert np.max(np.abs(g2.cpu().numpy() - dLdE @ gr)) < TOL


def _oracle_loss(args):
    n, d, theta, x, y = args
    E = orc.expectation(orc.hea(n, d), theta, x, "Z", threads=1)
    return orc.mse_loss(E, y)


def test_hea16_autograd_vs_central_fd():
    """autograd.Function gradient of the MSE loss vs central finite
    differences (h = 1e-3) of the float64 oracle's loss on 32 parameters."""
    w = workloads.WORKLOADS["hea16"]
    theta, x, y = workloads.make_inputs(w, B=2)
    model = HEA(w.n, w.d, max_batch=2, ckpt_layers=w.ckpt_layers, init=torch.from_numpy(theta))
    E = model(dev(x))
    loss = torch.mean((E - torch.as_tensor(y, dtype=torch.float64, device="cuda")) ** 2)
    loss.backward()
    g = model.theta.grad.double().cpu().numpy()
    # float32 cast of the gradient is exact enough: |g| <= ~1, float32 eps 6e-8
    ps = workloads.draw_fd_params(w.n_params, w.extra["fd_params"], w.extra["fd_seed"])
    h = w.extra["fd_h"]
    th64 = f64(theta)
    jobs = []
    for p in ps:
        for sgn in (+1, -1):
            t = th64.copy()
            t[p] += sgn * h
            jobs.append((w.n, w.d, t, f64(x), y))
    with mp.get_context("spawn").Pool(min(16, mp.cpu_count())) as pool:
        vals = pool.map(_oracle_loss, jobs)
    fd = (np.array(vals[0::2]) - np.array(vals[1::2])) / (2 * h)
    assert np.max(np.abs(fd - g[ps])) < TOL


def test_autograd_recomputes_when_workspace_reused():
    w = workloads.WORKLOADS["tiny"]
    theta, x, _ = workloads.make_inputs(w)
    model = HEA(w.n, w.d, max_batch=w.B, init=torch.from_numpy(theta))
    E1 = model(dev(x))
    _ = model(dev(x[::-1].copy()))  # second forward overwrites the workspace
    E1.sum().backward()
    gr, _ = orc.gradient(orc.hea(w.n, w.d), f64(theta), f64(x), "Z")
    assert np.max(np.abs(model.theta.grad.double().cpu().numpy() - gr)) < TOL


# ---------------------------------------------------------------- edge cases
@pytest.mark.parametrize("n,d,B,obs", [
    (1, 3, 5, "Z"), (2, 2, 3, "X"), (3, 4, 2, "YZ"), (4, 0, 3, "Z"), (5, 1, 1, "ZZZZZ"),
    (8, 5, 17, "IXYZ"), (9, 3, 33, "Y"), (11, 4, 3, "XIIIIIIIIIY"), (12, 3, 1, "IIIIIIIIIIIZ"),
])
def test_edge_shapes_and_observables(n, d, B, obs):
    rng = np.random.default_rng(n * 100 + d * 10 + B)
    theta = rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32)
    x = rng.uniform(0, np.pi, (B, n)).astype(np.float32)
    for path in ("fused", "per_gate"):
        E, g, _ = gpu_run(n, d, theta, x, obs=obs, path=path)
        gr, Er = orc.gradient(orc.hea(n, d), f64(theta), f64(x), obs, per_sample=True)
        assert np.max(np.abs(E - Er)) < TOL, path
        if d > 0:
            assert np.max(np.abs(g - gr)) < TOL, path


@pytest.mark.parametrize("n,d,K,ck", [(10, 6, 6, 1), (13, 4, 0, 1), (14, 3, 8, 2), (15, 5, 5, 2)])
def test_multi_pass_tiles_and_checkpoints(n, d, K, ck):
    """Tiles smaller than the state (several HBM passes), checkpoint anchors,
    a ragged batch."""
    rng = np.random.default_rng(7 * n + d)
    theta = rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32)
    x = rng.uniform(0, np.pi, (3, n)).astype(np.float32)
    E, g, sim = gpu_run(n, d, theta, x, obs="ZI" + "X" if n > 3 else "Z", tile_bits=K, ckpt=ck)
    assert sim.info()["n_passes"] > 1
    gr, Er = orc.gradient(orc.hea(n, d), f64(theta), f64(x), "ZIX", per_sample=True)
    assert np.max(np.abs(E - Er)) < TOL
    assert np.max(np.abs(g - gr)) < TOL


@pytest.mark.parametrize("seed", range(3))
def test_user_gate_lists(seed):
    """RX/RY/RZ, shared parameters, non-adjacent CZ and a ring closure."""
    rng = np.random.default_rng(40 + seed)
    n = [5, 9, 13][seed]
    n_params = 11
    rows = []
    for _ in range(60):
        k = int(rng.choice([orc.RX, orc.RY, orc.RZ, orc.CZ]))
        if k == orc.CZ:
            a, b = rng.choice(n, 2, replace=False)
            rows.append((k, int(a), int(b), -1))
        else:
            rows.append((k, int(rng.integers(n)), -1, int(rng.integers(n_params))))
    theta = rng.uniform(0, 2 * np.pi, n_params).astype(np.float32)
    x = rng.uniform(0, np.pi, (4, n)).astype(np.float32)
    c = orc.Circuit(n=n, gates=np.array(rows, np.int32), n_params=n_params)
    gr, Er = orc.gradient(c, f64(theta), f64(x), "Z", per_sample=True)
    for path in ("fused", "per_gate"):
        E, g, _ = gpu_run(n, 0, theta, x, path=path, gates=rows, n_params=n_params, ckpt=1)
        assert np.max(np.abs(E - Er)) < TOL, path
        assert np.max(np.abs(g - gr)) < TOL, path


def test_ring_entangler():
    n, d, B = 7, 4, 5
    rng = np.random.default_rng(77)
    theta = rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32)
    x = rng.uniform(0, np.pi, (B, n)).astype(np.float32)
    E, g, _ = gpu_run(n, d, theta, x, obs="ZZ", entangler="ring")
    gr, Er = orc.gradient(orc.hea(n, d, "ring"), f64(theta), f64(x), "ZZ", per_sample=True)
    assert np.max(np.abs(E - Er)) < TOL
    assert np.max(np.abs(g - gr)) < TOL


# ---------------------------------------------------------------- properties at large n
def test_n20_depth1_closed_form():
    """n = 20, d = 1, B = 64: E = cos x0 cos b0 - sin x0 cos a0 sin b0 and the
    two nonzero gradients in closed form; all other gradients vanish."""
    n, d, B = 20, 1, 64
    rng = np.random.default_rng(2020)
    theta = rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32)
    x = rng.uniform(0, np.pi, (B, n)).astype(np.float32)
    E, g, _ = gpu_run(n, d, theta, x)
    a0, b0 = f64(theta[:2])
    x0 = f64(x[:, 0])
    assert np.max(np.abs(E - (np.cos(x0) * np.cos(b0) - np.sin(x0) * np.cos(a0) * np.sin(b0)))) < TOL
    assert np.max(np.abs(g[:, 0] - np.sin(x0) * np.sin(a0) * np.sin(b0))) < TOL
    assert np.max(np.abs(g[:, 1] + np.cos(x0) * np.sin(b0) + np.sin(x0) * np.cos(a0) * np.cos(b0))) < TOL
    assert np.max(np.abs(g[:, 2:])) < TOL


def test_n20_light_cone_truncation():
    """n = 20, d = 6: E equals the oracle on the 6-qubit truncation (light
    cone of Z_0), and rotations outside the light cone have zero gradient."""
    n, d, B = 20, 6, 4
    rng = np.random.default_rng(2021)
    theta = rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32)
    x = rng.uniform(0, np.pi, (B, n)).astype(np.float32)
    E, g, sim = gpu_run(n, d, theta, x, ckpt=2)
    m = d
    tt = f64(theta).reshape(d, n, 3)[:, :m, :].reshape(-1)
    gr, Er = orc.gradient(orc.hea(m, d), tt, f64(x[:, :m]), "Z", per_sample=True)
    assert np.max(np.abs(E - Er)) < TOL
    gg = g.reshape(B, d, n, 3)
    assert np.max(np.abs(gg[:, :, :m, :].reshape(B, -1) - gr)) < TOL
    assert np.max(np.abs(gg[:, :, m:, :])) < TOL


def test_deterministic_repeat():
    w = workloads.WORKLOADS["hea12"]
    theta, x, _ = workloads.make_inputs(w, B=64)
    E1, g1, _ = gpu_run(w.n, w.d, theta, x)
    E2, g2, _ = gpu_run(w.n, w.d, theta, x)
    assert np.array_equal(E1, E2) and np.array_equal(g1, g2)


def test_fused_matches_per_gate_mid_size():
    n, d, B = 14, 12, 6
    rng = np.random.default_rng(14)
    theta = rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32)
    x = rng.uniform(0, np.pi, (B, n)).astype(np.float32)
    Ef, gf, _ = gpu_run(n, d, theta, x, obs="ZZ")
    Ep, gp, _ = gpu_run(n, d, theta, x, obs="ZZ", path="per_gate")
    assert np.max(np.abs(Ef - Ep)) < TOL
    assert np.max(np.abs(gf - gp)) < TOL


def test_workspace_and_batch_errors():
    sim = Simulator(6, 2, 4)
    th = torch.zeros(36, device="cuda")
    x = torch.zeros(4, 6, device="cuda")
    E = torch.empty(4, dtype=torch.float64, device="cuda")
    with pytest.raises(qfuse.QFError) as e:
        qfuse.qf_forward(sim.handle, th, x, 4, sim.obs, E, sim.ws, sim.ws_bytes - 1)
    assert e.value.status == qfuse.QF_ERR_WORKSPACE
    with pytest.raises(qfuse.QFError) as e:
        qfuse.qf_forward(sim.handle, th, x, 5, sim.obs, E, sim.ws, sim.ws_bytes)
    assert e.value.status == qfuse.QF_ERR_INVALID_ARG
    with pytest.raises(qfuse.QFError) as e:
        qfuse.qf_forward(sim.handle, th, x, 4, qfuse.qf_pauli(0, 1 << 7), E, sim.ws, sim.ws_bytes)
    assert e.value.status == qfuse.QF_ERR_INVALID_ARG


@pytest.mark.parametrize("seed", range(3))
def test_cnot_gate_lists(seed):
    """CNOTs fused into generic steps (and the per-gate comparator), against the oracle."""
    rng = np.random.default_rng(80 + seed)
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
    theta = rng.uniform(0, 2 * np.pi, n_params).astype(np.float32)
    x = rng.uniform(0, np.pi, (4, n)).astype(np.float32)
    c = orc.Circuit(n=n, gates=np.array(rows, np.int32), n_params=n_params)
    gr, Er = orc.gradient(c, f64(theta), f64(x), "ZX", per_sample=True)
    for path in ("fused", "per_gate"):
        E, g, _ = gpu_run(n, 0, theta, x, obs="ZX", path=path, gates=rows, n_params=n_params, ckpt=1)
        assert np.max(np.abs(E - Er)) < TOL, path
        assert np.max(np.abs(g - gr)) < TOL, path


@pytest.mark.parametrize("n", range(9, 20))
def test_round_programs_every_width(n):
    """Round programs at every width 9..19: single tiles with an overlapping
    group (9-11), and multi-tile plans whose 4-qubit groups straddle the
    progress frontier (13-15, 17-19), where the planner mixes full rounds with
    catch-up rounds of the least advanced qubits."""
    d, B = 9, 3
    rng = np.random.default_rng(9000 + n)
    theta = rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32)
    x = rng.uniform(0, np.pi, (B, n)).astype(np.float32)
    obs = "ZZ" + "I" * (n - 3) + "Z"
    E, g, sim = gpu_run(n, d, theta, x, obs=obs, ckpt=3)
    info = sim.info()
    assert info["n_eff"] == n and (n <= 12) == (info["n_passes"] == 1)
    gr, Er = orc.gradient(orc.hea(n, d), f64(theta), f64(x), obs, per_sample=True)
    assert np.max(np.abs(E - Er)) < TOL
    assert np.max(np.abs(g - gr)) < TOL


def test_train_step_cuda_graph_replay():
    """One qf_train_step captured in a CUDA graph (the C-ABI allocates and
    synchronises nothing after qf_plan) replays to the eager result bit for bit."""
    w = workloads.WORKLOADS["hea12"]
    theta, x, y = workloads.make_inputs(w, B=64)
    sim = Simulator(w.n, w.d, 64)
    th, xd, yd = dev(theta), dev(x), dev(y)
    loss_e, E_e, g_e = (t.clone() for t in sim.train_step(th, xd, yd, loss="mse"))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        sim.train_step(th, xd, yd, loss="mse")  # warm on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        out = sim.train_step(th, xd, yd, loss="mse")
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out[0], loss_e) and torch.equal(out[1], E_e) and torch.equal(out[2], g_e)


def test_device_step_graph_replay_tracks_inputs():
    """qf_train_step records its launches as a CUDA graph on the second call
    with the same buffers, batch, loss and observable, and replays it after:
    with the buffers' contents changed in place, every call must equal an
    eager step (fresh buffers each call, so no key repeats) bit for bit. With
    pass timing on, replays carry their timing events."""
    w = workloads.WORKLOADS["hea12"]
    theta, x, y = workloads.make_inputs(w, B=32)
    sim = Simulator(w.n, w.d, 32)
    ref = Simulator(w.n, w.d, 32)
    out = sim.device_outputs(32)
    th_d, x_d, y_d = dev(theta), dev(x), dev(y)
    rng = np.random.default_rng(8)
    keep = []
    for call in range(5):
        th = (theta + np.float32(0.1 * call)).astype(np.float32)
        xs = rng.uniform(0, np.pi, x.shape).astype(np.float32)
        th_d.copy_(torch.from_numpy(th))
        x_d.copy_(torch.from_numpy(xs))
        ld, Ed, gd = (t.clone() for t in sim.train_step(th_d, x_d, y_d, loss="mse", out=out))
        args = (dev(th), dev(xs), dev(y))
        res = ref.train_step(*args, loss="mse")
        keep.append((args, res))
        torch.cuda.synchronize()
        assert ld.item() == res[0].item(), call
        assert torch.equal(Ed, res[1]) and torch.equal(gd, res[2]), call
        assert sim.launches() == ref.launches()
    # call 0 ran eagerly, call 1 recorded the graph; calls 1-4 replayed it
    assert qfuse.qf_graph_stats(sim.handle) == {"recorded": 1, "replayed": 4}
    assert qfuse.qf_graph_stats(ref.handle) == {"recorded": 0, "replayed": 0}
    qfuse.qf_profile(sim.handle, True)
    seen = []
    for call in range(4):
        sim.train_step(th_d, x_d, y_d, loss="mse", out=out)
        p = qfuse.qf_profile_read(sim.handle)
        assert p["fwd_ms"] > 0 and p["bwd_ms"] > 0, (call, p)
        seen.append((p["fwd_launches"], p["bwd_launches"]))
    qfuse.qf_profile(sim.handle, False)
    assert len(set(seen)) == 1, seen
    assert qfuse.qf_graph_stats(sim.handle) == {"recorded": 2, "replayed": 7}
    torch.cuda.synchronize()
    assert torch.equal(out[2], gd)  # the same inputs as the last call above


def test_host_step_graph_replay_tracks_inputs():
    """qf_train_step_host records its device part (copies in, step, copies
    out) as a CUDA graph on the second call with the same workspace, batch,
    loss and observable, and replays it afterwards: every call must equal the
    device-buffer step on that call's inputs, bit for bit."""
    w = workloads.WORKLOADS["hea12"]
    theta, x, y = workloads.make_inputs(w, B=32)
    sim = Simulator(w.n, w.d, 32)
    out = sim.host_outputs(32)
    rng = np.random.default_rng(7)
    for call in range(4):
        th = (theta + np.float32(0.1 * call)).astype(np.float32)
        xs = rng.uniform(0, np.pi, x.shape).astype(np.float32)
        lh, Eh, gh = sim.train_step_host(torch.from_numpy(th).pin_memory(), torch.from_numpy(xs).pin_memory(),
                                         torch.from_numpy(y).pin_memory(), loss="mse", out=out)
        lh, Eh, gh = lh.clone(), Eh.clone(), gh.clone()
        ld, Ed, gd = sim.train_step(dev(th), dev(xs), dev(y), loss="mse")
        torch.cuda.synchronize()
        assert lh.item() == ld.item(), call
        assert torch.equal(Eh, Ed.cpu()) and torch.equal(gh, gd.cpu()), call
    assert qfuse.qf_graph_stats(sim.handle)["replayed"] >= 3  # host-buffer calls 1-3
