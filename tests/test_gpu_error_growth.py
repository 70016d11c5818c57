"""Error of the float32 fused path against the float64 oracle as depth grows
beyond 100 layers: n = 12 with checkpoints every 10 layers, and n = 20 through
the plan of the large workload's epoch (the n = 20 oracle runs in a spawned
worker process). Reported, with a loose bound: the
parity bar of 1e-5 applies up to 100 layers."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2603_02804_gb300 import build as qbuild
from paper_2603_02804_gb300 import qfuse, workloads
from paper_2603_02804_gb300.torch_api import Simulator
from tests import oracle_proc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    orc.build()


def test_error_growth_beyond_100_layers(capsys):
    n, B = 12, 2
    rows = []
    for d in (20, 100, 200, 500, 1000):
        theta = workloads.draw_theta(3 * n * d, 1000 + d)
        x = workloads.draw_x(B, n, 2000 + d)
        sim = Simulator(n, d, B, ckpt_layers=10)
        th, xd = torch.from_numpy(theta).cuda(), torch.from_numpy(x).cuda()
        E = sim.forward(th, xd)
        g = sim.backward(th, xd, torch.ones(B, dtype=torch.float64), per_sample=True)
        torch.cuda.synchronize()
        gr, Er = orc.gradient(orc.hea(n, d), theta.astype(np.float64), x.astype(np.float64), "Z",
                              per_sample=True)
        e_err = float(np.max(np.abs(E.cpu().numpy() - Er)))
        g_err = float(np.max(np.abs(g.cpu().numpy() - gr)))
        rows.append((d, e_err, g_err))
        if d <= 100:
            assert e_err < 1e-5 and g_err < 1e-5, (d, e_err, g_err)
        else:
            assert e_err < 1e-3 and g_err < 1e-3, (d, e_err, g_err)
    with capsys.disabled():
        print("\nerror growth, n=12, checkpoint every 10 layers (max abs vs float64 oracle):")
        for d, e, g in rows:
            print(f"  d={d:5d}  E {e:.2e}  grad {g:.2e}")


def test_error_growth_n20_epoch_plan(capsys):
    """n = 20 on one sample of the large workload, through the plan its epoch
    uses (checkpoint interval from memory for a micro-batch of 100): d = 100
    meets the 1e-5 bar; d = 250 is reported, with a loose bound. (The error
    at the full d = 1000 is measured by the benchmark on the same sample.)"""
    n, B = 20, 1
    w = workloads.WORKLOADS["hea20"]
    theta_all, x, _ = workloads.make_inputs(w, B=B)
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    h = qfuse.qf_hea_create(n, 1000)
    try:
        c, _ = qfuse.qf_plan_fit(h, 100, int(0.8 * free), host_only=True)
    finally:
        qfuse.qf_circuit_destroy(h)
    rows = []
    for d in (100, 250):
        theta = np.ascontiguousarray(theta_all[:3 * n * d])
        sim = Simulator(n, d, B, ckpt_layers=c)
        th, xd = torch.from_numpy(theta).cuda(), torch.from_numpy(x).cuda()
        E = sim.forward(th, xd)
        g = sim.backward(th, xd, torch.ones(B, dtype=torch.float64), per_sample=True)
        torch.cuda.synchronize()
        passes = sim.info()["n_passes"]
        del sim
        gr, Er = oracle_proc.call("gradient", orc.hea(n, d), theta.astype(np.float64), x.astype(np.float64), "Z",
                                  per_sample=True)
        e_err = float(np.max(np.abs(E.cpu().numpy() - Er)))
        g_err = float(np.max(np.abs(g.cpu().numpy() - gr)))
        rows.append((d, passes, e_err, g_err))
        if d <= 100:
            assert e_err < 1e-5 and g_err < 1e-5, (d, e_err, g_err)
        else:
            assert e_err < 1e-3 and g_err < 1e-3, (d, e_err, g_err)
    with capsys.disabled():
        print(f"\nerror growth, n=20, checkpoint every {c} layers (the epoch's plan), one sample "
              f"(max abs vs float64 oracle):")
        for d, p, e, g in rows:
            print(f"  d={d:5d}  passes {p:4d}  E {e:.2e}  grad {g:.2e}")
