"""Failure path of the bounded device waits, without a GPU fault: a wait on an
mbarrier that nothing arrives at gives up after its poll limit, records the
timeout in the device error word, and the context stays usable."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2603_02804_gb300 import build as qbuild
from paper_2603_02804_gb300 import qfuse
from paper_2603_02804_gb300.torch_api import Simulator

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    orc.build()


def test_bounded_wait_timeout_is_reported_and_cleared():
    torch.cuda.init()
    assert qfuse.qf_device_status() == 0
    qfuse.qf_check_bounded_wait(1000)
    assert qfuse.qf_device_status() == 1
    assert qfuse.qf_device_status() == 0  # read clears it
    with pytest.raises(qfuse.QFError):
        qfuse.qf_check_bounded_wait(0)


def test_context_usable_after_timeout():
    qfuse.qf_check_bounded_wait(100)
    assert qfuse.qf_device_status() == 1
    n, d, B = 12, 2, 3
    rng = np.random.default_rng(5)
    theta = rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32)
    x = rng.uniform(0, np.pi, (B, n)).astype(np.float32)
    sim = Simulator(n, d, B, tc_path=True)
    E = sim.forward(torch.from_numpy(theta).cuda(), torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    Er = orc.expectation(orc.hea(n, d), theta.astype(np.float64), x.astype(np.float64), "Z")
    assert np.max(np.abs(E.cpu().numpy() - Er)) < 1e-5
    assert qfuse.qf_device_status() == 0
