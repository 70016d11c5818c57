"""The checkpoint memory model (Sec. 3.4) against the values the paper prints
(tests/golden/memory_model.txt), and the memory-fitting planner."""
import math
import os

import pytest

from paper_2603_02804_gb300 import build as qbuild
from paper_2603_02804_gb300 import qfuse

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "memory_model.txt")


@pytest.fixture(scope="module", autouse=True)
def lib():
    qbuild.build()
    return qfuse.load()


def rows():
    out = []
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        f = line.split()
        out.append((f[0], float(f[1]), float(f[2]), float(f[3]), f[4], float(f[5])))
    return out


@pytest.mark.parametrize("case,k,d,value,qty,tol", rows())
def test_paper_printed_values(case, k, d, value, qty, tol):
    if qty == "ceil_60_over_9":
        assert math.ceil(60 / 9) == value
        return
    m, b_best = qfuse.qf_mem_model(k, d, 1.0)
    assert abs(b_best - value) <= tol, (case, b_best)
    # the minimiser really minimises k b + d / b
    m_best, _ = qfuse.qf_mem_model(k, d, b_best)
    for b in (0.5 * b_best, 0.9 * b_best, 1.1 * b_best, 2 * b_best):
        assert qfuse.qf_mem_model(k, d, b)[0] >= m_best - 1e-9
    assert abs(m_best - 2 * math.sqrt(k * d)) < 1e-9 * m_best  # Eqs. 6 and 8: 2 sqrt(k d)


def test_eq9_expression():
    # Eq. 9: M(b) = (7 b + 1000 / b) x 8 x 2^20 bytes
    for b in (1, 10, 12, 20, 100):
        states, _ = qfuse.qf_mem_model(7, 1000, b)
        assert states * 8 * 2 ** 20 == pytest.approx((7 * b + 1000 / b) * 8 * 2 ** 20)


def test_plan_fit_picks_smallest_interval_that_fits():
    h = qfuse.qf_hea_create(12, 40)
    try:
        ws = {}
        for c in (1, 2, 5, 10, 20, 40):
            ws[c] = qfuse.qf_plan(h, 8, ckpt_layers=c, host_only=True)
        assert ws[1] > ws[5] > ws[40]
        budget = ws[10] + 1
        c, got = qfuse.qf_plan_fit(h, 8, budget, host_only=True)
        assert got <= budget
        assert c <= 10
        if c > 1:
            assert qfuse.qf_plan(h, 8, ckpt_layers=c - 1, host_only=True) > budget
        with pytest.raises(qfuse.QFError) as e:
            qfuse.qf_plan_fit(h, 8, 1000, host_only=True)
        assert e.value.status == qfuse.QF_ERR_WORKSPACE
    finally:
        qfuse.qf_circuit_destroy(h)
