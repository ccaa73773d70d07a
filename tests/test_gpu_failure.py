"""Failure paths on the GPU, exercised without a fault.

A library kernel whose bounded device wait runs out records QTT_ERR_TIMEOUT
in a status word and returns; the host reads it at qtt_sync_status, and the
context stays usable (the wait here is on a barrier phase that nothing ever
completes, with a short budget).  (Non-convergence is a status code too:
test_gpu_solve.py.)"""
import pytest

import oracle
from paper_1511_06029_gb300 import inputs
from conftest import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qtt():
    from paper_1511_06029_gb300 import build, qtt as q
    build.build()
    q.load_library()
    return q


def test_bounded_wait_reports_timeout_and_context_survives(qtt):
    import torch
    qtt.sync_status()  # nothing pending
    qtt.selftest_wait(0.05)
    with pytest.raises(qtt.QTTError) as e:
        qtt.sync_status()
    assert e.value.status == qtt.QTT_ERR_TIMEOUT
    qtt.sync_status()  # reported once, then cleared
    # the context still computes
    data = inputs.synthetic_operator(10, 8, 3)
    x = inputs.gaussian_rhs(data.N, 1, 4)
    op = qtt.Operator(data)
    y = op.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    qtt.sync_status()
    op.close()
    assert rel_l2(y, oracle.apply(data, x)) <= 1e-12


def test_selftest_rejects_bad_budget(qtt):
    for bad in (0.0, -1.0, 11.0):
        with pytest.raises(qtt.QTTError) as e:
            qtt.selftest_wait(bad)
        assert e.value.status == qtt.QTT_ERR_INVALID_ARG

