"""Recorded applies (qtt_plan_*): one qtt_apply captured as a CUDA graph and
replayed.  A replay runs the same kernels on whatever the fixed buffers hold,
so its result is bitwise that of qtt_apply with the same arguments."""
import numpy as np
import pytest

import oracle
from paper_1511_06029_gb300 import inputs
from conftest import rel_l2, laplace_qtt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qtt():
    from paper_1511_06029_gb300 import build, qtt as q
    build.build()
    q.load_library()
    return q


@pytest.mark.parametrize("compute,dtype,packs", [
    ("f64", "float64", ()), ("bf16", "bfloat16", ("bf16",)), ("f32", "float32", ("f32",))])
def test_replay_is_bitwise_the_apply(qtt, compute, dtype, packs):
    import torch
    data = inputs.synthetic_operator(12, 16, 7)
    op = qtt.Operator(data, packs=packs)
    dt = getattr(torch, dtype)
    x = torch.from_numpy(inputs.gaussian_rhs(data.N, 3, 8)).cuda().to(dt)
    y = torch.empty_like(x)
    plan = op.plan(x, y, compute=compute)
    for seed in (8, 9):  # new contents in the same buffer between replays
        x.copy_(torch.from_numpy(inputs.gaussian_rhs(data.N, 3, seed)).to(dt))
        n0 = qtt.kernel_launches()
        plan.run()
        n1 = qtt.kernel_launches()
        ref = op.apply(x, compute=compute)
        torch.cuda.synchronize()
        assert n1 > n0  # a replay counts the kernels it launches
        assert torch.equal(y, ref)
    if compute == "f64":
        assert rel_l2(y.cpu().numpy(), oracle.apply(data, x.cpu().numpy())) <= 1e-12
    plan.close()
    op.close()


def test_small_operator_replays(qtt):
    """The 8^3 volume operator (d = 9), many replays on one stream."""
    import torch
    data, _ = laplace_qtt(oracle, 8, 1e-8)
    op = qtt.Operator(data)
    x = torch.from_numpy(inputs.gaussian_rhs(data.N, 1, 1)).cuda()
    y = torch.empty_like(x)
    plan = op.plan(x, y)
    for _ in range(50):
        plan.run()
    qtt.sync_status()
    assert rel_l2(y.cpu().numpy(), oracle.apply(data, x.cpu().numpy())) <= 1e-12
    plan.close()
    op.close()


def test_plan_rejects_bad_arguments(qtt):
    import torch
    op = qtt.Operator(inputs.synthetic_operator(6, 4, 1))
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(qtt.QTTError):
        op.plan(x, x)  # x and y overlap
    y = torch.zeros(64, dtype=torch.float32, device="cuda")
    with pytest.raises(qtt.QTTError):
        op.plan(x, y)  # dtype mismatch
    op.close()
