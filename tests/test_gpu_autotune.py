"""The fusion-plan tuner (qtt_apply_autotune, qtt_apply_set/get_plan) and
the batch's rank-class waves: every candidate plan computes the product
(within the precision's bound of the oracle), the tuner keeps one of them,
a cached choice is reused without timing, and bad plan codes are refused."""
import math

import numpy as np
import pytest

import oracle
from paper_1511_06029_gb300 import inputs
from conftest import rel_l2

pytestmark = pytest.mark.gpu

BF16_PLANS = [21, 29, 19, 17, 20]  # default, two groups, mma.sync pairs, no pairs, no fusion
F32_PLANS = [21, 5, 20, 4]         # default, unstaged, no fusion, neither
TF32_PLANS = [21, 17, 5, 20, 4]    # default (tcgen05 pairs), no pairs, unstaged, no fusion, neither


@pytest.fixture(scope="module")
def qtt():
    from paper_1511_06029_gb300 import build, qtt as q
    build.build()
    q.load_library()
    return q


@pytest.mark.parametrize("compute,plans,tol", [("bf16", BF16_PLANS, 4 * 2.0 ** -8),
                                               ("f32", F32_PLANS, 4 * 2.0 ** -24),
                                               ("tf32", TF32_PLANS, 4 * 2.0 ** -11)])
def test_every_plan_computes_the_product(qtt, compute, plans, tol):
    import torch
    data = inputs.synthetic_operator(16, 32, 2)
    op = qtt.Operator(data, packs=(compute,))
    x = inputs.gaussian_rhs(data.N, 3, 5)
    dt = torch.bfloat16 if compute == "bf16" else torch.float32
    xd = torch.from_numpy(x).cuda().to(dt)
    ref = oracle.apply(data, xd.double().cpu().numpy())
    bound = tol * math.sqrt(data.d)
    for p in plans:
        op.set_plan(compute, p)
        assert op.get_plan(compute) == p
        y = op.apply(xd, compute=compute).double().cpu().numpy()
        qtt.sync_status()
        assert rel_l2(y, ref) <= bound, (p, rel_l2(y, ref))
    chosen, sec = op.autotune(3, compute)
    assert chosen in plans and sec > 0
    assert op.get_plan(compute) == chosen
    op.close()


def test_plan_cache_and_bad_codes(qtt, tmp_path):
    data = inputs.synthetic_operator(14, 16, 3)
    op = qtt.Operator(data, packs=("bf16",))
    cache = str(tmp_path / "plans.json")
    p1, s1 = op.autotune(2, "bf16", cache=cache)
    assert s1 is not None
    op.set_plan("bf16", 16)
    p2, s2 = op.autotune(2, "bf16", cache=cache)  # reused, not timed
    assert p2 == p1 and s2 is None and op.get_plan("bf16") == p1
    for bad in (-1, 32, 6, 7):  # pairs = 3 does not exist
        with pytest.raises(qtt.QTTError) as e:
            op.set_plan("bf16", bad)
        assert e.value.status == qtt.QTT_ERR_INVALID_ARG
    op.close()


def test_batch_waves_follow_rank_classes(qtt):
    """Operators of ranks <= 16 and of ranks 40 in one batch: they run in
    separate waves (each sized for its own class) and every result matches
    the oracle."""
    import torch
    items = [(10, 8), (11, 40), (10, 16), (12, 40), (9, 12)]
    datas, ops, xs, ys, xh = [], [], [], [], []
    for i, (d, r) in enumerate(items):
        data = inputs.synthetic_operator(d, r, 50 + i)
        x = inputs.gaussian_rhs(data.N, 2, 60 + i)
        datas.append(data)
        xh.append(x)
        ops.append(qtt.Operator(data, packs=("f32",)))
        xs.append(torch.from_numpy(x.astype(np.float32)).cuda())
        ys.append(torch.full_like(xs[-1], float("nan")))
    B = qtt.Batch(ops, xs, ys, compute="f32")
    assert B.info()["waves"] >= 2
    B.run()
    B.status()
    torch.cuda.synchronize()
    for data, x, y in zip(datas, xh, ys):
        assert rel_l2(y.double().cpu().numpy(), oracle.apply(data, x)) <= 4 * math.sqrt(data.d) * 2.0 ** -24
    B.close()
    for o in ops:
        o.close()
