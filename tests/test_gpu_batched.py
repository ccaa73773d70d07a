"""Batched uneven operators in one persistent launch per wave, replayed from a
captured CUDA graph: every operator's result against the FP64 oracle, within
the FP32/TF32 error bound 4 sqrt(d) u used for the single applies."""
import math

import numpy as np
import pytest

import oracle
from paper_1511_06029_gb300 import inputs
from conftest import rel_l2

pytestmark = pytest.mark.gpu

U = {"tf32": 2.0 ** -11, "f32": 2.0 ** -24}


@pytest.fixture(scope="module")
def qtt():
    from paper_1511_06029_gb300 import build, qtt as q
    build.build()
    q.load_library()
    return q


def _batch(count, seed, d_range=(5, 12), r_range=(3, 40), rhs_range=(1, 5)):
    return inputs.batched_workload(count=count, seed=seed, d_range=d_range, r_range=r_range,
                                   rhs_range=rhs_range)


def _setup(qtt, items, compute):
    import torch
    datas, ops, xs, ys, xh = [], [], [], [], []
    for it in items:
        data = inputs.synthetic_operator(it["d"], it["rmax"], it["op_seed"])
        x = inputs.gaussian_rhs(data.N, it["nrhs"], it["rhs_seed"])
        datas.append(data)
        xh.append(x)
        ops.append(qtt.Operator(data, packs=(compute,)))
        xs.append(torch.from_numpy(x.astype(np.float32)).cuda())
        ys.append(torch.full_like(xs[-1], float("nan")))
    return datas, ops, xs, ys, xh


@pytest.mark.parametrize("compute", ["f32", "tf32"])
@pytest.mark.parametrize("budget", [0, 16 << 20])
def test_batch_matches_oracle(qtt, compute, budget):
    """24 operators (d 5..12, r_max 3..40, 1-5 RHS); budget 0 = one wave per
    rank class, 16 MiB = waves within the budget."""
    import torch
    items = _batch(24, 11)
    datas, ops, xs, ys, xh = _setup(qtt, items, compute)
    B = qtt.Batch(ops, xs, ys, compute=compute, mem_budget=budget)
    info = B.info()
    # at least one wave per rank class (largest rank <= 16, <= 24, <= 32,
    # <= 48); a budget may split a class further.  TF32 operators whose apply
    # runs tcgen05 pairs leave the waves for that path.
    cls = {0 if r <= 16 else 1 if r <= 24 else 2 if r <= 32 else 3
           for r in (max(dt.ranks) for dt in datas)}
    if compute == "f32":
        # d 5..12: no operator reaches the direct-apply size (d >= 16)
        assert info["direct_ops"] == 0
        assert info["waves"] >= len(cls) and (budget != 0 or info["waves"] == len(cls))
    else:
        assert info["direct_ops"] >= 1 and info["waves"] >= 1
    for _ in range(2):  # replaying the graph gives the same result
        B.run()
        B.status()
        torch.cuda.synchronize()
        for data, x, y in zip(datas, xh, ys):
            err = rel_l2(y.double().cpu().numpy(), oracle.apply(data, x))
            assert err <= 4 * math.sqrt(data.d) * U[compute], (data.d, data.ranks, err)
    B.close()
    for o in ops:
        o.close()


def test_tf32_batch_on_tensor_cores(qtt):
    """A TF32 batch whose operators all have middle ranks 8..32 runs every one
    of them on the tcgen05 pair path (no wave); each result matches the
    oracle within the TF32 bound and a second run gives the same bits."""
    import torch
    items = _batch(8, 13, d_range=(10, 14), r_range=(9, 32), rhs_range=(1, 4))
    datas, ops, xs, ys, xh = _setup(qtt, items, "tf32")
    B = qtt.Batch(ops, xs, ys, compute="tf32")
    info = B.info()
    assert info["direct_ops"] == len(items) and info["waves"] == 0
    B.run()
    B.status()
    torch.cuda.synchronize()
    first = [y.clone() for y in ys]
    for data, x, y in zip(datas, xh, ys):
        err = rel_l2(y.double().cpu().numpy(), oracle.apply(data, x))
        assert err <= 4 * math.sqrt(data.d) * U["tf32"], (data.d, data.ranks, err)
    B.run()
    B.status()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(first, ys))
    B.close()
    for o in ops:
        o.close()


def test_batch_autotune_and_single_apply_agree(qtt):
    """After autotuning the tile variant, the batch agrees with the FP32
    single applies of the same operators within FP32 rounding."""
    import torch
    items = _batch(10, 12, d_range=(6, 11), r_range=(8, 40), rhs_range=(1, 3))
    datas, ops, xs, ys, xh = _setup(qtt, items, "f32")
    B = qtt.Batch(ops, xs, ys, compute="f32")
    v, t = B.autotune(reps=1)
    assert v % 100 in (2, 4) and 1 <= (v // 100) % 100 <= 64 and v // 10000 in (2, 3) and t > 0
    B.run()
    B.status()
    torch.cuda.synchronize()
    for op, x, y, data in zip(ops, xs, ys, datas):
        y1 = op.apply(x, compute="f32")
        assert rel_l2(y.double().cpu().numpy(), y1.double().cpu().numpy()) <= \
            4 * math.sqrt(data.d) * U["f32"]
    B.close()
    for o in ops:
        o.close()


def test_batch_rejects_bad_input(qtt):
    import torch
    data = inputs.synthetic_operator(6, 4, 1)
    op64 = qtt.Operator(data)  # no FP32 pack
    x = torch.zeros(64, dtype=torch.float32, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(qtt.QTTError) as e:
        qtt.Batch([op64], [x], [y], compute="f32")
    assert e.value.status == qtt.QTT_ERR_INVALID_ARG
    with pytest.raises(qtt.QTTError) as e:
        qtt.Batch([op64], [x], [y], compute="bf16")
    assert e.value.status == qtt.QTT_ERR_UNSUPPORTED
    op64.close()


def test_batch_odd_leading_dimension(qtt):
    """Outputs with a leading dimension that is not a multiple of 4 (vector
    stores must fall back to scalar ones)."""
    import torch
    items = _batch(4, 13, d_range=(6, 9), r_range=(8, 20), rhs_range=(2, 3))
    datas, ops, xs, ys = [], [], [], []
    for it in items:
        data = inputs.synthetic_operator(it["d"], it["rmax"], it["op_seed"])
        N = data.N
        datas.append(data)
        ops.append(qtt.Operator(data, packs=("f32",)))
        x = torch.from_numpy(inputs.gaussian_rhs(N, it["nrhs"], it["rhs_seed"]).astype(np.float32))
        xbig = torch.zeros((it["nrhs"], N + 3), dtype=torch.float32, device="cuda")
        xbig[:, 1:N + 1] = x.cuda()
        xs.append(xbig[:, 1:N + 1])  # ld = N + 3, rows start at odd offsets
        big = torch.full((it["nrhs"], N + 3), float("nan"), dtype=torch.float32, device="cuda")
        ys.append(big[:, 1:N + 1])
    B = qtt.Batch(ops, xs, ys, compute="f32")
    B.run()
    B.status()
    torch.cuda.synchronize()
    for data, x, y in zip(datas, xs, ys):
        err = rel_l2(y.double().cpu().numpy(), oracle.apply(data, x.double().cpu().numpy()))
        assert err <= 4 * math.sqrt(data.d) * U["f32"]
    B.close()
    for o in ops:
        o.close()


@pytest.mark.parametrize("compute,d_range", [("f32", (12, 17)), ("tf32", (6, 13))])
def test_batch_run_host_is_bitwise_the_device_run(qtt, compute, d_range):
    """qtt_batch_run_host (vectors in page-locked host memory, copies
    overlapping the run) gives every operator bitwise what qtt_batch_run
    gives it; the batches hold both wave operators and directly applied ones
    (FP32: d >= 16; TF32: operators with a tcgen05 pair), and two host runs
    in a row agree."""
    import torch
    items = _batch(12, 21, d_range=d_range, r_range=(3, 32), rhs_range=(1, 3))
    datas, ops, xs, ys, xh = _setup(qtt, items, compute)
    B = qtt.Batch(ops, xs, ys, compute=compute)
    info = B.info()
    assert info["direct_ops"] >= 1 and info["waves"] >= 1, info
    B.run()
    B.status()
    torch.cuda.synchronize()
    ref = [y.cpu().clone() for y in ys]
    xs_host = [torch.from_numpy(x.astype(np.float32)).pin_memory() for x in xh]
    for _ in range(2):
        for y in ys:
            y.fill_(float("nan"))
        ys_host = [torch.full(x.shape, float("nan"), dtype=torch.float32).pin_memory()
                   for x in xs_host]
        B.run_host(xs_host, ys_host)
        B.status()
        torch.cuda.synchronize()
        for a, b in zip(ys_host, ref):
            assert torch.equal(a.view(torch.int32), b.contiguous().view(torch.int32))
    with pytest.raises(qtt.QTTError):
        B.run_host(xs_host[:-1], ys_host[:-1])
    B.close()
    for o in ops:
        o.close()
