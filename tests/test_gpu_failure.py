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



def test_batch_dependency_wait_times_out_and_batch_survives(qtt):
    """The batch kernel's bounded dependency wait, made to run out on the
    host's say-so: the first wave starts past every item without a
    dependency, so the items it runs wait on work nobody does.  Every CTA
    gives up after 0.2 s, the status reads QTT_ERR_TIMEOUT once, and the
    next normal run is correct."""
    import time

    import numpy as np
    import torch
    items = inputs.batched_workload(count=6, seed=21, d_range=(8, 11), r_range=(4, 16),
                                    rhs_range=(1, 3))
    datas, ops, xs, ys, xh = [], [], [], [], []
    for it in items:
        data = inputs.synthetic_operator(it["d"], it["rmax"], it["op_seed"])
        x = inputs.gaussian_rhs(data.N, it["nrhs"], it["rhs_seed"])
        datas.append(data)
        xh.append(x)
        ops.append(qtt.Operator(data, packs=("f32",)))
        xs.append(torch.from_numpy(x.astype(np.float32)).cuda())
        ys.append(torch.full_like(xs[-1], float("nan")))
    B = qtt.Batch(ops, xs, ys, compute="f32")
    B.run()
    B.status()
    t0 = time.perf_counter()
    B.selftest_timeout(0.2)
    with pytest.raises(qtt.QTTError) as e:
        B.status()
    elapsed = time.perf_counter() - t0
    assert e.value.status == qtt.QTT_ERR_TIMEOUT
    assert elapsed < 5.0  # every wait ended near its 0.2 s budget
    B.status()  # reported once, then cleared
    for y in ys:
        y.fill_(float("nan"))
    B.run()
    B.status()
    torch.cuda.synchronize()
    for data, x, y in zip(datas, xh, ys):
        assert rel_l2(y.double().cpu().numpy(), oracle.apply(data, x)) <= 4 * data.d ** 0.5 * 2.0 ** -24
    with pytest.raises(qtt.QTTError) as e:
        B.selftest_timeout(0.0)
    assert e.value.status == qtt.QTT_ERR_INVALID_ARG
    B.close()
    for op in ops:
        op.close()


@pytest.mark.parametrize("compute,dtype", [("f64", "float64"), ("f32", "float32"),
                                           ("bf16", "bfloat16")])
def test_scratch_limit_chunks_rhs_bitwise_and_reports_oom(qtt, compute, dtype):
    """A cap on the library's scratch (qtt_set_scratch_limit) makes the apply
    process the right-hand sides in chunks: the result is bitwise the
    unchunked one; a cap below one right-hand side's scratch gives
    QTT_ERR_OOM and launches nothing."""
    import torch
    data = inputs.synthetic_operator(13, 16, 5)
    nrhs = 7
    x = torch.from_numpy(inputs.gaussian_rhs(data.N, nrhs, 6)).cuda().to(getattr(torch, dtype))
    op = qtt.Operator(data, packs=() if compute == "f64" else (compute,))
    esz = x.element_size()
    per_rhs = 2 * max(data.ranks[1:-1]) * data.N * esz
    try:
        y_full = op.apply(x, compute=compute)
        torch.cuda.synchronize()
        for cap_rhs in (1, 2, 3):
            qtt.set_scratch_limit(cap_rhs * per_rhs + per_rhs // 2)
            launches0 = qtt.kernel_launches()
            y = op.apply(x, compute=compute)
            torch.cuda.synchronize()
            assert qtt.kernel_launches() > launches0
            assert torch.equal(y.view(torch.uint8), y_full.view(torch.uint8))
        qtt.set_scratch_limit(per_rhs // 2)
        launches0 = qtt.kernel_launches()
        with pytest.raises(qtt.QTTError) as e:
            op.apply(x, compute=compute)
        assert e.value.status == qtt.QTT_ERR_OOM
        assert qtt.kernel_launches() == launches0
    finally:
        qtt.set_scratch_limit(0)
    y = op.apply(x, compute=compute)
    torch.cuda.synchronize()
    assert torch.equal(y.double(), y_full.double())
    op.close()


def test_destroy_waits_only_for_its_own_work(qtt):
    """qtt_destroy returns at once and holds up no other stream: an
    operator destroyed while a server request runs on another operator
    comes back in milliseconds, the request finishes correctly, and an
    operator destroyed with its own applies still queued gives correct
    results (its memory goes back to the pool after them)."""
    import time

    import numpy as np
    import torch
    # a request of a second or more on the server (d = 21, 8 right-hand sides)
    K = inputs.scaled_operator(21, 32, 5021)
    f = inputs.gaussian_rhs(K.N, 8, 77)
    small = inputs.synthetic_operator(10, 8, 3)
    op2 = qtt.Operator(small)
    xs = torch.from_numpy(inputs.gaussian_rhs(small.N, 1, 4)).cuda()
    Kop = qtt.Operator(K)
    S = qtt.Server(slots=1, kind="gmres", tol=1e-10, restart=30, precond_compute="f64")
    rid = S.submit(Kop, None, f)
    t_wait = time.perf_counter()
    while S.stats()["running"] != 1 and time.perf_counter() - t_wait < 10.0:
        time.sleep(0.005)
    time.sleep(0.05)
    y2 = op2.apply(xs)
    t0 = time.perf_counter()
    op2.close()
    t_destroy = time.perf_counter() - t0
    still_running = S.stats()["running"] == 1
    x, info, _ = S.wait(rid)
    assert still_running, "the request finished before the destroy could be timed"
    assert t_destroy < 0.1, f"qtt_destroy took {t_destroy:.3f} s while other work ran"
    assert all(st == qtt.QTT_OK and rel <= 1e-10 for (_, rel, st) in info)
    torch.cuda.synchronize()
    assert rel_l2(y2.cpu().numpy(), oracle.apply(small, xs.cpu().numpy())) <= 1e-12
    S.close()
    # destroy with the operator's own work still queued on a side stream
    big = inputs.synthetic_operator(20, 32, 9)
    opb = qtt.Operator(big)
    xb = torch.from_numpy(inputs.gaussian_rhs(big.N, 1, 10)).cuda()
    side = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(side):
        xb2 = xb.clone()
        for _ in range(6):
            outs.append(opb.apply(xb2, stream=side))
    opb.close()
    junk = qtt.Operator(inputs.synthetic_operator(20, 32, 11))  # may reuse pool memory
    junk.apply(torch.randn(big.N, dtype=torch.float64, device="cuda"))
    side.synchronize()
    torch.cuda.synchronize()
    ref = oracle.apply(big, xb.cpu().numpy())
    for y in outs:
        assert rel_l2(y.cpu().numpy(), ref) <= 1e-12
    junk.close()
    Kop.close()
