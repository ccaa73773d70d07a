"""Parity at the full workload sizes, in the configuration the benchmark
times, on samples the oracle can afford:

* mixed-precision refinement, d = 21, r_max = 48, ||K||_2 = 0.5: the true
  residual of the GPU solution recomputed by the oracle's FP64 apply;
  with cond(I + K) <= 3 a relative residual of 3e-11 bounds the error by 1e-10;
* a d = 22 request through the solve server (GMRES(30), BF16 P, FP64
  residual), its residual recomputed by the oracle;
* the full batch of 256 uneven operators (FP32): whole outputs of the smallest
  operators and one right-hand side of a d = 20 operator against the oracle;
* the BF16 apply of the d = 21, r_max = 48 operator to 64 right-hand sides
  (head kernel, tcgen05 step pairs, single steps): two of the 64 outputs
  against the oracle's FP64 apply of the same BF16 inputs;
* the FP32, TF32 and BF16 applies of the d = 24, r_max = 32 operator to one
  right-hand side under the tuned plan: 2048 sampled outputs against the
  oracle's entry formula.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1511_06029_gb300 import inputs
from conftest import rel_l2, neumann

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qtt():
    from paper_1511_06029_gb300 import build, qtt as q
    build.build()
    q.load_library()
    return q


def _true_residual(K, f, x):
    return np.linalg.norm(f - (x + oracle.apply(K, x))) / np.linalg.norm(f)


def test_refinement_full_size(qtt):
    import torch
    K = inputs.scaled_operator(21, 48, 3)
    f = inputs.gaussian_rhs(K.N, 1, 4)
    Kg = qtt.Operator(K, packs=("bf16",))
    x, info = qtt.solve(Kg, None, torch.from_numpy(f).cuda(), kind="refine", tol=3e-11,
                        max_iter=60, precond_compute="bf16", inner_iters=6)
    Kg.close()
    x = x.cpu().numpy()[0]
    assert info[0][2] == qtt.QTT_OK
    res = _true_residual(K, f[0], x)
    assert res <= 3.1e-11, res
    assert abs(res - info[0][1]) <= 1e-3 * res + 1e-14  # the GPU's own residual agrees


def test_serving_request_full_size(qtt):
    K = inputs.scaled_operator(22, 32, 5022)
    P = neumann(oracle, K, 1e-4)
    f = inputs.gaussian_rhs(K.N, 1, 6)
    Kg, Pg = qtt.Operator(K), qtt.Operator(P, packs=("bf16",))
    S = qtt.Server(slots=2, kind="gmres", tol=3e-11, precond_compute="bf16")
    x, info, _ = S.wait(S.submit(Kg, Pg, f))
    S.close()
    Kg.close(), Pg.close()
    assert info[0][2] == qtt.QTT_OK
    assert _true_residual(K, f[0], x[0]) <= 3.1e-11


def test_batched_full_size_samples(qtt):
    import torch
    items = inputs.batched_workload()
    datas, ops, xs, ys = [], [], [], []
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4)
    for it in items:
        data = inputs.synthetic_operator(it["d"], it["rmax"], it["op_seed"])
        datas.append(data)
        ops.append(qtt.Operator(data, packs=("f32",)))
        x = torch.randn(it["nrhs"], data.N, device="cuda", dtype=torch.float32, generator=gen)
        xs.append(x)
        ys.append(torch.full_like(x, float("nan")))
    B = qtt.Batch(ops, xs, ys, compute="f32")
    B.run()
    B.status()
    torch.cuda.synchronize()
    order = sorted(range(len(items)), key=lambda i: items[i]["d"] * 64 + items[i]["nrhs"])
    samples = [(i, None) for i in order[:4]]
    big = max(range(len(items)), key=lambda i: (items[i]["d"], items[i]["rmax"]))
    samples.append((big, 0))
    for i, c in samples:
        x = xs[i].double().cpu().numpy()
        y = ys[i].double().cpu().numpy()
        if c is not None:
            x, y = x[c:c + 1], y[c:c + 1]
        ref = oracle.apply(datas[i], x)
        assert rel_l2(y, ref) <= 4 * math.sqrt(datas[i].d) * 2.0 ** -24, (i, items[i])
    B.close()
    for o in ops:
        o.close()


def test_bf16_apply_full_size_samples(qtt):
    import torch
    data = inputs.synthetic_operator(21, 48, 3)
    x = torch.from_numpy(inputs.gaussian_rhs(data.N, 64, 4)).to(torch.bfloat16).cuda()
    op = qtt.Operator(data, packs=("bf16",))
    y = op.apply(x, compute="bf16")
    qtt.sync_status()
    op.close()
    for c in (0, 63):
        xc = x[c:c + 1].double().cpu().numpy()
        ref = oracle.apply(data, xc)
        err = rel_l2(y[c:c + 1].double().cpu().numpy(), ref)
        assert err <= 4 * math.sqrt(data.d) * 2.0 ** -8, (c, err)


@pytest.mark.parametrize("compute", ["f32", "tf32", "bf16"])
def test_low_precision_apply_d24_sampled_outputs(qtt, compute):
    """d = 24, r_max = 32 in FP32, TF32 and BF16, in the launch configuration
    the benchmark times (the plan the library's tuner picks for one
    right-hand side).  x has 6 nonzeros (values representable in the input
    type), so each output is y(i) = sum_s x(j_s) A(i, j_s); 2048 sampled
    outputs are checked against the oracle's entry formula within the
    arithmetic's bound 4 sqrt(d) u."""
    import torch
    dt = {"f32": torch.float32, "tf32": torch.float32, "bf16": torch.bfloat16}[compute]
    u = {"f32": 2.0 ** -24, "tf32": 2.0 ** -11, "bf16": 2.0 ** -8}[compute]
    op_data = inputs.synthetic_operator(24, 32, 2)
    N = op_data.N
    rng = np.random.default_rng(91)
    J = rng.choice(N, size=6, replace=False)
    c = torch.from_numpy(rng.standard_normal(6)).to(dt)
    x = torch.zeros(1, N, dtype=dt, device="cuda")
    x[0, torch.from_numpy(J).cuda()] = c.cuda()
    op = qtt.Operator(op_data, packs=(compute,))
    op.autotune(1, compute, reps=1)
    y = op.apply(x, compute=compute)
    qtt.sync_status()
    y = y[0].double().cpu().numpy()
    op.close()
    I = np.concatenate([rng.integers(0, N, size=2040),
                        [0, N - 1, 1, N - 2, 2 ** 23, 4321, 2 ** 23 - 1, 7]])
    cd = c.double().numpy()
    ref = np.zeros(I.shape[0])
    for s in range(6):
        ref += cd[s] * oracle.entries(op_data, I, np.full(I.shape[0], J[s]))
    err = rel_l2(y[I], ref)
    assert err <= 4 * math.sqrt(op_data.d) * u, (compute, err)
