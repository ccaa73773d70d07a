"""Edge cases of the apply paths: the smallest d in every precision, more
right-hand sides than one grid dimension holds, empty calls, and batches that
mix one-core operators with ordinary ones."""
import math

import numpy as np
import pytest

import oracle
from paper_1511_06029_gb300 import inputs
from conftest import rel_l2

pytestmark = pytest.mark.gpu

U = {"bf16": 2.0 ** -8, "tf32": 2.0 ** -11, "f32": 2.0 ** -24, "f64": 2.0 ** -52}
TORCH = {"f64": "float64", "f32": "float32", "tf32": "float32", "bf16": "bfloat16"}


@pytest.fixture(scope="module")
def qtt():
    from paper_1511_06029_gb300 import build, qtt as q
    build.build()
    q.load_library()
    return q


@pytest.mark.parametrize("compute", ["f64", "f32", "tf32", "bf16"])
@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_small_d_every_precision(qtt, compute, d):
    import torch
    data = inputs.random_cores(d, inputs.random_ranks(d, 5, d), d)
    x = inputs.gaussian_rhs(1 << d, 3, d + 1)
    packs = () if compute == "f64" else (compute,)
    op = qtt.Operator(data, packs=packs)
    xt = torch.from_numpy(x).cuda().to(getattr(torch, TORCH[compute]))
    y = op.apply(xt, compute=compute).double().cpu().numpy()
    op.close()
    ref = oracle.apply(data, xt.double().cpu().numpy())
    tol = 1e-12 if compute == "f64" else 4 * math.sqrt(d) * U[compute] * 4
    assert rel_l2(y, ref) <= tol


@pytest.mark.parametrize("compute", ["f64", "f32", "bf16"])
def test_more_rhs_than_one_grid_dimension(qtt, compute):
    """70,000 right-hand sides of length 64: the launches split the RHS over
    several grids (grid.z holds at most 65,535)."""
    import torch
    d, nrhs = 6, 70000
    data = inputs.synthetic_operator(d, 4, 3)
    x = np.random.default_rng(1).integers(-2, 3, size=(nrhs, 1 << d)).astype(np.float64)
    packs = () if compute == "f64" else (compute,)
    op = qtt.Operator(data, packs=packs)
    xt = torch.from_numpy(x).cuda().to(getattr(torch, TORCH[compute]))
    y = op.apply(xt, compute=compute).double().cpu().numpy()
    op.close()
    sel = np.r_[0:3, 65533:65540, nrhs - 3:nrhs]
    ref = oracle.apply(data, xt.double().cpu().numpy()[sel])
    tol = 1e-12 if compute == "f64" else 4 * math.sqrt(d) * U[compute] * 4
    assert rel_l2(y[sel], ref) <= tol


def test_zero_rhs_is_a_no_op(qtt):
    import ctypes
    op = qtt.Operator(inputs.synthetic_operator(5, 4, 1))
    lib = qtt.load_library()
    assert lib.qtt_apply(op.handle, ctypes.c_void_p(16), ctypes.c_void_p(4096), 0, 32, 0, 0,
                         None) == qtt.QTT_OK
    op.close()


def test_batch_with_one_core_operators(qtt):
    import torch
    specs = [(1, 1, 3), (2, 2, 2), (3, 4, 1), (9, 24, 2), (1, 1, 1), (12, 40, 3)]
    datas, ops, xs, ys, xh = [], [], [], [], []
    for n, (d, r, nrhs) in enumerate(specs):
        data = inputs.synthetic_operator(d, r, 50 + n) if d > 1 else \
            inputs.random_cores(1, [1, 1], 50 + n)
        x = inputs.gaussian_rhs(data.N, nrhs, 60 + n)
        datas.append(data)
        xh.append(x)
        ops.append(qtt.Operator(data, packs=("f32",)))
        xs.append(torch.from_numpy(x.astype(np.float32)).cuda())
        ys.append(torch.full_like(xs[-1], float("nan")))
    B = qtt.Batch(ops, xs, ys, compute="f32")
    B.run()
    B.status()
    torch.cuda.synchronize()
    for data, x, y in zip(datas, xh, ys):
        ref = oracle.apply(data, x.astype(np.float32).astype(np.float64))
        assert rel_l2(y.double().cpu().numpy(), ref) <= 4 * math.sqrt(data.d) * U["f32"] * 4
    B.close()
    for o in ops:
        o.close()
