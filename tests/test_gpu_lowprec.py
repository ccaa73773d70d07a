"""Reduced-precision applies (FP32, TF32, BF16 operands; FP32 accumulation)
against the FP64 oracle.  Exact cases are compared bitwise; otherwise the
error against the oracle is bounded by a tolerance derived from the unit
roundoff u of the storage format (BF16 u = 2^-8, TF32 operands u = 2^-11,
FP32 u = 2^-24): each of the d steps rounds its stored output once and
accumulates 2 r_k products, so the relative L2 error stays below
c sqrt(d) u with a small constant; the tests use 4 sqrt(d) u."""
import math

import numpy as np
import pytest

import oracle
from paper_1511_06029_gb300 import inputs
from conftest import rel_l2

pytestmark = pytest.mark.gpu

U = {"bf16": 2.0 ** -8, "tf32": 2.0 ** -11, "f32": 2.0 ** -24}
TORCH_IO = {"bf16": "bfloat16", "tf32": "float32", "f32": "float32"}


@pytest.fixture(scope="module")
def qtt():
    from paper_1511_06029_gb300 import build, qtt as q
    build.build()
    q.load_library()
    return q


def _run(qtt, data, x, compute, io=None):
    import torch
    io = io or TORCH_IO[compute]
    op = qtt.Operator(data, packs=(compute,))
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda().to(getattr(torch, io))
    y = op.apply(xt, compute=compute)
    out = y.double().cpu().numpy()
    op.close()
    return out


def _tf32_rne(a):
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x0FFF + ((u >> 13) & 1)) & 0xFFFFE000
    return u.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("compute", ["f32", "tf32", "bf16"])
def test_identity_rounds_input_only(qtt, compute):
    """Identity operator: y is x rounded once to the operand format."""
    import torch
    d = 11
    x = inputs.gaussian_rhs(1 << d, 2, 1).astype(np.float32)
    y = _run(qtt, inputs.identity(d), x, compute, io="float32")
    if compute == "bf16":
        expect = torch.from_numpy(x).to(torch.bfloat16).double().numpy()
    elif compute == "tf32":
        expect = _tf32_rne(x).astype(np.float64)
    else:
        expect = x.astype(np.float64)
    assert np.array_equal(y, expect)


@pytest.mark.parametrize("compute", ["f32", "tf32", "bf16"])
def test_integer_exact(qtt, compute):
    """Cores in {-1, 0, 1}, x in {-1, 0, 1}, ranks [1,2,2,1,1,1]: step k sums
    at most 2 r_k terms, so every intermediate is an integer of magnitude
    <= 2, 8, 32, 64, 128 < 2^8 -- exact in BF16, TF32 and FP32."""
    d = 5
    data = inputs.random_cores(d, [1, 2, 2, 1, 1, 1], 3, integer=True)
    x = np.random.default_rng(3).integers(-1, 2, size=(2, 1 << d)).astype(np.float64)
    ref = oracle.apply(data, x)
    assert np.abs(ref).max() < 256
    assert np.array_equal(_run(qtt, data, x, compute, io="float32"), ref)


@pytest.mark.parametrize("compute", ["f32", "tf32", "bf16"])
@pytest.mark.parametrize("d,rmax,nrhs", [(9, 7, 2), (14, 32, 1), (16, 48, 3)])
def test_error_bound(qtt, compute, d, rmax, nrhs):
    data = inputs.synthetic_operator(d, rmax, 5)
    x = inputs.gaussian_rhs(data.N, nrhs, 6)
    ref = oracle.apply(data, x)
    y = _run(qtt, data, x, compute, io="float32")
    err = rel_l2(y, ref)
    assert err <= 4 * math.sqrt(d) * U[compute], err


def test_bf16_io_and_fp64_io(qtt):
    """BF16 vectors in and out, and FP64 vectors in and out with BF16
    arithmetic, agree with the FP32-vector run within rounding."""
    data = inputs.synthetic_operator(12, 16, 7)
    x = inputs.gaussian_rhs(data.N, 1, 8)
    ref = oracle.apply(data, x)
    y_b = _run(qtt, data, x, "bf16", io="bfloat16")
    y_d = _run(qtt, data, x, "bf16", io="float64")
    for y in (y_b, y_d):
        assert rel_l2(y, ref) <= 4 * math.sqrt(12) * U["bf16"]


def test_missing_pack_is_rejected(qtt):
    import torch
    op = qtt.Operator(inputs.synthetic_operator(8, 4, 1))  # FP64 only
    x = torch.zeros(256, dtype=torch.float32, device="cuda")
    with pytest.raises(qtt.QTTError) as e:
        op.apply(x, compute="bf16")
    assert e.value.status == qtt.QTT_ERR_INVALID_ARG
    op.close()
