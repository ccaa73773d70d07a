"""qtt_apply_host: the apply with x and y in host memory.  The right-hand
sides pass through the device in chunks whose copies overlap the applies;
every right-hand side must come back bitwise as the device-side qtt_apply
gives it, padding rows of y untouched, with page-locked or pageable memory,
on the default or a caller's stream; FP64 also against the oracle."""
import math

import numpy as np
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


def _host(a, dtype, pinned, pad=0):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).to(dtype)
    if pad:
        full = torch.full((t.shape[0], t.shape[1] + pad), 7.0, dtype=dtype)
        full[:, :t.shape[1]] = t
        t = full[:, :t.shape[1]]
        if pinned:
            full = full.pin_memory()
            t = full[:, :a.shape[1]]
        return t, full
    return (t.pin_memory() if pinned else t), None


CASES = [
    # d, rmax, nrhs, chunk, compute, pinned, pad
    (12, 16, 5, 2, "f64", True, 8),     # three chunks, the last ragged; ld > N
    (11, 12, 7, 3, "bf16", True, 0),    # BF16 storage
    (12, 16, 8, 0, "f32", False, 0),    # pageable memory, chunk chosen by the library
    (10, 8, 1, 0, "f64", True, 0),      # one right-hand side: no pipeline
    (13, 24, 6, 1, "tf32", True, 4),    # one right-hand side per chunk
]


@pytest.mark.parametrize("case", CASES)
def test_host_apply_is_bitwise_the_device_apply(qtt, case):
    import torch
    d, rmax, nrhs, chunk, comp, pinned, pad = case
    data = inputs.synthetic_operator(d, rmax, d + rmax)
    x = inputs.gaussian_rhs(data.N, nrhs, d + 1)
    dt = {"f64": torch.float64, "f32": torch.float32, "tf32": torch.float32,
          "bf16": torch.bfloat16}[comp]
    op = qtt.Operator(data, packs=(() if comp == "f64" else (comp,)))
    xh, _ = _host(x, dt, pinned, pad)
    yh, yfull = _host(np.zeros_like(x), dt, pinned, pad)
    out = op.apply_host(xh, out=yh, compute=comp, chunk=chunk)
    torch.cuda.synchronize()
    qtt.sync_status()
    ref = op.apply(xh.contiguous().cuda(), compute=comp).cpu()
    op.close()
    assert out.data_ptr() == yh.data_ptr()
    a = yh.contiguous().view(torch.int16 if comp == "bf16" else
                             (torch.int64 if comp == "f64" else torch.int32))
    b = ref.view(a.dtype)
    assert torch.equal(a, b), case
    if pad:
        assert torch.all(yfull[:, data.N:] == 7.0)
    if comp == "f64":
        assert rel_l2(yh.contiguous().numpy(), oracle.apply(data, x)) <= 1e-12


def test_host_apply_on_a_caller_stream(qtt):
    import torch
    data = inputs.synthetic_operator(12, 16, 5)
    x = inputs.gaussian_rhs(data.N, 6, 9)
    op = qtt.Operator(data)
    xh = torch.from_numpy(x).pin_memory()
    s = torch.cuda.Stream()
    y = op.apply_host(xh, compute="f64", chunk=2, stream=s)
    s.synchronize()
    ref = op.apply(xh.cuda()).cpu()
    op.close()
    assert torch.equal(y, ref)


def test_host_apply_rejects_device_tensors(qtt):
    import torch
    op = qtt.Operator(inputs.synthetic_operator(6, 4, 1))
    with pytest.raises(qtt.QTTError) as e:
        op.apply_host(torch.zeros(2, 64, dtype=torch.float64, device="cuda"))
    assert e.value.status == qtt.QTT_ERR_INVALID_ARG
    x = torch.zeros(3, 64, dtype=torch.float64)
    with pytest.raises(qtt.QTTError):
        op.apply_host(x, out=x)  # x and y overlap
    op.close()
