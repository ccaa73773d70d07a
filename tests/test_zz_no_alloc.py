"""qtt_apply_noalloc: the FP64 apply for callers that cannot allocate device
memory when they apply an operator (their device memory is already reserved
by another allocator, or they run a latency-bound loop in which an allocation
could synchronise the device or fail).  Its intermediate lives in a static
64 MiB device array inside the library.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It also passes alone in a
fresh process (the first call sets the array's address up itself).
"""
import ctypes

import numpy as np
import pytest

from paper_1511_06029_gb300 import inputs
from conftest import rel_l2

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-12  # the FP64 tolerance of the other parity tests


@pytest.fixture(scope="module")
def lib():
    from paper_1511_06029_gb300 import build, qtt
    build.build()
    return qtt.load_library()


def _noalloc(lib, op, x, y):
    import torch
    nrhs = 1 if x.dim() == 1 else x.shape[0]
    st = lib.qtt_apply_noalloc(op.handle, ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(y.data_ptr()), nrhs, op.N,
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


def test_noalloc_matches_apply_on_two_calls(lib):
    """Two calls in a row (different inputs, the second with two right-hand
    sides) give the same result as qtt_apply, within the FP64 tolerance."""
    import torch
    from paper_1511_06029_gb300 import qtt
    cases = [(inputs.synthetic_operator(16, 32, 2), 1, 3),
             (inputs.synthetic_operator(14, 32, 4), 2, 5)]
    for data, nrhs, seed in cases:
        op = qtt.Operator(data)
        x = torch.from_numpy(inputs.gaussian_rhs(data.N, nrhs, seed)).cuda()
        y_ref = op.apply(x)
        y = torch.full_like(x, float("nan"))
        assert _noalloc(lib, op, x, y) == qtt.QTT_OK, lib.qtt_last_error()
        torch.cuda.synchronize()
        assert rel_l2(y.cpu().numpy(), y_ref.cpu().numpy()) <= TOL_F64
        op.close()


def test_noalloc_rejects_sizes_beyond_the_static_area(lib):
    import torch
    from paper_1511_06029_gb300 import qtt
    data = inputs.synthetic_operator(18, 32, 2)  # needs 2 x 32 x 2^18 doubles > 2^23
    op = qtt.Operator(data)
    x = torch.zeros(data.N, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    assert _noalloc(lib, op, x, y) == qtt.QTT_ERR_INVALID_ARG
    msg = lib.qtt_last_error().decode()
    assert "static area" in msg and "use qtt_apply" in msg
    op.close()
