"""qtt_apply_noalloc: the FP64 apply for callers that cannot allocate device
memory when they apply an operator (their device memory is already reserved
by another allocator, or they run a latency-bound loop in which an allocation
could synchronise the device or fail).  Its intermediate lives in a static
64 MiB device array inside the library, committed by qtt_create.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It also passes alone in a
fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1511_06029_gb300 import inputs
from conftest import rel_l2

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-12        # the FP64 tolerance of the other parity tests
LIMIT = 8_388_608      # doubles in the static array: 2 x max rank x N x nrhs


@pytest.fixture(scope="module")
def lib():
    from paper_1511_06029_gb300 import build, qtt
    build.build()
    return qtt.load_library()


def _noalloc(lib, op, x, y, nrhs, ld):
    import torch
    return lib.qtt_apply_noalloc(op.handle, ctypes.c_void_p(x.data_ptr()),
                                 ctypes.c_void_p(y.data_ptr()), nrhs, ld,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_apply_and_oracle_on_two_calls(lib):
    """Two calls in a row (different operators and inputs, the second with two
    right-hand sides): each is bitwise qtt_apply's result (the same step
    kernel runs) and within the FP64 tolerance of the CPU oracle."""
    import torch
    from paper_1511_06029_gb300 import qtt
    cases = [(inputs.synthetic_operator(16, 32, 2), 1, 3),
             (inputs.synthetic_operator(14, 32, 4), 2, 5)]
    for data, nrhs, seed in cases:
        op = qtt.Operator(data)
        xh = inputs.gaussian_rhs(data.N, nrhs, seed)
        x = torch.from_numpy(xh).cuda()
        y_ref = op.apply(x)
        y = torch.full_like(x, float("nan"))
        assert _noalloc(lib, op, x, y, nrhs, data.N) == qtt.QTT_OK, lib.qtt_last_error()
        torch.cuda.synchronize()
        assert torch.equal(y, y_ref)
        assert rel_l2(y.cpu().numpy(), oracle.apply(data, xh)) <= TOL_F64
        op.close()


def test_noalloc_at_the_exact_limit_with_padding(lib):
    """d = 16, max rank 32, two right-hand sides need exactly 2 x 32 x 2^16 x
    2 = 8,388,608 doubles -- the whole array -- and are accepted; x and y
    have a leading dimension N + 24 whose padding stays untouched."""
    import torch
    from paper_1511_06029_gb300 import qtt
    data = inputs.synthetic_operator(16, 32, 6)
    nrhs, pad = 2, 24
    assert 2 * max(data.ranks[1:-1]) * data.N * nrhs == LIMIT
    ld = data.N + pad
    op = qtt.Operator(data)
    xh = inputs.gaussian_rhs(data.N, nrhs, 7)
    xbuf = torch.full((nrhs, ld), 7.0, dtype=torch.float64, device="cuda")
    xbuf[:, :data.N] = torch.from_numpy(xh).cuda()
    ybuf = torch.full((nrhs, ld), -3.5, dtype=torch.float64, device="cuda")
    assert _noalloc(lib, op, xbuf, ybuf, nrhs, ld) == qtt.QTT_OK, lib.qtt_last_error()
    torch.cuda.synchronize()
    yref_buf = torch.empty_like(xbuf)
    y_ref = op.apply(xbuf[:, :data.N], out=yref_buf[:, :data.N])
    torch.cuda.synchronize()
    assert torch.equal(ybuf[:, :data.N], y_ref)
    assert bool((ybuf[:, data.N:] == -3.5).all())
    assert rel_l2(ybuf[:, :data.N].cpu().numpy(), oracle.apply(data, xh)) <= TOL_F64
    op.close()


def test_noalloc_allocates_nothing_once_warm(lib):
    """After one warm call, further calls change neither the library's scratch
    accounting and pool nor the device's free memory."""
    import torch
    from paper_1511_06029_gb300 import qtt
    data = inputs.synthetic_operator(15, 32, 8)
    op = qtt.Operator(data)
    x = torch.from_numpy(inputs.gaussian_rhs(data.N, 3, 9)).cuda()
    y = torch.empty_like(x)
    assert _noalloc(lib, op, x, y, 3, data.N) == qtt.QTT_OK, lib.qtt_last_error()
    torch.cuda.synchronize()
    before = (qtt.scratch_stats(), torch.cuda.mem_get_info()[0])
    for _ in range(3):
        assert _noalloc(lib, op, x, y, 3, data.N) == qtt.QTT_OK, lib.qtt_last_error()
    torch.cuda.synchronize()
    after = (qtt.scratch_stats(), torch.cuda.mem_get_info()[0])
    assert before == after
    assert rel_l2(y.cpu().numpy(), oracle.apply(data, x.cpu().numpy())) <= TOL_F64
    op.close()


def test_noalloc_rejects_sizes_beyond_the_static_area(lib):
    import torch
    from paper_1511_06029_gb300 import qtt
    data = inputs.synthetic_operator(16, 32, 2)  # 3 RHS: 1.5 x the array
    op = qtt.Operator(data)
    x = torch.zeros((3, data.N), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    launches = qtt.kernel_launches()
    assert _noalloc(lib, op, x, y, 3, data.N) == qtt.QTT_ERR_INVALID_ARG
    assert qtt.kernel_launches() == launches
    msg = lib.qtt_last_error().decode()
    assert "static area" in msg and "use qtt_apply" in msg
    op.close()
