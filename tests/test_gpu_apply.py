"""GPU parity of the FP64 apply (qtt_apply, qtt_residual) against the CPU
oracle, through the C-ABI.  Tolerance: relative L2 <= 1e-12 for FP64; bitwise
where the arithmetic is exact (identity, integer cores)."""
import numpy as np
import pytest

import oracle
from paper_1511_06029_gb300 import inputs
from conftest import rel_l2, laplace_qtt

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-12


@pytest.fixture(scope="module")
def qtt():
    from paper_1511_06029_gb300 import build, qtt as q
    build.build()
    q.load_library()
    return q


def _gpu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _apply(q, op_data, x, **kw):
    op = q.Operator(op_data)
    y = op.apply(_gpu(x), **kw).cpu().numpy()
    op.close()
    return y


def test_hand_example_bitwise(qtt):
    from test_oracle_pins import _read_hand_example
    op, A, x, y = _read_hand_example()
    assert np.array_equal(_apply(qtt, op, x), y)


@pytest.mark.parametrize("d", [1, 2, 5, 13])
def test_identity_bitwise(qtt, d):
    x = inputs.gaussian_rhs(1 << d, 3, d)
    assert np.array_equal(_apply(qtt, inputs.identity(d), x), x)


@pytest.mark.parametrize("d,rmax,seed", [(3, 3, 1), (9, 5, 2), (12, 4, 3), (14, 9, 4)])
def test_integer_exact_bitwise(qtt, d, rmax, seed):
    op = inputs.random_cores(d, inputs.random_ranks(d, rmax, seed), seed, integer=True)
    x = np.random.default_rng(seed).integers(-8, 9, size=(2, 1 << d)).astype(np.float64)
    assert np.array_equal(_apply(qtt, op, x), oracle.apply(op, x))


@pytest.mark.parametrize("d,rmax,seed,nrhs", [
    (1, 1, 1, 1), (2, 2, 2, 3), (5, 7, 3, 2), (8, 13, 4, 1), (11, 37, 5, 2),
    (13, 20, 6, 5)])
def test_random_ranks_ragged(qtt, d, rmax, seed, nrhs):
    """Ranks not multiples of the 8-rank block, pair counts not multiples of
    the 128-pair tile, several right-hand sides."""
    op = inputs.random_cores(d, inputs.random_ranks(d, rmax, seed), seed)
    x = inputs.gaussian_rhs(1 << d, nrhs, seed + 7)
    assert rel_l2(_apply(qtt, op, x), oracle.apply(op, x)) <= TOL_F64


def test_laplace_volume_8cubed(qtt):
    """The 8^3 Laplace volume operator compressed by TT-SVD at 1e-8: GPU vs
    oracle on the same cores to 1e-12, and vs the dense 512 x 512 product
    within the TT-SVD bound eps ||A||_F ||x||."""
    op, A = laplace_qtt(oracle, 8, 1e-8)
    x = inputs.gaussian_rhs(512, 1, 1)
    y = _apply(qtt, op, x)
    assert rel_l2(y, oracle.apply(op, x)) <= TOL_F64
    assert np.linalg.norm(y[0] - A @ x[0]) <= 1e-8 * np.linalg.norm(A) * np.linalg.norm(x)


@pytest.mark.parametrize("d,rmax", [(16, 32), (18, 32)])
def test_synthetic_full_parity(qtt, d, rmax):
    op = inputs.synthetic_operator(d, rmax, 2)
    x = inputs.gaussian_rhs(op.N, 1, 3)
    assert rel_l2(_apply(qtt, op, x), oracle.apply(op, x)) <= TOL_F64


def test_leading_dimension_and_many_rhs(qtt):
    import torch
    op_data = inputs.synthetic_operator(10, 16, 5)
    N = op_data.N
    X = inputs.gaussian_rhs(N + 24, 4, 6)  # rows padded: ld = N + 24
    xt = _gpu(X)[:, :N]
    yt = torch.full((4, N + 24), 7.0, dtype=torch.float64, device="cuda")[:, :N]
    op = qtt.Operator(op_data)
    op.apply(xt, out=yt)
    y = yt.cpu().numpy()
    assert rel_l2(y, oracle.apply(op_data, X[:, :N])) <= TOL_F64
    # the padding after each right-hand side is untouched
    full = yt.as_strided((4, N + 24), (N + 24, 1)).cpu().numpy()
    assert np.all(full[:, N:] == 7.0)
    op.close()


def test_residual_fused(qtt):
    """r = f - (a x + K x) in FP64 with the subtraction in the last step."""
    K = inputs.synthetic_operator(12, 16, 8).scaled(1e4)
    f = inputs.gaussian_rhs(K.N, 3, 9)
    x = inputs.gaussian_rhs(K.N, 3, 10)
    op = qtt.Operator(K)
    r = op.residual(_gpu(f), _gpu(x), a=1.25).cpu().numpy()
    op.close()
    expect = f - (1.25 * x + oracle.apply(K, x))
    assert rel_l2(r, expect) <= TOL_F64


def test_full_size_sampled_outputs(qtt):
    """d = 24, r_max = 32 (the full-size FP64 workload) in the launch
    configuration the benchmark times.  x has 6 nonzeros, so every output is
    y(i) = sum_s x(j_s) A(i, j_s); 2048 sampled outputs are checked against
    entries from the oracle's entry formula."""
    import torch
    op_data = inputs.synthetic_operator(24, 32, 2)
    N = op_data.N
    rng = np.random.default_rng(77)
    J = rng.choice(N, size=6, replace=False)
    c = rng.standard_normal(6)
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    x[torch.from_numpy(J).cuda()] = torch.from_numpy(c).cuda()
    op = qtt.Operator(op_data)
    y = op.apply(x).cpu().numpy()
    op.close()
    I = np.concatenate([rng.integers(0, N, size=2040), [0, N - 1, 1, N - 2, 2 ** 23, 12345, 2 ** 23 - 1, 5]])
    ref = np.zeros(I.shape[0])
    for s in range(6):
        ref += c[s] * oracle.entries(op_data, I, np.full(I.shape[0], J[s]))
    assert rel_l2(y[I], ref) <= TOL_F64


def test_full_size_adjoint_identity(qtt):
    """<u, A v> = <A^T u, v> at d = 24 with dense random u, v (A^T built by
    the oracle's core transpose)."""
    import torch
    op_data = inputs.synthetic_operator(24, 32, 2)
    opT_data = oracle.transpose(op_data)
    u, v = inputs.gaussian_rhs(op_data.N, 2, 11)
    A = qtt.Operator(op_data)
    AT = qtt.Operator(opT_data)
    ut, vt = _gpu(u), _gpu(v)
    Av = A.apply(vt)
    ATu = AT.apply(ut)
    lhs = float(torch.dot(ut, Av))
    rhs = float(torch.dot(ATu, vt))
    scale = min(float(torch.linalg.norm(ut) * torch.linalg.norm(Av)),
                float(torch.linalg.norm(ATu) * torch.linalg.norm(vt)))
    A.close()
    AT.close()
    assert abs(lhs - rhs) <= 1e-12 * scale


def test_bad_arguments(qtt):
    import torch
    op = qtt.Operator(inputs.synthetic_operator(6, 4, 1))
    x = torch.zeros(2, 64, dtype=torch.float64, device="cuda")
    with pytest.raises(qtt.QTTError) as e:
        op.apply(x, out=x)  # aliasing
    assert e.value.status == qtt.QTT_ERR_INVALID_ARG
    with pytest.raises(qtt.QTTError):
        op.apply(torch.zeros(2, 63, dtype=torch.float64, device="cuda"))
    op.close()
