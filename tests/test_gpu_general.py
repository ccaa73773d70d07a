"""General mode sizes, rectangular and transposed applies on the GPU
(qtt_gcreate / qtt_gapply): the mixed-radix sweep against the oracle's
apply_general (itself pinned by mixed-radix brute force), element by element
within the FP64 tolerance of the binary applies."""
import numpy as np
import pytest

import oracle
from paper_1511_06029_gb300 import inputs
from conftest import rel_l2

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-12


@pytest.fixture(scope="module")
def qtt():
    from paper_1511_06029_gb300 import build, qtt as q
    build.build()
    q.load_library()
    return q


def _cores(m, n, rmax, seed):
    """Gaussian cores (r_k, m_k, n_k, r_{k+1}), variance 1/(r_k m_k n_k)
    scaled so every step keeps the intermediate's size of order one."""
    rng = np.random.default_rng(seed)
    d = len(m)
    ranks = [1]
    for k in range(1, d):
        left = int(np.prod([m[l] * n[l] for l in range(k)]))
        right = int(np.prod([m[l] * n[l] for l in range(k, d)]))
        ranks.append(min(rmax, left, right))
    ranks.append(1)
    return [rng.standard_normal((ranks[k], m[k], n[k], ranks[k + 1]))
            / np.sqrt(ranks[k] * n[k]) for k in range(d)]


CASES = [
    ("rect_mixed", [3, 2, 4, 1, 5], [2, 5, 3, 4, 1], 6, 1),
    ("square_4x4", [4] * 7, [4] * 7, 16, 3),
    ("tall", [3] * 6, [2] * 6, 9, 2),
    ("wide", [2] * 6, [3] * 6, 9, 2),
    ("modes_16", [16, 1, 16, 8], [8, 16, 2, 16], 12, 2),
    ("single_core", [5], [7], 1, 3),
]


@pytest.mark.parametrize("name,m,n,rmax,nrhs", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("transpose", [False, True])
def test_general_apply_matches_oracle(qtt, name, m, n, rmax, nrhs, transpose):
    import torch
    cores = _cores(m, n, rmax, 11 + len(name))
    A = qtt.GeneralOperator(cores)
    assert A.rows == int(np.prod(m)) and A.cols == int(np.prod(n))
    nin = A.rows if transpose else A.cols
    x = np.random.default_rng(5).standard_normal((nrhs, nin))
    y = A.apply(torch.from_numpy(x).cuda(), transpose=transpose).cpu().numpy()
    ref_cores = [np.transpose(c, (0, 2, 1, 3)) for c in cores] if transpose else cores
    ref = oracle.apply_general(ref_cores, x)
    assert y.shape == ref.shape
    assert rel_l2(y, ref) <= TOL_F64
    A.close()


def test_binary_modes_agree_with_the_binary_operator_and_its_transpose(qtt):
    """m = n = 2 everywhere: the general operator is the binary one; its
    apply matches qtt_apply, its transposed apply the oracle's transpose."""
    import torch
    data = inputs.synthetic_operator(14, 24, 8)
    G = qtt.GeneralOperator(data.cores)
    B = qtt.Operator(data)
    x = torch.from_numpy(inputs.gaussian_rhs(data.N, 3, 9)).cuda()
    yg = G.apply(x)
    yb = B.apply(x)
    assert rel_l2(yg.cpu().numpy(), yb.cpu().numpy()) <= TOL_F64
    yt = G.apply(x, transpose=True).cpu().numpy()
    assert rel_l2(yt, oracle.apply(oracle.transpose(data), x.cpu().numpy())) <= TOL_F64
    # <y, A x> = <A^T y, x>
    ya = yb.cpu().numpy()
    lhs = np.sum(x.cpu().numpy() * ya)
    rhs = np.sum(yt * x.cpu().numpy())
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(ya) * np.linalg.norm(x.cpu().numpy()) * 10
    assert G.flops() == pytest.approx(B.flops(), rel=1e-15)
    G.close()
    B.close()


def test_general_leading_dimensions_and_padding(qtt):
    import torch
    m, n = [3, 4, 2], [2, 3, 5]
    cores = _cores(m, n, 5, 4)
    A = qtt.GeneralOperator(cores)
    nrhs, padx, pady = 3, 7, 5
    x = np.random.default_rng(1).standard_normal((nrhs, A.cols))
    xb = torch.full((nrhs, A.cols + padx), 9.0, dtype=torch.float64, device="cuda")
    xb[:, :A.cols] = torch.from_numpy(x).cuda()
    yb = torch.full((nrhs, A.rows + pady), -2.0, dtype=torch.float64, device="cuda")
    A.apply(xb[:, :A.cols], out=yb[:, :A.rows])
    torch.cuda.synchronize()
    assert rel_l2(yb[:, :A.rows].cpu().numpy(), oracle.apply_general(cores, x)) <= TOL_F64
    assert bool((yb[:, A.rows:] == -2.0).all())
    A.close()


def test_general_rejects_bad_arguments(qtt):
    import torch
    with pytest.raises(qtt.QTTError) as e:
        qtt.GeneralOperator([np.ones((1, 17, 2, 1))])
    assert e.value.status == qtt.QTT_ERR_INVALID_ARG
    A = qtt.GeneralOperator(_cores([3, 2], [2, 2], 4, 1))
    with pytest.raises(qtt.QTTError):
        A.apply(torch.zeros(A.rows, dtype=torch.float64, device="cuda"))  # wrong length
    launches = qtt.kernel_launches()
    buf = torch.zeros(A.rows + A.cols, dtype=torch.float64, device="cuda")
    with pytest.raises(qtt.QTTError) as e:
        A.apply(buf[:A.cols], out=buf[1:1 + A.rows])  # x and y overlap
    assert e.value.status == qtt.QTT_ERR_INVALID_ARG
    assert qtt.kernel_launches() == launches
    A.close()


def test_general_large(qtt):
    """4 x 4 modes, d = 9 (262,144 x 262,144), ranks up to 32: the whole
    output against the oracle's mixed-radix sweep."""
    import torch
    m = n = [4] * 9
    cores = _cores(m, n, 32, 21)
    A = qtt.GeneralOperator(cores)
    x = np.random.default_rng(2).standard_normal((1, A.cols))
    y = A.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel_l2(y, oracle.apply_general(cores, x)) <= TOL_F64
    A.close()
