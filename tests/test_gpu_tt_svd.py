"""Algorithm 1 (TT-SVD) on the GPU (qtt_tt_svd) against the oracle's tt_svd:
the same ranks, reconstructions within eps ||A||_F of A and of each other,
and cores in qtt_create's layout (an operator built from them applies like
A)."""
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


def _gpu_tt_svd(qtt, A, eps):
    import torch
    ranks, flat = qtt.tt_svd(torch.from_numpy(np.ascontiguousarray(A)).cuda(), eps)
    host = flat.cpu().numpy()
    cores, off = [], 0
    for k in range(len(ranks) - 1):
        sz = 4 * ranks[k] * ranks[k + 1]
        cores.append(host[off:off + sz].reshape(ranks[k], 2, 2, ranks[k + 1]))
        off += sz
    assert off == host.size
    return oracle.Op(ranks, cores)


def _low_rank(d, rank, seed):
    rng = np.random.default_rng(seed)
    N = 1 << d
    return rng.standard_normal((N, rank)) @ rng.standard_normal((rank, N))


CASES = [
    ("laplace_8^3", lambda: inputs.laplace_volume_dense(8), 1e-8),
    ("low_rank_d8", lambda: _low_rank(8, 3, 1), 1e-10),
    ("random_d6", lambda: np.random.default_rng(2).standard_normal((64, 64)), 1e-3),
    ("kron_d7", lambda: np.kron(np.kron(np.random.default_rng(3).standard_normal((8, 8)),
                                        np.eye(4)), np.random.default_rng(4).standard_normal((4, 4))),
     1e-12),
    ("d1", lambda: np.array([[1.0, 2.0], [3.0, 4.0]]), 1e-12),
]


@pytest.mark.parametrize("name,make,eps", CASES, ids=[c[0] for c in CASES])
def test_tt_svd_matches_oracle(qtt, name, make, eps):
    A = make()
    g = _gpu_tt_svd(qtt, A, eps)
    ref = oracle.tt_svd(A, eps)
    assert g.ranks == ref.ranks
    nA = np.linalg.norm(A)
    Dg = oracle.dense(g)
    assert np.linalg.norm(Dg - A) <= eps * nA * (1 + 1e-6) + 1e-13 * nA
    assert np.linalg.norm(Dg - oracle.dense(ref)) <= 2 * eps * nA + 1e-13 * nA


def test_tt_svd_cores_build_an_operator(qtt):
    """The GPU decomposition of the 8^3 volume operator fed to qtt_create
    applies like the dense matrix (within eps ||A||_F ||x||)."""
    import torch
    A = inputs.laplace_volume_dense(8)
    g = _gpu_tt_svd(qtt, A, 1e-8)
    op = qtt.Operator(inputs.QTTData(g.ranks, g.cores))
    x = inputs.gaussian_rhs(A.shape[0], 2, 5)
    y = op.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    op.close()
    ref = x @ A.T
    assert np.linalg.norm(y - ref) <= 1e-8 * np.linalg.norm(A) * np.linalg.norm(x) * 1.01


def test_tt_svd_larger(qtt):
    """d = 11 (2048 x 2048): a sum of two Kronecker products (QTT ranks 2)
    plus noise at 1e-9; eps 1e-6 finds the ranks of the structure."""
    rng = np.random.default_rng(8)
    def kron_all(ms):
        out = np.ones((1, 1))
        for m in ms:
            out = np.kron(m, out)
        return out
    A = kron_all([rng.standard_normal((2, 2)) for _ in range(11)])
    A += kron_all([rng.standard_normal((2, 2)) for _ in range(11)])
    A += 1e-9 * np.linalg.norm(A) / 2048 * rng.standard_normal(A.shape)
    g = _gpu_tt_svd(qtt, A, 1e-6)
    ref = oracle.tt_svd(A, 1e-6)
    assert g.ranks == ref.ranks
    assert max(g.ranks) == 2
    assert rel_l2(oracle.dense(g), A) <= 1e-6


def test_tt_svd_rejects_bad_arguments(qtt):
    import torch
    with pytest.raises(qtt.QTTError):
        qtt.tt_svd(torch.zeros((3, 3), dtype=torch.float64, device="cuda"), 1e-3)
    with pytest.raises(qtt.QTTError):
        qtt.tt_svd(torch.zeros((4, 4), dtype=torch.float64, device="cuda"), -1.0)
