"""Exact QTT arithmetic on the GPU: the core-wise product of two QTT
matrices (qtt_op_product) and the weighted sum (qtt_tt_sum) bitwise against
the oracle's tt_product and tt_sum (both evaluate each entry the same way),
and the Neumann preconditioner round(I - K + K^2) built on the GPU against
the one the oracle builds."""
import numpy as np
import pytest

import oracle
from paper_1511_06029_gb300 import inputs
from conftest import rel_l2, neumann, neumann_unrounded

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qtt():
    from paper_1511_06029_gb300 import build, qtt as q
    build.build()
    q.load_library()
    return q


def _split(ranks, flat, n=4):
    cores, off = [], 0
    for k in range(len(ranks) - 1):
        sz = n * ranks[k] * ranks[k + 1]
        cores.append(flat[off:off + sz].reshape(ranks[k], 2, 2, ranks[k + 1]))
        off += sz
    assert off == flat.size
    return cores


@pytest.mark.parametrize("d,ra,rb", [(1, [1, 1], [1, 1]), (5, [1, 3, 4, 2, 3, 1],
                                                           [1, 2, 5, 5, 1, 1])])
def test_op_product_bitwise(qtt, d, ra, rb):
    A = inputs.random_cores(d, ra, 3)
    B = inputs.random_cores(d, rb, 4)
    oa, ob = qtt.Operator(A), qtt.Operator(B)
    ranks, flat = qtt.op_product(oa, ob)
    ref = oracle.tt_product(A, B)
    assert ranks == list(ref.ranks)
    got = _split(ranks, flat.cpu().numpy())
    for g, r in zip(got, ref.cores):
        assert np.array_equal(g, r)
    oa.close()
    ob.close()


def test_tt_sum_bitwise_and_coefficients(qtt):
    import torch
    d = 6
    A = inputs.random_cores(d, [1, 2, 3, 3, 2, 2, 1], 5)
    B = inputs.random_cores(d, [1, 3, 1, 4, 2, 1, 1], 6)
    dev = lambda T: torch.from_numpy(T.flat()).cuda()
    ranks, flat = qtt.tt_sum([(1.0, A.ranks, dev(A)), (1.0, B.ranks, dev(B))], 4)
    ref = oracle.tt_sum(A, B)
    assert ranks == list(ref.ranks)
    for g, r in zip(_split(ranks, flat.cpu().numpy()), ref.cores):
        assert np.array_equal(g, r)
    # 2 A - 0.5 B + I against the dense combination
    I = inputs.identity(d)
    ranks, flat = qtt.tt_sum([(2.0, A.ranks, dev(A)), (-0.5, B.ranks, dev(B)),
                              (1.0, I.ranks, dev(I))], 4)
    D = oracle.dense(oracle.Op(ranks, _split(ranks, flat.cpu().numpy())))
    ref = 2 * oracle.dense(A) - 0.5 * oracle.dense(B) + np.eye(1 << d)
    assert rel_l2(D, ref) <= 1e-15


def test_neumann_preconditioner_on_the_gpu(qtt):
    """P = round(I - K + K^2, 1e-4) from the GPU's product, sum and rounding
    (d = 10, r = 32, ||K||_2 = 0.5): the unrounded sum is bitwise the
    oracle's, the oracle's rounding gives the same ranks, and both rounded
    matrices lie within 1e-4 ||P||_F of the unrounded P (dense check)."""
    import torch
    K0 = inputs.synthetic_operator(10, 32, 77)
    K = inputs.scaled_operator(10, 32, 77, sigma=np.linalg.norm(oracle.dense(K0), 2))
    Kop = qtt.Operator(K)
    r2, k2 = qtt.op_product(Kop, Kop)
    ident = torch.from_numpy(np.tile(np.eye(2).ravel(), K.d)).cuda()
    kflat = torch.from_numpy(K.flat()).cuda()
    rs, s = qtt.tt_sum([(1.0, [1] * (K.d + 1), ident), (-1.0, K.ranks, kflat), (1.0, r2, k2)], 4)
    U = neumann_unrounded(oracle, K)
    assert rs == list(U.ranks)
    for g, r in zip(_split(rs, s.cpu().numpy()), U.cores):
        assert np.array_equal(g, r)
    rp, pcores = qtt.neumann_preconditioner(Kop, 1e-4)
    ref = neumann(oracle, K, 1e-4)
    assert rp == list(ref.ranks)
    DU = oracle.dense(U)
    nU = np.linalg.norm(DU)
    for D in (oracle.dense(oracle.Op(rp, pcores)), oracle.dense(ref)):
        assert np.linalg.norm(D - DU) <= 1e-4 * nU * (1 + 1e-9)
    Kop.close()


def test_op_product_rejects_mismatched(qtt):
    a = qtt.Operator(inputs.random_cores(3, [1, 2, 2, 1], 1))
    b = qtt.Operator(inputs.random_cores(4, [1, 2, 2, 2, 1], 2))
    with pytest.raises(qtt.QTTError):
        qtt.op_product(a, b)
    a.close()
    b.close()
