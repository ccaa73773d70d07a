"""TT rounding on the GPU (qtt_tt_round) against the oracle's tt_round
(left-to-right QR, right-to-left truncated SVDs with the Algorithm 1
threshold): the same ranks, both within eps ||t||_F of t, and t's
redundancies (t + t, the compressed product A b) removed."""
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


def _vec(ranks, seed, decay=0.0):
    """Gaussian QTT vector; decay > 0 scales rank index j of every core by
    10^(-decay j), so the unfoldings' singular values fall off."""
    rng = np.random.default_rng(seed)
    d = len(ranks) - 1
    cores = []
    for k in range(d):
        c = rng.standard_normal((ranks[k], 2, ranks[k + 1]))
        c *= 10.0 ** (-decay * np.arange(ranks[k + 1]))[None, None, :]
        cores.append(c)
    return oracle.Vec(ranks, cores)


def _gpu_round(qtt, t, n, eps):
    import torch
    flat = torch.from_numpy(np.concatenate([np.asarray(c).ravel() for c in t.cores])).cuda()
    ranks, out = qtt.tt_round(t.ranks, n, flat, eps)
    host = out.cpu().numpy()
    cores, off = [], 0
    for k in range(len(ranks) - 1):
        sz = ranks[k] * n * ranks[k + 1]
        shape = (ranks[k], 2, ranks[k + 1]) if n == 2 else (ranks[k], 2, 2, ranks[k + 1])
        cores.append(host[off:off + sz].reshape(shape))
        off += sz
    assert off == host.size
    return ranks, cores


@pytest.mark.parametrize("d,rmax,decay,eps,seed", [
    (1, 1, 0.0, 1e-6, 1),
    (6, 8, 0.3, 1e-2, 2),
    (10, 20, 0.15, 1e-6, 3),
    (12, 24, 0.1, 1e-10, 4),
    (11, 30, 0.0, 0.3, 5),
])
def test_round_vector_matches_oracle(qtt, d, rmax, decay, eps, seed):
    ranks = [min(1 << k, 1 << (d - k), rmax) for k in range(d + 1)]
    t = _vec(ranks, seed, decay)
    rg, cg = _gpu_round(qtt, t, 2, eps)
    ref = oracle.tt_round(t, eps)
    assert rg == ref.ranks
    full = oracle.vec_full(t)
    got = oracle.vec_full(oracle.Vec(rg, cg))
    nrm = np.linalg.norm(full)
    assert np.linalg.norm(got - full) <= eps * nrm * (1 + 1e-6) + 1e-13 * nrm
    assert rel_l2(got, oracle.vec_full(ref)) <= max(2 * eps, 1e-12)


def test_round_removes_exact_redundancy(qtt):
    """t + t has twice the ranks and is 2 t: rounding at 1e-12 returns t's
    ranks and 2 t."""
    d = 9
    ranks = [min(1 << k, 1 << (d - k), 6) for k in range(d + 1)]
    t = _vec(ranks, 9, 0.0)
    # the sum by rank concatenation: block-diagonal middle cores
    cores = []
    for k in range(d):
        c = t.cores[k]
        if k == 0:
            cores.append(np.concatenate([c, c], axis=2))
        elif k == d - 1:
            cores.append(np.concatenate([c, c], axis=0))
        else:
            z = np.zeros((2 * c.shape[0], 2, 2 * c.shape[2]))
            z[:c.shape[0], :, :c.shape[2]] = c
            z[c.shape[0]:, :, c.shape[2]:] = c
            cores.append(z)
    tt2 = oracle.Vec([1] + [2 * r for r in ranks[1:-1]] + [1], cores)
    rg, cg = _gpu_round(qtt, tt2, 2, 1e-12)
    assert rg == ranks
    assert rel_l2(oracle.vec_full(oracle.Vec(rg, cg)), 2 * oracle.vec_full(t)) <= 1e-12


def test_round_operator_cores(qtt):
    """A binary QTT matrix (n = 4 per core): K + K rounds back to K's ranks;
    the rounded operator applies like 2 K within the bound."""
    K = inputs.synthetic_operator(8, 12, 7)
    S = oracle.tt_sum(K, K)
    rg, cg = _gpu_round(qtt, S, 4, 1e-10)
    assert rg == K.ranks
    ref = oracle.tt_round(S, 1e-10)
    assert rg == ref.ranks
    dense = oracle.dense(oracle.Op(rg, cg))
    assert rel_l2(dense, 2 * oracle.dense(K)) <= 1e-10


def test_round_compressed_product(qtt):
    """c = A b on the GPU (ranks r s), then rounded on the GPU: the oracle's
    rounding of the oracle's product has the same ranks, and the rounded c is
    within eps of A b computed densely."""
    import torch
    d, eps = 10, 1e-7
    A = inputs.synthetic_operator(d, 16, 11)
    rb = [min(1 << k, 1 << (d - k), 8) for k in range(d + 1)]
    b = _vec(rb, 12, 0.2)
    op = qtt.Operator(A)
    flat = torch.from_numpy(np.concatenate([c.ravel() for c in b.cores])).cuda()
    pr, pc = op.apply_tt(b.ranks, flat)
    rg, out = qtt.tt_round(pr, 2, pc, eps)
    host = out.cpu().numpy()
    op.close()
    cores, off = [], 0
    for k in range(d):
        sz = rg[k] * 2 * rg[k + 1]
        cores.append(host[off:off + sz].reshape(rg[k], 2, rg[k + 1]))
        off += sz
    ref = oracle.tt_round(oracle.apply_tt(A, b), eps)
    assert rg == ref.ranks
    exact = oracle.dense(A) @ oracle.vec_full(b)
    got = oracle.vec_full(oracle.Vec(rg, cores))
    assert np.linalg.norm(got - exact) <= eps * np.linalg.norm(exact) * (1 + 1e-6)


def test_round_full_size_product(qtt):
    """d = 21: a rank-48 operator times a rank-48 QTT vector (product ranks up
    to 2304, 0.85 GB of cores) rounded at 1e-6 on the GPU; the whole rounded
    vector against the oracle's apply of A to the full b."""
    import torch
    d, eps = 21, 1e-6
    A = inputs.synthetic_operator(d, 48, 3)
    rb = [min(1 << k, 1 << (d - k), 48) for k in range(d + 1)]
    b = _vec(rb, 60, 0.05)
    op = qtt.Operator(A)
    flat = torch.from_numpy(np.concatenate([c.ravel() for c in b.cores])).cuda()
    pr, pc = op.apply_tt(b.ranks, flat)
    assert max(pr) == 2304
    rg, out = qtt.tt_round(pr, 2, pc, eps)
    del pc
    host = out.cpu().numpy()
    op.close()
    assert max(rg) < 2304
    cores, off = [], 0
    for k in range(d):
        sz = rg[k] * 2 * rg[k + 1]
        cores.append(host[off:off + sz].reshape(rg[k], 2, rg[k + 1]))
        off += sz
    exact = oracle.apply(A, oracle.vec_full(b))
    got = oracle.vec_full(oracle.Vec(rg, cores))
    assert np.linalg.norm(got - exact) <= eps * np.linalg.norm(exact) * (1 + 1e-6)


def test_round_rejects_bad_arguments(qtt):
    import torch
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    for ranks, n in (([2, 2, 1], 2), ([1, 0, 1], 2), ([1, 2, 1], 0)):
        need = sum(ranks[k] * n * ranks[k + 1] for k in range(2))
        with pytest.raises(qtt.QTTError):
            qtt.tt_round(ranks, n, x[:need], 1e-3)
    with pytest.raises(qtt.QTTError) as e:
        qtt.tt_round([1, 2, 1], 2, x, -1.0)
    assert e.value.status == qtt.QTT_ERR_INVALID_ARG
