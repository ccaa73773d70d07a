"""The compressed matrix-vector product c = A b (Sec. 4.2) on the GPU
(qtt_apply_tt) against the oracle's apply_tt, core by core; c's full vector
against the dense product for small d; full size (d = 21, ranks 48 x 48);
argument checks."""
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


def _vec(d, ranks, seed):
    rng = np.random.default_rng(seed)
    return oracle.Vec(ranks, [rng.standard_normal((ranks[k], 2, ranks[k + 1])) for k in range(d)])


def _gpu_product(qtt, A, b):
    import torch
    op = qtt.Operator(A)
    flat = torch.from_numpy(np.concatenate([c.ravel() for c in b.cores])).cuda()
    ranks, out = op.apply_tt(b.ranks, flat)
    host = out.cpu().numpy()
    qtt.sync_status()
    op.close()
    cores, off = [], 0
    for k in range(A.d):
        n = ranks[k] * 2 * ranks[k + 1]
        cores.append(host[off:off + n].reshape(ranks[k], 2, ranks[k + 1]))
        off += n
    assert off == host.size
    return oracle.Vec(ranks, cores)


def _close_to_oracle(A, b, c):
    """Every entry of c equals the oracle's up to the rounding of one
    two-term sum.  The oracle forms fl(fl(a_0 b_0) + fl(a_1 b_1)), within
    u (2 |a_0 b_0| + 2 |a_1 b_1|) of the exact sum; the GPU forms
    fma(a_1, b_1, fl(a_0 b_0)), within u (|a_0 b_0| + |a_0 b_0 + a_1 b_1|)
    <= 2 u (|a_0 b_0| + |a_1 b_1|); so they differ by at most 4 u (|a_0 b_0|
    + |a_1 b_1|) = 2^-51 (|a_0 b_0| + |a_1 b_1|), u = 2^-53."""
    ref = oracle.apply_tt(A, b)
    assert c.ranks == ref.ranks
    for k in range(A.d):
        GA, Gb = np.asarray(A.cores[k]), b.cores[k]
        mag = np.einsum("aijc,bje->abice", np.abs(GA), np.abs(Gb)).reshape(ref.cores[k].shape)
        assert np.all(np.abs(c.cores[k] - ref.cores[k]) <= 2.0 ** -51 * mag), k


@pytest.mark.parametrize("d,ra,rb,seed", [
    (1, [1, 1], [1, 1], 1),
    (4, [1, 2, 3, 2, 1], [1, 3, 1, 2, 1], 2),
    (7, [1, 2, 4, 7, 5, 3, 2, 1], [1, 2, 4, 4, 4, 2, 2, 1], 3),     # ragged ranks
    (10, [1, 2, 4, 8, 16, 16, 16, 8, 4, 2, 1], [1, 2, 4, 8, 8, 8, 8, 8, 4, 2, 1], 4),
])
def test_compressed_product_matches_oracle(qtt, d, ra, rb, seed):
    A = inputs.random_cores(d, ra, seed)
    b = _vec(d, rb, seed + 50)
    c = _gpu_product(qtt, A, b)
    _close_to_oracle(A, b, c)
    if d <= 10:
        ref = oracle.dense(A) @ oracle.vec_full(b)
        assert rel_l2(oracle.vec_full(c), ref) <= 1e-13


def test_compressed_product_full_size(qtt):
    """d = 21 operator of ranks up to 48 times a vector of ranks up to 48:
    product ranks up to 2304, 0.85 GB of output cores, every entry checked."""
    A = inputs.synthetic_operator(21, 48, 3)
    rb = [min(1 << k, 1 << (21 - k), 48) for k in range(22)]
    b = _vec(21, rb, 60)
    c = _gpu_product(qtt, A, b)
    _close_to_oracle(A, b, c)


def test_compressed_product_rejects_bad_vectors(qtt):
    import torch
    A = inputs.random_cores(3, [1, 2, 2, 1], 5)
    op = qtt.Operator(A)

    def cores_for(ranks):
        n = sum(2 * ranks[k] * ranks[k + 1] for k in range(3))
        return torch.zeros(n, dtype=torch.float64, device="cuda")

    # sized correctly for the ranks given, so the library's checks decide
    for ranks in ([2, 2, 2, 1], [1, 2, 2, 2], [1, 0, 2, 1], [1, 5000, 2, 1]):
        with pytest.raises(qtt.QTTError):
            op.apply_tt(ranks, cores_for(ranks))
    with pytest.raises(qtt.QTTError):
        op.apply_tt([1, 2, 2, 1], cores_for([1, 2, 2, 1])[:-1])  # wrong number of elements
    ranks, out = op.apply_tt([1, 2, 2, 1], cores_for([1, 2, 2, 1]))
    assert ranks == [1, 4, 4, 1] and out.numel() == 2 * (4 + 16 + 4)
    op.close()
