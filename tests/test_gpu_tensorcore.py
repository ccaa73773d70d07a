"""The BF16 tensor-core step (mma.sync, FP32 accumulate) used for BF16 steps
with k >= 3 and ranks in [4, 64]: exact on integer data and within the BF16
error bound otherwise, including partial chunks and many right-hand sides."""
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


def _signed_permutation(rng):
    P = np.eye(2) if rng.integers(2) == 0 else np.array([[0.0, 1.0], [1.0, 0.0]])
    return P * rng.choice([-1.0, 1.0], size=(2, 1))


def _rank_diagonal_operator(d, r, seed):
    """A = sum over alpha of a Kronecker product of signed 2x2 permutations:
    every core is diagonal in the rank index, so every intermediate entry is
    a signed copy of an x entry and the output a sum of r of them."""
    rng = np.random.default_rng(seed)
    ranks = [1] + [r] * (d - 1) + [1]
    cores = []
    for k in range(d):
        ra, rb = ranks[k], ranks[k + 1]
        g = np.zeros((ra, 2, 2, rb))
        for a in range(ra):
            for b in range(rb):
                if ra == 1 or rb == 1 or a == b:
                    g[a, :, :, b] = _signed_permutation(rng)
        cores.append(g)
    return inputs.QTTData(ranks, cores)


@pytest.mark.parametrize("d,r,nrhs", [(7, 4, 1), (9, 8, 3), (12, 16, 2), (13, 64, 1)])
def test_integer_exact_on_tensor_cores(qtt, d, r, nrhs):
    import torch
    data = _rank_diagonal_operator(d, r, d + r)
    x = np.random.default_rng(d).integers(-1, 2, size=(nrhs, 1 << d)).astype(np.float64)
    op = qtt.Operator(data, packs=("bf16",))
    y = op.apply(torch.from_numpy(x).float().cuda(), compute="bf16").double().cpu().numpy()
    op.close()
    assert np.array_equal(y, oracle.apply(data, x))


@pytest.mark.parametrize("d,rmax,nrhs", [(10, 24, 5), (15, 40, 2), (18, 48, 1)])
def test_bf16_error_bound_tensor_cores(qtt, d, rmax, nrhs):
    import torch
    data = inputs.synthetic_operator(d, rmax, 9)
    x = inputs.gaussian_rhs(data.N, nrhs, 10)
    op = qtt.Operator(data, packs=("bf16",))
    y = op.apply(torch.from_numpy(x).to(torch.bfloat16).cuda(), compute="bf16")
    err = rel_l2(y.double().cpu().numpy(), oracle.apply(data, x))
    op.close()
    assert err <= 4 * math.sqrt(d) * 2.0 ** -8, err
