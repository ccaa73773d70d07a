"""BF16 applies against the oracle run on the SAME BF16-rounded cores and
inputs, so that only the arithmetic of the GPU path separates the two: FP32
accumulation of exact BF16 products (error ~ 2r 2^-24, negligible) and the
rounding of every stored intermediate -- and of the output -- to BF16.

Bound.  A round-to-nearest BF16 rounding (8 significant bits) of a value in
[2^e, 2^(e+1)) has absolute error uniform on half an ulp, ulp = 2^(e-7), so
its relative error has RMS at most 2^-7 / sqrt(12) = 2.26e-3.  The sweep
rounds d - 1 intermediates and the BF16 output: d independent relative
perturbations, each carried to the result by the rest of the sweep with gain
about one (orthonormal-like cores, or Gaussian cores scaled to unit gain), so
the RMS relative L2 error is about sqrt(d) 2.26e-3 and the test allows three
times that: rel L2 <= 3 sqrt(d) 2^-7 / sqrt(12).  (The same model with the
cores' own rounding added explains the error measured against FP64 cores,
7.7e-3 at d = 12.)

Cases include Gaussian cores with no decay and ranks 40-56, so that every
rank plane -- and every row of the 128-row MMA tile in use -- carries signal:
a wrong plane would cost about 1 / sqrt(r) of the result, far above the
bound."""
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


def bf16_round(a):
    """Round to nearest even with 8 significant bits (BF16's precision),
    directly from FP64 -- as the library converts its cores."""
    a = np.asarray(a, dtype=np.float64)
    m, e = np.frexp(a)
    return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)


def bound(d):
    return 3.0 * math.sqrt(d) * 2.0 ** -7 / math.sqrt(12.0)


def _gaussian_unit_gain(d, ranks, seed):
    """Gaussian cores (no decay, every entry off the diagonal of the rank
    indices alike) scaled by 1 / sqrt(2 r_k), so each step keeps the
    intermediate's size."""
    rng = np.random.default_rng(seed)
    cores = [rng.standard_normal((ranks[k], 2, 2, ranks[k + 1])) / math.sqrt(2 * ranks[k])
             for k in range(d)]
    return inputs.QTTData(list(ranks), cores, {"kind": "gaussian_unit_gain"})


def _ranks_between(d, lo, hi, seed):
    rng = np.random.default_rng(seed)
    r = [1]
    for k in range(1, d):
        cap = min(2 ** k, 2 ** (d - k))
        r.append(int(min(cap, rng.integers(lo, hi + 1))))
    return r + [1]


def _check(qtt, data, nrhs, seed):
    import torch
    rounded = inputs.QTTData(list(data.ranks), [bf16_round(c) for c in data.cores])
    x = bf16_round(inputs.gaussian_rhs(data.N, nrhs, seed))
    op = qtt.Operator(data, packs=("bf16",))
    y = op.apply(torch.from_numpy(x).cuda().to(torch.bfloat16), compute="bf16")
    qtt.sync_status()
    y = y.double().cpu().numpy()
    op.close()
    ref = oracle.apply(rounded, x)
    err = rel_l2(y, ref)
    assert err <= bound(data.d), (err, bound(data.d))
    return err


@pytest.mark.parametrize("d,r,seed", [(12, 16, 2), (16, 32, 5)])
def test_bf16_synthetic_against_rounded_oracle(qtt, d, r, seed):
    _check(qtt, inputs.synthetic_operator(d, r, seed), 3, seed + 1)


@pytest.mark.parametrize("d,lo,hi,nrhs,seed", [(18, 40, 56, 2, 7), (20, 48, 48, 1, 8)])
def test_bf16_gaussian_high_ranks_against_rounded_oracle(qtt, d, lo, hi, nrhs, seed):
    data = _gaussian_unit_gain(d, _ranks_between(d, lo, hi, seed), seed)
    assert max(data.ranks) >= 40
    _check(qtt, data, nrhs, seed + 1)


def test_bf16_bound_catches_a_wrong_plane(qtt):
    """The bound is tight enough to see one rank plane gone wrong: the oracle
    on cores whose rank plane 47 of one core is zeroed differs from the
    correct result by about 1 / sqrt(48) = 0.14, more than four times the
    bound (checked on the CPU side of the same comparison)."""
    d = 14
    data = _gaussian_unit_gain(d, _ranks_between(d, 48, 48, 3), 3)
    rounded = inputs.QTTData(list(data.ranks), [bf16_round(c) for c in data.cores])
    broken = inputs.QTTData(list(data.ranks), [c.copy() for c in rounded.cores])
    k = d // 2
    broken.cores[k][:, :, :, -1] = 0.0
    x = bf16_round(inputs.gaussian_rhs(data.N, 1, 4))
    assert rel_l2(oracle.apply(broken, x), oracle.apply(rounded, x)) > 4 * bound(d)
