"""TF32 steps on the tcgen05 tensor cores: two consecutive middle steps of
Algorithm 2 per launch, as kind::tf32 MMAs with FP32 accumulation in TMEM.

The product stays within the TF32 bound of the oracle (FP64) -- the
operands are TF32 (unit roundoff 2^-11) and every stored intermediate is
rounded to TF32, so the relative error is at most about sqrt(d) 2^-11 --
the launch count shows that the pairs ran (fewer launches than the plan
without pairs), and the result agrees with the FP32-pipe TF32 sweep within
the same bound.  The cases cover ranks from 8 to 40 (powers of two and
not; above 32 the one-group shape) in both MMAs, pairs
starting at bits 3 and 4 (unswizzled boxes over several high-bit rows) and
at 5 and above, an output rank that is not a multiple of anything (5), a
single chunk per CTA and many chunks per CTA (the stage ring and both
epilogue groups wrap)."""
import math

import numpy as np
import pytest

import oracle
from paper_1511_06029_gb300 import inputs
from conftest import rel_l2

pytestmark = pytest.mark.gpu

PLAN_PAIRS, PLAN_NO_PAIRS = 21, 17
CASES = [
    ("profile", 12, 32, 1),
    ("profile", 12, 16, 3),
    ("profile", 16, 32, 3),
    ("ranks", [1, 2, 4, 8, 16, 16, 32, 5, 4, 2, 1], None, 2),
    ("ranks", [1, 2, 4, 8, 16, 32, 16, 32, 16, 32, 8, 4, 2, 1], None, 1),
    ("ranks", [1, 2, 4, 8, 8, 16, 8, 32, 8, 4, 2, 1], None, 2),
    ("profile", 13, 40, 2),
    ("ranks", [1, 2, 4, 8, 16, 36, 33, 39, 20, 8, 4, 2, 1], None, 2),
    ("ranks", [1, 2, 4, 8, 12, 27, 9, 31, 23, 17, 8, 4, 2, 1], None, 3),
]


@pytest.fixture(scope="module")
def qtt():
    from paper_1511_06029_gb300 import build, qtt as q
    build.build()
    q.load_library()
    return q


def _data(kind, a, b, seed):
    if kind == "profile":
        return inputs.synthetic_operator(a, b, seed)
    return inputs.random_cores(len(a) - 1, a, seed)


def _apply(qtt, op, xd, plan):
    import torch
    op.set_plan("tf32", plan)
    torch.cuda.synchronize()
    n0 = qtt.kernel_launches()
    y = op.apply(xd, compute="tf32")
    torch.cuda.synchronize()
    n = qtt.kernel_launches() - n0
    qtt.sync_status()
    return y.double().cpu().numpy(), n


@pytest.mark.parametrize("case", range(len(CASES)))
def test_tf32_pairs_match_oracle(qtt, case):
    import torch
    kind, a, b, nrhs = CASES[case]
    data = _data(kind, a, b, 11 + case)
    x = inputs.gaussian_rhs(data.N, nrhs, 21 + case)
    ref = oracle.apply(data, x)
    op = qtt.Operator(data, packs=("tf32",))
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    y_tc, n_tc = _apply(qtt, op, xd, PLAN_PAIRS)
    y_fp, n_fp = _apply(qtt, op, xd, PLAN_NO_PAIRS)
    bound = 4 * math.sqrt(data.d) * 2.0 ** -11
    assert np.isfinite(y_tc).all()
    assert rel_l2(y_tc, ref) <= bound, rel_l2(y_tc, ref)
    assert rel_l2(y_fp, ref) <= bound
    assert rel_l2(y_tc, y_fp) <= bound
    # every eligible pair replaced two launches by one
    assert n_tc < n_fp, (n_tc, n_fp)
    op.close()


def test_tf32_pairs_zero_and_repeat(qtt):
    """x = 0 gives exactly 0; the same input twice gives the same bits
    (the MMA order and the chunk schedule do not depend on timing)."""
    import torch
    data = inputs.synthetic_operator(13, 32, 4)
    op = qtt.Operator(data, packs=("tf32",))
    z = torch.zeros((2, data.N), dtype=torch.float32, device="cuda")
    y0, _ = _apply(qtt, op, z, PLAN_PAIRS)
    assert np.array_equal(y0, np.zeros_like(y0))
    x = torch.from_numpy(inputs.gaussian_rhs(data.N, 2, 9).astype(np.float32)).cuda()
    y1, _ = _apply(qtt, op, x, PLAN_PAIRS)
    y2, _ = _apply(qtt, op, x, PLAN_PAIRS)
    assert np.array_equal(y1, y2)
    op.close()


def test_tf32_pairs_linearity(qtt):
    """A (2 x) = 2 A x bit for bit: scaling by a power of two commutes with
    every TF32 rounding and every FP32 sum."""
    import torch
    data = inputs.synthetic_operator(12, 32, 8)
    op = qtt.Operator(data, packs=("tf32",))
    x = torch.from_numpy(inputs.gaussian_rhs(data.N, 1, 3).astype(np.float32)).cuda()
    y1, _ = _apply(qtt, op, x, PLAN_PAIRS)
    y2, _ = _apply(qtt, op, 2 * x, PLAN_PAIRS)
    assert np.array_equal(y2, 2 * y1)
    op.close()


def _sparse_sign_cores(ranks, heavy, seed):
    """Cores with entries in {-1, 0, 1}: for each output (b, i), one nonzero
    (a, j) at a random place (any a, so off the rank diagonal), or three for
    the cores in `heavy`.  |y| grows at most 3x per heavy core and not at all
    elsewhere, so with x in {-1, 0, 1} every intermediate is an integer below
    3^len(heavy) -- exact in TF32 (11 significant bits) -- and every FP32 sum
    of such integers is exact."""
    rng = np.random.default_rng(seed)
    cores = []
    for k in range(len(ranks) - 1):
        ra, rb = ranks[k], ranks[k + 1]
        G = np.zeros((ra, 2, 2, rb))
        for b in range(rb):
            for i in range(2):
                for _ in range(3 if k in heavy else 1):
                    G[rng.integers(ra), i, rng.integers(2), b] = rng.choice([-1.0, 1.0])
        cores.append(G)
    return inputs.QTTData(list(ranks), cores, {"kind": "sparse-sign"})


def test_tf32_pairs_integer_exact(qtt):
    """The pair kernel reproduces the oracle bit for bit when every value it
    rounds is a small integer: d = 12, ranks up to 32 (pairs (5, 6) and
    (7, 8) on the tensor cores), three signed nonzeros per output in those
    four cores."""
    import torch
    ranks = inputs.rank_profile(12, 32)
    data = _sparse_sign_cores(ranks, heavy={5, 6, 7, 8}, seed=3)
    x = np.random.default_rng(4).integers(-1, 2, size=(3, data.N)).astype(np.float64)
    ref = oracle.apply(data, x)
    assert np.abs(ref).max() < 2 ** 11 and np.abs(ref).max() >= 2
    op = qtt.Operator(data, packs=("tf32",))
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    y_tc, n_tc = _apply(qtt, op, xd, PLAN_PAIRS)
    _, n_fp = _apply(qtt, op, xd, PLAN_NO_PAIRS)
    assert n_tc < n_fp
    assert np.array_equal(y_tc, ref)
    op.close()
