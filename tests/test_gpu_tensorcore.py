"""The BF16 tensor-core steps (FP32 accumulate): the single mma.sync step
used for k >= 3 and ranks in [4, 64], and the fused pair of steps (TMA +
tcgen05 with a TMEM accumulator for k >= 4, N >= 256, r_k % 8 == 0 and ranks
in [8, 56] -- position runs of 16, 32 or 64 with the matching swizzle --
else mma.sync for ranks in [16, 48]), k + 2 < d.  Exact on integer data and within
the BF16 error bound otherwise, including partial chunks, uneven rank
profiles and many right-hand sides."""
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


def _rank_diagonal_operator(d, r, seed, ranks=None):
    """A = sum over alpha of a Kronecker product of signed 2x2 permutations:
    every core is diagonal in the rank index, so every intermediate entry is
    a signed copy of an x entry and the output a sum of at most r of them."""
    rng = np.random.default_rng(seed)
    ranks = ranks or [1] + [r] * (d - 1) + [1]
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


@pytest.mark.parametrize("ranks,nrhs", [
    ([1, 2, 4, 16, 16, 16, 1], 3),                           # d=6: one fused pair, 16 quads
    ([1, 2, 4, 8, 17, 33, 20, 1], 2),                        # d=7: ragged ranks, 32 quads
    ([1, 2, 4, 8, 48, 24, 48, 40, 19, 16, 9, 1], 4),         # d=11: pairs (3,4),(5,6),(7,8)
    ([1, 2, 4, 8, 16, 48, 48, 48, 48, 48, 48, 48, 48, 1], 1),
    ([1, 2, 4, 8, 8, 8, 9, 64, 64, 64, 12, 1], 2),           # ranks 8 and 64 (M = 128 full)
    ([1, 2, 4, 8, 16, 32, 56, 40, 56, 24, 8, 8, 1], 3),      # TMA pairs at k = 6, 8
    ([1, 2, 4, 8, 8, 8, 8, 8, 8, 8, 8, 1], 2),               # TMA pairs of rank 8
    ([1, 2, 4, 6, 16, 24, 16, 32, 8, 1], 3),                 # TMA pairs at k = 4 and 6
])
def test_fused_pairs_integer_exact(qtt, ranks, nrhs):
    """Uneven rank profiles through the fused pair kernel: every padded
    shape (2 r rounded up to 16) from 32 to 96 on both sides of the pair."""
    import torch
    d = len(ranks) - 1
    data = _rank_diagonal_operator(d, 0, sum(ranks), ranks=ranks)
    x = np.random.default_rng(d).integers(-1, 2, size=(nrhs, 1 << d)).astype(np.float64)
    op = qtt.Operator(data, packs=("bf16",))
    y = op.apply(torch.from_numpy(x).float().cuda(), compute="bf16").double().cpu().numpy()
    qtt.sync_status()  # no bounded wait of a tensor-core kernel gave up
    op.close()
    assert np.array_equal(y, oracle.apply(data, x))


@pytest.mark.parametrize("ranks,nrhs", [
    ([1, 2, 4, 8, 16, 32, 32, 32, 32, 32, 32, 32, 16, 8, 8, 8, 4, 2, 1], 3),   # four groups
    ([1, 2, 4, 8, 16, 48, 48, 48, 48, 40, 32, 24, 16, 16, 8, 8, 4, 2, 1], 2),  # two and four
])
def test_fused_pairs_integer_exact_many_chunks(qtt, ranks, nrhs):
    """d = 18: thousands of 64-quad chunks, so every CTA of the pair kernel
    cycles each ring stage, TMEM buffer and epilogue group many times."""
    import torch
    d = len(ranks) - 1
    data = _rank_diagonal_operator(d, 0, sum(ranks) + 1, ranks=ranks)
    x = np.random.default_rng(d + 1).integers(-1, 2, size=(nrhs, 1 << d)).astype(np.float64)
    op = qtt.Operator(data, packs=("bf16",))
    y = op.apply(torch.from_numpy(x).float().cuda(), compute="bf16").double().cpu().numpy()
    qtt.sync_status()
    op.close()
    assert np.array_equal(y, oracle.apply(data, x))


GROUPS_CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1511_06029_gb300 import inputs, qtt
data = inputs.synthetic_operator(18, 32, 31)
x = torch.from_numpy(inputs.gaussian_rhs(data.N, 3, 32)).to(torch.bfloat16).cuda()
op = qtt.Operator(data, packs=("bf16",))
np.save(sys.argv[2], op.apply(x, compute="bf16").float().cpu().numpy())
op.close()
"""


def test_epilogue_group_count_is_bitwise_neutral(qtt, tmp_path):
    """Four epilogue groups (ranks <= 32) against two (QTT_TC2_GROUPS=2): the
    group count only schedules, so the results agree bit for bit."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for groups in ("4", "2"):
        f = tmp_path / f"y{groups}.npy"
        env = dict(os.environ, QTT_TC2_GROUPS=groups)
        r = subprocess.run([sys.executable, "-c", GROUPS_CHILD, root, str(f)], env=env,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        outs.append(np.load(f))
    assert np.array_equal(outs[0].view(np.uint32), outs[1].view(np.uint32))


@pytest.mark.parametrize("case,nrhs", [
    ([1, 2, 4, 16, 16, 16, 1], 2), ([1, 3, 8, 24, 40, 31, 48, 17, 1], 3), (11, 3), (20, 2)])
def test_fused_pairs_bf16_error_bound(qtt, case, nrhs):
    import torch
    if isinstance(case, list):
        data = inputs.random_cores(len(case) - 1, case, 21)
    else:
        data = inputs.synthetic_operator(case, 48, 21)
    d = data.d
    x = inputs.gaussian_rhs(data.N, nrhs, 22)
    op = qtt.Operator(data, packs=("bf16",))
    y = op.apply(torch.from_numpy(x).to(torch.bfloat16).cuda(), compute="bf16")
    err = rel_l2(y.double().cpu().numpy(), oracle.apply(data, x))
    op.close()
    assert err <= 4 * math.sqrt(d) * 2.0 ** -8, err


@pytest.mark.parametrize("d,rmax,nrhs", [(12, 16, 2), (14, 48, 1), (16, 32, 3)])
def test_bench_byte_accounting_matches_the_launches(qtt, d, rmax, nrhs):
    """The benchmark's HBM roofline counts the bytes of the launches the
    library makes (head kernel, fused pairs, single steps); its plan must be
    the dispatch the library actually performs, launch for launch."""
    import torch
    import bench
    data = inputs.synthetic_operator(d, rmax, 5)

    class Spec:
        pass
    run = Spec()
    run.data, run.nrhs, run.compute = data, nrhs, "bf16"
    _, plan = bench.ApplyRun.fused_bytes(run)
    op = qtt.Operator(data, packs=("bf16",))
    x = torch.from_numpy(inputs.gaussian_rhs(data.N, nrhs, 6)).to(torch.bfloat16).cuda()
    op.apply(x, compute="bf16")  # first call: one-time setup outside the count
    torch.cuda.synchronize()
    n0 = qtt.kernel_launches()
    op.apply(x, compute="bf16")
    torch.cuda.synchronize()
    op.close()
    assert qtt.kernel_launches() - n0 == len(plan), plan
