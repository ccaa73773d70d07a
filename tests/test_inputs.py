"""Pins for the seeded input generator (the synthetic recipe, the Laplace
volume matrix, workload draws) and for the operators the tests build from it
with the oracle (Algorithm 1 on the Laplace matrix, the Neumann
preconditioner)."""
import math

import numpy as np
import pytest

from paper_1511_06029_gb300 import inputs
from conftest import rel_l2, laplace_qtt, neumann_unrounded


def test_morton_order_bits():
    pts = inputs.morton_points(8)
    assert pts.shape == (512, 3)
    # each grid point exactly once
    assert len({tuple(p) for p in pts}) == 512
    # bit 3l + c of the index is bit l of coordinate c
    for idx in (0, 1, 2, 4, 8, 73, 511):
        for lev in range(3):
            for c in range(3):
                assert ((pts[idx, c] >> lev) & 1) == ((idx >> (3 * lev + c)) & 1)


def test_laplace_dense_closed_form():
    A = inputs.laplace_volume_dense(8)
    pts = inputs.morton_points(8)
    h = 1.0 / 8
    i, j = 5, 300
    dist = h * np.linalg.norm(pts[i] - pts[j])
    assert A[i, j] == pytest.approx(h ** 3 / (4 * math.pi * dist), rel=1e-15)
    assert np.all(np.diag(A) == 1.0)
    assert np.allclose(A, A.T)


def test_laplace_qtt_error_bound(oracle_mod):
    """The 8^3 operator from the oracle's Algorithm 1 with the eps/sqrt(d-1)
    threshold: ||A - A_tt||_F <= eps ||A||_F, hence ||A x - A_tt x|| <=
    eps ||A||_F ||x||."""
    eps = 1e-8
    op, A = laplace_qtt(oracle_mod, 8, eps)
    assert op.d == 9 and op.ranks[0] == 1 and op.ranks[-1] == 1
    for k in range(op.d + 1):
        assert op.ranks[k] <= min(4 ** k, 4 ** (op.d - k))
    Att = oracle_mod.dense(op)
    nA = np.linalg.norm(A)
    assert np.linalg.norm(A - Att) <= eps * nA
    x = inputs.gaussian_rhs(512, 1, 1)[0]
    err = np.linalg.norm(A @ x - oracle_mod.apply(op, x))
    assert err <= eps * nA * np.linalg.norm(x)


def test_synthetic_recipe():
    op = inputs.synthetic_operator(10, 8, 2)
    assert op.ranks == [1, 2, 4, 8, 8, 8, 8, 8, 4, 2, 1]
    for k in range(op.d - 1):
        rb = op.ranks[k + 1]
        M = op.cores[k].reshape(-1, rb) / (10.0 ** (-np.arange(rb) / 8.0))[None, :]
        assert np.allclose(M.T @ M, np.eye(rb), atol=1e-13)
    # deterministic in the seed
    op2 = inputs.synthetic_operator(10, 8, 2)
    assert all(np.array_equal(a, b) for a, b in zip(op.cores, op2.cores))


def test_d24_rank_profile_sigma():
    r = inputs.rank_profile(24, 32)
    assert r[:6] == [1, 2, 4, 8, 16, 32] and r[-6:] == [32, 16, 8, 4, 2, 1]
    sigma = sum(r[k] * r[k + 1] for k in range(24))
    assert sigma == 15700
    assert 4.0 * (1 << 24) * sigma == pytest.approx(1.054e12, rel=1e-3)


def test_neumann_preconditioner_exact_and_rounded(oracle_mod):
    """Unrounded P = I - K + K^2 satisfies I - P (I + K) = -K^3 exactly;
    rounding at eps keeps ||P_r - P||_F <= eps ||P||_F."""
    d = 7
    K = inputs.random_cores(d, inputs.random_ranks(d, 3, 5), 5)
    DK = oracle_mod.dense(K)
    K = K.scaled(0.5 / np.linalg.norm(DK, 2))
    DK = oracle_mod.dense(K)
    P = neumann_unrounded(oracle_mod, K)
    assert P.ranks[1:-1] == [1 + r + r * r for r in K.ranks[1:-1]]
    DP = oracle_mod.dense(P)
    I = np.eye(1 << d)
    assert np.allclose(DP, I - DK + DK @ DK, atol=1e-14)
    for eps in (1e-4, 1e-8):
        Pr = oracle_mod.tt_round(P, eps)
        assert max(Pr.ranks) <= max(P.ranks)
        assert np.linalg.norm(oracle_mod.dense(Pr) - DP) <= eps * np.linalg.norm(DP) * (1 + 1e-9)


def test_tt_round_lossless_at_tiny_eps(oracle_mod):
    op = inputs.random_cores(6, [1, 3, 5, 5, 4, 2, 1], 9)
    r = oracle_mod.tt_round(op, 1e-14)
    assert rel_l2(oracle_mod.dense(r), oracle_mod.dense(op)) <= 1e-12


def test_batched_and_serving_draws():
    items = inputs.batched_workload()
    assert len(items) == 256
    assert all(12 <= it["d"] <= 20 and 16 <= it["rmax"] <= 40 and 1 <= it["nrhs"] <= 32
               for it in items)
    assert items == inputs.batched_workload()
    reqs = inputs.serving_trace(100, rate=2.0)
    arr = [r["arrival"] for r in reqs]
    assert arr == sorted(arr)
    assert all(14 <= r["d"] <= 22 and 1 <= r["nrhs"] <= 16 for r in reqs)
    # mean gap close to 1/rate
    assert abs(np.mean(np.diff([0.0] + arr)) - 0.5) < 0.15
