"""Pins for the CPU oracle, none of which reuse the oracle's own code path.

Each test checks the oracle against something the paper or mathematics fixes:
a hand-derived example, numpy's Kronecker product, brute force by numpy
matmul, integer-exact arithmetic, algebraic identities, and a long-double
re-run bounding its rounding error.
"""
import os

import numpy as np
import pytest

from paper_1511_06029_gb300 import inputs
from conftest import rel_l2, neumann_unrounded

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_hand_example():
    vals = {"A": []}
    with open(os.path.join(GOLDEN, "hand_d2_rank2.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *nums = line.split()
            nums = [float(v) for v in nums]
            if key == "A":
                vals["A"].append(nums)
            else:
                vals[key] = nums
    c0 = np.array(vals["core0"]).reshape(1, 2, 2, 2)
    c1 = np.array(vals["core1"]).reshape(2, 2, 2, 1)
    op = inputs.QTTData([1, 2, 1], [c0, c1])
    return op, np.array(vals["A"]), np.array(vals["x"]), np.array(vals["y"])


def test_hand_example(oracle_mod):
    """Sec. 2.2 entry formula with the Sec. 2.1 index order, worked by hand."""
    op, A, x, y = _read_hand_example()
    assert np.array_equal(oracle_mod.dense(op), A)
    assert np.array_equal(oracle_mod.apply(op, x), y)


@pytest.mark.parametrize("k", [0, 1, 3])
def test_index_convention_shift(oracle_mod, k):
    """Least-significant-bit-first convention: a rank-1 operator whose core k
    is [[0, 1], [0, 0]] (others I_2) maps j = i + 2^k onto i for every i with
    bit k clear, and nothing else."""
    d = 5
    mats = [np.eye(2)] * d
    mats[k] = np.array([[0.0, 1.0], [0.0, 0.0]])
    A = oracle_mod.dense(inputs.kronecker(mats))
    N = 1 << d
    expect = np.zeros((N, N))
    for i in range(N):
        if not (i >> k) & 1:
            expect[i, i + (1 << k)] = 1.0
    assert np.array_equal(A, expect)


@pytest.mark.parametrize("d", [1, 2, 7, 12])
def test_identity_is_bitwise(oracle_mod, d):
    """All ranks 1, every core I_2 (identity has QTT rank 1, Sec. 3.3):
    y = x exactly."""
    x = inputs.gaussian_rhs(1 << d, 3, seed=d)
    assert np.array_equal(oracle_mod.apply(inputs.identity(d), x), x)


@pytest.mark.parametrize("d", [1, 3, 6])
def test_kronecker_matches_numpy(oracle_mod, d):
    """Rank-1 QTT = G_{d-1} kron ... kron G_0 (bit 0 fastest), checked
    against numpy.kron, for both the dense form and the apply."""
    rng = np.random.default_rng(10 + d)
    mats = [rng.standard_normal((2, 2)) for _ in range(d)]
    op = inputs.kronecker(mats)
    K = np.array([[1.0]])
    for m in mats:
        K = np.kron(m, K)
    A = oracle_mod.dense(op)
    assert np.allclose(A, K, rtol=1e-14, atol=1e-15)
    x = rng.standard_normal(1 << d)
    assert rel_l2(oracle_mod.apply(op, x), K @ x) <= 1e-14


@pytest.mark.parametrize("d,rmax,seed", [(4, 3, 1), (8, 6, 2), (10, 16, 3), (12, 4, 4)])
def test_dense_bruteforce(oracle_mod, d, rmax, seed):
    """Sweep apply vs the dense reconstruction times x (numpy matmul)."""
    op = inputs.random_cores(d, inputs.random_ranks(d, rmax, seed), seed)
    A = oracle_mod.dense(op)
    x = inputs.gaussian_rhs(1 << d, 2, seed + 100)
    y_dense = x @ A.T
    assert rel_l2(oracle_mod.apply(op, x), y_dense) <= 1e-13
    assert rel_l2(oracle_mod.dense_matvec(A, x), y_dense) <= 1e-14


def test_dense_entries_by_slice_products(oracle_mod):
    """qo_dense against entries formed here by explicit numpy slice products
    (the entry formula, no shared code)."""
    d = 9
    op = inputs.random_cores(d, inputs.random_ranks(d, 7, 5), 5)
    A = oracle_mod.dense(op)
    rng = np.random.default_rng(0)
    for _ in range(200):
        i, j = (int(v) for v in rng.integers(0, 1 << d, size=2))
        v = np.ones((1, 1))
        for k in range(d):
            v = v @ op.cores[k][:, (i >> k) & 1, (j >> k) & 1, :]
        assert abs(A[i, j] - v[0, 0]) <= 1e-13 * max(1.0, abs(v[0, 0]))


@pytest.mark.parametrize("d,rmax,seed", [(6, 4, 1), (10, 4, 2), (12, 3, 3)])
def test_integer_exact(oracle_mod, d, rmax, seed):
    """Cores in {-1, 0, 1} and integer x: every intermediate is an integer
    below 2^53, so the sweep and the brute-force product agree bitwise."""
    op = inputs.random_cores(d, inputs.random_ranks(d, rmax, seed), seed, integer=True)
    x = np.random.default_rng(seed).integers(-8, 9, size=(2, 1 << d)).astype(np.float64)
    A = oracle_mod.dense(op)
    assert np.array_equal(oracle_mod.apply(op, x), x @ A.T)


def test_long_double_bound(oracle_mod):
    """The FP64 sweep is within 1e-14 (relative L2) of the same sweep in
    long double: the oracle's own rounding is far below the 1e-12 parity
    tolerance it judges."""
    op = inputs.synthetic_operator(14, 32, 2)
    x = inputs.gaussian_rhs(op.N, 1, 3)[0]
    y = oracle_mod.apply(op, x)
    yl = oracle_mod.apply(op, x, long_double=True)
    assert rel_l2(y, yl) <= 1e-14


def test_sum_and_product(oracle_mod):
    """apply(A + B) = apply(A) + apply(B); apply(A B, x) = A (B x); dense
    forms against numpy sums and matmuls (rank addition and the core-wise
    product, Sec. 3.3 and Sec. 4.2)."""
    d = 7
    A = inputs.random_cores(d, inputs.random_ranks(d, 4, 11), 11)
    B = inputs.random_cores(d, inputs.random_ranks(d, 3, 12), 12)
    S = oracle_mod.tt_sum(A, B)
    Pm = oracle_mod.tt_product(A, B)
    DA, DB = oracle_mod.dense(A), oracle_mod.dense(B)
    assert np.allclose(oracle_mod.dense(S), DA + DB, rtol=1e-13, atol=1e-12)
    assert rel_l2(oracle_mod.dense(Pm), DA @ DB) <= 1e-13
    x = inputs.gaussian_rhs(1 << d, 1, 13)[0]
    assert rel_l2(oracle_mod.apply(S, x), oracle_mod.apply(A, x) + oracle_mod.apply(B, x)) <= 1e-13
    assert rel_l2(oracle_mod.apply(Pm, x), oracle_mod.apply(A, oracle_mod.apply(B, x))) <= 1e-13
    assert S.ranks == [1] + [A.ranks[k] + B.ranks[k] for k in range(1, d)] + [1]
    assert Pm.ranks == [A.ranks[k] * B.ranks[k] for k in range(d + 1)]


def test_transpose_adjoint(oracle_mod):
    """dense(A^T) = dense(A)^T and <y, A x> = <A^T y, x>."""
    d = 8
    A = inputs.random_cores(d, inputs.random_ranks(d, 5, 21), 21)
    AT = oracle_mod.transpose(A)
    assert np.array_equal(oracle_mod.dense(AT), oracle_mod.dense(A).T)
    x, y = inputs.gaussian_rhs(1 << d, 2, 22)
    lhs = float(y @ oracle_mod.apply(A, x))
    rhs = float(oracle_mod.apply(AT, y) @ x)
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_multiple_rhs_are_independent(oracle_mod):
    op = inputs.synthetic_operator(9, 8, 1)
    X = inputs.gaussian_rhs(op.N, 4, 2)
    Y = oracle_mod.apply(op, X)
    for c in range(4):
        assert np.array_equal(Y[c], oracle_mod.apply(op, X[c]))


def test_power_norm_matches_lapack(oracle_mod):
    op = inputs.random_cores(7, inputs.random_ranks(7, 4, 31), 31)
    v0 = np.random.default_rng(1).standard_normal(op.N)
    s, _ = oracle_mod.power_norm(op, v0, max_iter=2000, rtol=1e-13)
    ref = np.linalg.norm(oracle_mod.dense(op), 2)
    assert abs(s - ref) <= 1e-6 * ref


# ------------------------------------------------------------------ solves
def _small_solve_problem(d=8):
    K = inputs.random_cores(d, inputs.random_ranks(d, 4, 41), 41)
    return K


def _scaled(oracle_mod, K, target=0.5):
    s = np.linalg.norm(oracle_mod.dense(K), 2)
    return K.scaled(target / s)


def test_gmres_matches_dense_solve(oracle_mod):
    """GMRES(m) without and with a preconditioner reaches the LAPACK
    solution of the dense (a I + K) x = f."""
    d = 8
    K = _scaled(oracle_mod, _small_solve_problem(d), 0.9)
    A = np.eye(1 << d) + oracle_mod.dense(K)
    f = inputs.gaussian_rhs(1 << d, 2, 42)
    xs = np.linalg.solve(A, f.T).T
    x, it, rel = oracle_mod.solve_gmres(K, None, f, a=1.0, tol=1e-13, restart=10,
                                        max_iter=400)
    assert rel_l2(x, xs) <= 1e-11 and (rel <= 1e-13).all()
    P = neumann_unrounded(oracle_mod, K)
    x2, it2, rel2 = oracle_mod.solve_gmres(K, P, f, a=1.0, tol=1e-13, restart=30)
    assert rel_l2(x2, xs) <= 1e-11
    assert it2.max() < it.max()


def test_gmres_zero_rhs(oracle_mod):
    K = _scaled(oracle_mod, _small_solve_problem(6))
    x, it, rel = oracle_mod.solve_gmres(K, None, np.zeros(64), a=1.0)
    assert np.array_equal(x, np.zeros(64)) and it[0] == 0


def test_refine_contracts_like_neumann(oracle_mod):
    """With the unrounded P = I - K + K^2, the error of refinement contracts by
    the error operator -K^3 each step (Neumann series): iterations needed for
    1e-13 are bounded by ceil(13 / -log10 ||K^3||) + 1."""
    d = 8
    K = _scaled(oracle_mod, _small_solve_problem(d), 0.5)
    P = neumann_unrounded(oracle_mod, K)
    DK = oracle_mod.dense(K)
    E = np.eye(1 << d) - oracle_mod.dense(P) @ (np.eye(1 << d) + DK)
    assert np.allclose(E, -DK @ DK @ DK, atol=1e-14)
    f = inputs.gaussian_rhs(1 << d, 1, 43)[0]
    x, it, rel = oracle_mod.solve_refine(K, P, f, a=1.0, tol=1e-13)
    xs = np.linalg.solve(np.eye(1 << d) + DK, f)
    assert rel_l2(x, xs) <= 1e-12
    c = np.linalg.norm(DK @ DK @ DK, 2)
    assert it[0] <= int(np.ceil(13 / -np.log10(c))) + 2


def test_refine_not_converged_reports(oracle_mod):
    K = _scaled(oracle_mod, _small_solve_problem(6), 0.5)
    f = inputs.gaussian_rhs(64, 1, 44)[0]
    x, it, rel = oracle_mod.solve_refine(K, None, f, a=1.0, tol=1e-13, max_iter=1,
                                         raise_on_fail=False)
    assert it[0] == 1 and rel[0] > 1e-13
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.solve_refine(K, None, f, a=1.0, tol=1e-13, max_iter=1)


def test_direct_is_apply(oracle_mod):
    P = inputs.synthetic_operator(9, 8, 3)
    f = inputs.gaussian_rhs(P.N, 2, 4)
    assert np.array_equal(oracle_mod.solve_direct(P, f), oracle_mod.apply(P, f))


def test_entries_match_dense(oracle_mod):
    op = inputs.random_cores(9, inputs.random_ranks(9, 6, 51), 51)
    A = oracle_mod.dense(op)
    rng = np.random.default_rng(52)
    I = rng.integers(0, 512, size=300)
    J = rng.integers(0, 512, size=300)
    assert np.allclose(oracle_mod.entries(op, I, J), A[I, J], rtol=1e-13, atol=1e-15)


# ------------------------------------------- compressed vectors and rounding
def _random_vec(oracle_mod, d, ranks, seed):
    rng = np.random.default_rng(seed)
    cores = [rng.standard_normal((ranks[k], 2, ranks[k + 1])) for k in range(d)]
    return oracle_mod.Vec(ranks, cores)


def _vec_dense_bruteforce(v):
    """Entry formula element by element (Sec. 2.2): t's bits pick one slice
    of each core; small d only."""
    d = len(v.ranks) - 1
    out = np.empty(1 << d)
    for t in range(1 << d):
        m = np.eye(1)
        for k in range(d):
            m = m @ v.cores[k][:, (t >> k) & 1, :]
        out[t] = m[0, 0]
    return out


def test_qtt_vector_entries(oracle_mod):
    """vec_full against the entry formula and, for rank 1, numpy's kron."""
    v = _random_vec(oracle_mod, 6, [1, 2, 3, 3, 2, 2, 1], 40)
    assert rel_l2(oracle_mod.vec_full(v), _vec_dense_bruteforce(v)) <= 1e-14
    rng = np.random.default_rng(41)
    parts = [rng.standard_normal(2) for _ in range(5)]
    kron = parts[-1]
    for p in parts[-2::-1]:
        kron = np.kron(kron, p)  # bit 0 (first core) varies fastest
    v1 = oracle_mod.Vec([1] * 6, [p.reshape(1, 2, 1) for p in parts])
    assert np.array_equal(oracle_mod.vec_full(v1), kron)


@pytest.mark.parametrize("d,seed", [(6, 42), (9, 43)])
def test_compressed_matvec_matches_dense(oracle_mod, d, seed):
    """Sec. 4.2 compressed product: the full vector of A b equals the dense
    matrix (numpy slice products) times the full vector b; ranks multiply."""
    rng = np.random.default_rng(seed)
    ra = [1] + list(rng.integers(1, 5, d - 1)) + [1]
    rb = [1] + list(rng.integers(1, 4, d - 1)) + [1]
    A = inputs.random_cores(d, ra, seed)
    b = _random_vec(oracle_mod, d, rb, seed + 100)
    c = oracle_mod.apply_tt(A, b)
    assert c.ranks == [x * y for x, y in zip(ra, rb)]
    ref = oracle_mod.dense(A) @ _vec_dense_bruteforce(b)
    assert rel_l2(oracle_mod.vec_full(c), ref) <= 1e-13


@pytest.mark.parametrize("eps", [1e-1, 1e-3, 1e-6])
def test_rounding_error_bound(oracle_mod, eps):
    """||T - round(T)||_F <= eps ||T||_F (the Algorithm 1 threshold per
    unfolding, d - 1 unfoldings), ranks never above the input's."""
    d = 7
    A = inputs.random_cores(d, [1, 2, 4, 6, 6, 4, 2, 1], 44)
    B = inputs.random_cores(d, [1, 2, 3, 5, 3, 3, 2, 1], 45)
    T = oracle_mod.tt_sum(A, B)
    R = oracle_mod.tt_round(T, eps)
    full_t, full_r = oracle_mod.dense(T), oracle_mod.dense(R)
    err = np.linalg.norm(full_t - full_r) / np.linalg.norm(full_t)
    assert err <= eps * (1 + 1e-10), err
    assert all(r <= t for r, t in zip(R.ranks, T.ranks))
    # the same on a compressed vector
    v = _random_vec(oracle_mod, d, [1, 2, 4, 8, 8, 4, 2, 1], 46)
    w = oracle_mod.tt_round(v, eps)
    fv, fw = oracle_mod.vec_full(v), oracle_mod.vec_full(w)
    assert np.linalg.norm(fv - fw) <= eps * np.linalg.norm(fv) * (1 + 1e-10)


def test_rounding_recovers_redundant_ranks(oracle_mod):
    """A + A has twice A's ranks but is 2 A: rounding at a tiny eps returns
    ranks no larger than A's and the same matrix; a Kronecker product (rank
    1) summed with itself rounds back to rank 1."""
    ra = [1, 2, 4, 3, 2, 1]
    A = inputs.random_cores(5, ra, 47)
    R = oracle_mod.tt_round(oracle_mod.tt_sum(A, A), 1e-12)
    assert all(r <= a for r, a in zip(R.ranks, ra))
    assert rel_l2(oracle_mod.dense(R), 2 * oracle_mod.dense(A)) <= 1e-12
    K = inputs.random_cores(5, [1] * 6, 48)
    RK = oracle_mod.tt_round(oracle_mod.tt_sum(K, K), 1e-12)
    assert RK.ranks == [1] * 6
    assert rel_l2(oracle_mod.dense(RK), 2 * oracle_mod.dense(K)) <= 1e-12


def test_rounded_compressed_matvec(oracle_mod):
    """The compressed product followed by rounding stays within eps of the
    dense product, with ranks below the product ranks."""
    d = 8
    A = inputs.random_cores(d, [1, 2, 4, 4, 4, 4, 4, 2, 1], 49)
    b = _random_vec(oracle_mod, d, [1, 2, 2, 2, 2, 2, 2, 2, 1], 50)
    c = oracle_mod.tt_round(oracle_mod.apply_tt(A, b), 1e-8)
    ref = oracle_mod.dense(A) @ oracle_mod.vec_full(b)
    assert rel_l2(oracle_mod.vec_full(c), ref) <= 1e-8 * (1 + 1e-6)
    assert max(c.ranks) <= 8


# ------------------------------------------------------------ TT-SVD (Alg. 1)
def test_tt_svd_recovers_low_rank_operator(oracle_mod):
    """Algorithm 1 at a tiny eps on the dense matrix of a QTT operator with
    generic cores returns its ranks and its matrix."""
    ranks = [1, 2, 4, 3, 4, 2, 1]
    A = inputs.random_cores(6, ranks, 51)
    D = oracle_mod.dense(A)
    T = oracle_mod.tt_svd(D, 1e-13)
    assert T.ranks == ranks
    assert rel_l2(oracle_mod.dense(T), D) <= 1e-13


@pytest.mark.parametrize("eps", [3e-1, 1e-2])
def test_tt_svd_error_bound(oracle_mod, eps):
    """||A - A_tt||_F <= eps ||A||_F on a full-rank random matrix."""
    D = np.random.default_rng(52).standard_normal((64, 64))
    T = oracle_mod.tt_svd(D, eps)
    assert np.linalg.norm(oracle_mod.dense(T) - D) <= eps * np.linalg.norm(D) * (1 + 1e-12)


def test_tt_svd_kronecker_is_rank_one(oracle_mod):
    """A Kronecker product of 2 x 2 matrices (last factor outermost, bit 0
    innermost) has every QTT rank 1."""
    rng = np.random.default_rng(53)
    parts = [rng.standard_normal((2, 2)) for _ in range(5)]
    D = parts[-1]
    for p in parts[-2::-1]:
        D = np.kron(D, p)
    T = oracle_mod.tt_svd(D, 1e-12)
    assert T.ranks == [1] * 6
    assert rel_l2(oracle_mod.dense(T), D) <= 1e-13


def test_tt_svd_laplace_volume(oracle_mod):
    """The 8^3 Laplace volume matrix at eps = 1e-8: within the bound, and the
    same ranks as an independent Algorithm 1 written here (modes built by an
    explicit bit transpose, rank chosen by a cumulative tail search)."""
    D = inputs.laplace_volume_dense(8)
    T = oracle_mod.tt_svd(D, 1e-8)
    assert np.linalg.norm(oracle_mod.dense(T) - D) <= 1e-8 * np.linalg.norm(D) * (1 + 1e-9)
    assert T.ranks == _alg1_ranks(D, 1e-8)


def _alg1_ranks(A, eps):
    """Ranks of Algorithm 1 on the 2^d x 2^d matrix A, computed independently
    of the oracle: the tensor with modes b_k = 2 i_k + j_k (k = 0 first) by an
    axis transpose of A's bits, then successive SVDs, each keeping the
    smallest r with ||S[r:]|| <= eps ||A||_F / sqrt(d - 1)."""
    N = A.shape[0]
    d = int(round(np.log2(N)))
    T = A.reshape([2] * (2 * d))          # axes i_{d-1} .. i_0, j_{d-1} .. j_0
    perm = []
    for k in range(d):
        perm += [d - 1 - k, 2 * d - 1 - k]
    T = np.ascontiguousarray(T.transpose(perm))
    delta = eps * np.linalg.norm(A) / np.sqrt(max(d - 1, 1))
    ranks, M = [1], T.reshape(4, -1)
    for k in range(d - 1):
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
        tail = np.sqrt(np.cumsum((S ** 2)[::-1]))[::-1]
        r = next(c for c in range(1, len(S) + 1) if (tail[c] if c < len(S) else 0.0) <= delta)
        ranks.append(r)
        M = (S[:r, None] * Vt[:r]).reshape(r * 4, -1)
    return ranks + [1]


# ------------------------------------------------ general mode sizes (Sec. 3.1)
def _general_cores(ms, ns, ranks, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((ranks[k], ms[k], ns[k], ranks[k + 1])) for k in range(len(ms))]


def _general_dense_bruteforce(cores):
    """A(i, j) element by element: the mixed-radix digits of i and j (first
    mode fastest) pick one slice of each core, multiplied in order."""
    ms = [c.shape[1] for c in cores]
    ns = [c.shape[2] for c in cores]
    M, N = int(np.prod(ms)), int(np.prod(ns))
    D = np.empty((M, N))
    for i in range(M):
        for j in range(N):
            p, ii, jj = np.eye(1), i, j
            for c, m, n in zip(cores, ms, ns):
                p = p @ c[:, ii % m, jj % n, :]
                ii, jj = ii // m, jj // n
            D[i, j] = p[0, 0]
    return D


@pytest.mark.parametrize("ms,ns,ranks", [
    ([3, 2, 4], [2, 5, 3], [1, 2, 3, 1]),        # rectangular 24 x 30
    ([2, 3, 3, 2], [3, 2, 2, 3], [1, 3, 2, 2, 1]),
    ([4, 4], [4, 4], [1, 5, 1]),
])
def test_general_modes_match_bruteforce(oracle_mod, ms, ns, ranks):
    cores = _general_cores(ms, ns, ranks, sum(ms) + sum(ns))
    D = _general_dense_bruteforce(cores)
    x = np.random.default_rng(54).standard_normal((3, D.shape[1]))
    y = oracle_mod.apply_general(cores, x)
    assert y.shape == (3, D.shape[0])
    assert rel_l2(y, x @ D.T) <= 1e-14


def test_general_modes_kronecker_and_binary_case(oracle_mod):
    """Rank 1: A is the Kronecker product of the mode matrices (last mode
    outermost); m = n = 2: the binary oracle's apply."""
    rng = np.random.default_rng(55)
    mats = [rng.standard_normal((m, n)) for m, n in [(3, 2), (2, 4), (5, 3)]]
    D = mats[-1]
    for p in mats[-2::-1]:
        D = np.kron(D, p)
    cores = [mt.reshape(1, *mt.shape, 1) for mt in mats]
    x = rng.standard_normal(D.shape[1])
    assert rel_l2(oracle_mod.apply_general(cores, x), D @ x) <= 1e-14
    A = inputs.random_cores(7, [1, 2, 4, 5, 5, 4, 2, 1], 56)
    xb = rng.standard_normal((2, 128))
    assert rel_l2(oracle_mod.apply_general(A.cores, xb), oracle_mod.apply(A, xb)) <= 1e-14


# ------------------------------------------------- inversion local systems
@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_local_system_apply_is_the_projected_product(oracle_mod, k):
    """Entry e = (beta_{k-1}, i_k, p_k, beta_k) of the local left-hand side
    is the Frobenius inner product <X_e, A X>, X_e being X with core k
    replaced by the unit tensor at e: the projected system P^T (I (x) A) P
    vec(W_k) computed with dense matrices."""
    d = 4
    A = inputs.random_cores(d, [1, 2, 3, 2, 1], 57)
    X = inputs.random_cores(d, [1, 3, 2, 3, 1], 58)
    DA, DX = oracle_mod.dense(A), oracle_mod.dense(X)
    AX = DA @ DX
    psi, phi = oracle_mod.local_frames(A.cores, X.cores, k)
    y = oracle_mod.local_apply(psi, A.cores[k], phi, X.cores[k])
    Wk = X.cores[k]
    assert y.shape == Wk.shape
    ref = np.empty_like(Wk)
    for e in np.ndindex(*Wk.shape):
        unit = np.zeros_like(Wk)
        unit[e] = 1.0
        cores = list(X.cores)
        cores[k] = unit
        ref[e] = np.sum(oracle_mod.dense(inputs.QTTData(X.ranks, cores)) * AX)
    assert rel_l2(y, ref) <= 1e-13
