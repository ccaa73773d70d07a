"""Seeded synthetic inputs for the QTT apply and solves.

This module is the only code that both the CUDA path and the CPU oracle
consume.  It produces operators (QTT cores) and right-hand sides; it holds
none of the apply or solve arithmetic under test.  Building the operators does
use the paper's compression tools (TT-SVD, Algorithm 1; TT rounding) and the
core-wise product/sum needed to form a preconditioner; those are set-up steps,
never the hot path, and the tests pin them separately.

Recipes (all draws from ``numpy.random.default_rng(seed)``, PCG64, which gives
the same stream on every platform):

* ``laplace_volume`` -- second-kind volume operator A = I + h^3 K on a
  uniform n x n x n grid, h = 1/n, K(x, y) = 1/(4 pi |x - y|) for x != y and
  0 on the diagonal (punctured trapezoid rule, Sec. 5.2), points in Morton
  order (bit 3l + c of the index is bit l of coordinate c), compressed by
  TT-SVD (Algorithm 1) at accuracy eps.
* ``synthetic_operator`` -- ranks r_k = min(2^k, 2^(d-k), r_max); every core
  but the last is drawn i.i.d. N(0, 1/(4 r_{k-1})), reshaped to a
  (4 r_{k-1}) x r_k matrix, replaced by the Q of its thin QR and its columns
  scaled by 10^(-j/8), j = 0..r_k-1; the last core stays Gaussian.
* ``gaussian_rhs`` -- i.i.d. N(0, 1) right-hand sides.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

_DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")


@dataclass
class QTTData:
    """A QTT matrix as plain data: ranks[0..d] (ends 1) and d float64 cores,
    core k shaped (ranks[k], 2, 2, ranks[k+1]) with index order
    [alpha_k][row bit i][column bit j][alpha_{k+1}]."""

    ranks: list
    cores: list
    meta: dict = field(default_factory=dict)

    @property
    def d(self) -> int:
        return len(self.ranks) - 1

    @property
    def N(self) -> int:
        return 1 << self.d

    @property
    def sigma(self) -> int:
        """sum_k r_k r_{k+1}: the apply costs 4 N sigma flops per RHS."""
        return int(sum(self.ranks[k] * self.ranks[k + 1] for k in range(self.d)))

    def flops(self, nrhs: int = 1) -> float:
        return 4.0 * self.N * nrhs * self.sigma

    def flat(self) -> np.ndarray:
        return np.concatenate([np.ascontiguousarray(c, dtype=np.float64).ravel()
                               for c in self.cores])

    def scaled(self, s: float) -> "QTTData":
        cores = [c.copy() for c in self.cores]
        cores[-1] = cores[-1] * s
        return QTTData(list(self.ranks), cores, dict(self.meta, scale=s))


# ---------------------------------------------------------------- structure
def rank_profile(d: int, rmax: int) -> list:
    return [min(2 ** k, 2 ** (d - k), rmax) for k in range(d + 1)]


def identity(d: int) -> QTTData:
    """All ranks 1, every core the 2 x 2 identity."""
    eye = np.eye(2).reshape(1, 2, 2, 1)
    return QTTData([1] * (d + 1), [eye.copy() for _ in range(d)], {"kind": "identity"})


def kronecker(mats) -> QTTData:
    """Rank-1 QTT from 2 x 2 matrices, mats[k] acting on bit k."""
    cores = [np.asarray(m, dtype=np.float64).reshape(1, 2, 2, 1) for m in mats]
    return QTTData([1] * (len(mats) + 1), cores, {"kind": "kronecker"})


def random_cores(d: int, ranks, seed: int, integer: bool = False) -> QTTData:
    """Unstructured cores: N(0,1) entries, or integers in {-1, 0, 1}."""
    rng = np.random.default_rng(seed)
    cores = []
    for k in range(d):
        shape = (ranks[k], 2, 2, ranks[k + 1])
        if integer:
            cores.append(rng.integers(-1, 2, size=shape).astype(np.float64))
        else:
            cores.append(rng.standard_normal(shape))
    return QTTData(list(ranks), cores, {"kind": "integer" if integer else "gaussian",
                                        "seed": seed})


def random_ranks(d: int, rmax: int, seed: int) -> list:
    rng = np.random.default_rng(seed)
    return [1] + [int(v) for v in rng.integers(1, rmax + 1, size=d - 1)] + [1]


def synthetic_operator(d: int, rmax: int, seed: int) -> QTTData:
    """Synthetic QTT operator shaped like a compressed volume operator."""
    rng = np.random.default_rng(seed)
    ranks = rank_profile(d, rmax)
    cores = []
    for k in range(d):
        ra, rb = ranks[k], ranks[k + 1]
        g = rng.standard_normal((ra, 2, 2, rb)) * math.sqrt(1.0 / (4.0 * ra))
        if k < d - 1:
            q, _ = np.linalg.qr(g.reshape(4 * ra, rb))
            q = q * (10.0 ** (-np.arange(rb) / 8.0))[None, :]
            g = q.reshape(ra, 2, 2, rb)
        cores.append(np.ascontiguousarray(g))
    return QTTData(ranks, cores, {"kind": "synthetic", "d": d, "rmax": rmax, "seed": seed})


def gaussian_rhs(N: int, nrhs: int, seed: int) -> np.ndarray:
    """(nrhs, N) i.i.d. N(0, 1); row c is right-hand side c."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nrhs, N))


# ------------------------------------------------------- 3-D Laplace volume
def morton_points(n: int) -> np.ndarray:
    """Integer grid coordinates (N, 3) of an n^3 grid (n a power of two) in
    Morton order: bit 3l + c of the linear index is bit l of coordinate c."""
    L = int(round(math.log2(n)))
    if 2 ** L != n:
        raise ValueError("grid side must be a power of two")
    idx = np.arange(n ** 3)
    pts = np.zeros((n ** 3, 3), dtype=np.int64)
    for lev in range(L):
        for c in range(3):
            pts[:, c] |= ((idx >> (3 * lev + c)) & 1) << lev
    return pts


def laplace_volume_dense(n: int = 8) -> np.ndarray:
    """Dense A = I + h^3 K, h = 1/n, K = 1/(4 pi |x-y|), zero diagonal."""
    h = 1.0 / n
    p = morton_points(n).astype(np.float64)
    diff = p[:, None, :] - p[None, :, :]
    dist = np.sqrt((diff ** 2).sum(-1)) * h
    with np.errstate(divide="ignore"):
        K = 1.0 / (4.0 * math.pi * dist)
    np.fill_diagonal(K, 0.0)
    return np.eye(p.shape[0]) + h ** 3 * K


def matrix_to_qtt_tensor(A: np.ndarray) -> np.ndarray:
    """Tensorise a 2^d x 2^d matrix on the product tree (Sec. 3.1): mode k is
    b_k = 2 i_k + j_k, modes ordered k = 0..d-1 (finest first)."""
    N = A.shape[0]
    d = int(round(math.log2(N)))
    # C-order reshape gives axes (i_{d-1}, ..., i_0, j_{d-1}, ..., j_0)
    T = A.reshape([2] * (2 * d))
    perm = []
    for k in range(d):
        perm += [d - 1 - k, 2 * d - 1 - k]  # i_k, j_k
    return np.ascontiguousarray(T.transpose(perm)).reshape([4] * d)


def tt_svd(T: np.ndarray, eps: float):
    """Algorithm 1 (TT decomposition by successive truncated SVDs).  Each
    unfolding keeps the smallest rank whose discarded singular values have
    Frobenius norm <= eps ||T||_F / sqrt(d-1) (rank >= 1).  Returns
    (ranks, cores) with cores shaped (r_k, n_k, r_{k+1})."""
    dims = T.shape
    d = len(dims)
    delta = eps * np.linalg.norm(T.ravel()) / math.sqrt(max(d - 1, 1))
    ranks = [1]
    cores = []
    M = T.reshape(dims[0], -1)
    for k in range(d - 1):
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
        tail = np.sqrt(np.cumsum((S ** 2)[::-1]))[::-1]  # tail[r] = ||S[r:]||
        r = len(S)
        for cand in range(1, len(S) + 1):
            rest = tail[cand] if cand < len(S) else 0.0
            if rest <= delta:
                r = cand
                break
        cores.append(U[:, :r].reshape(ranks[-1], dims[k], r))
        ranks.append(r)
        M = (S[:r, None] * Vt[:r]).reshape(r * dims[k + 1], -1)
    cores.append(M.reshape(ranks[-1], dims[d - 1], 1))
    ranks.append(1)
    return ranks, cores


def laplace_volume(n: int = 8, eps: float = 1e-8):
    """The n^3 Laplace volume operator A = I + h^3 K (Sec. 5.2) compressed by
    TT-SVD at eps.  Returns (QTTData, dense A)."""
    A = laplace_volume_dense(n)
    ranks, cores = tt_svd(matrix_to_qtt_tensor(A), eps)
    cores = [c.reshape(c.shape[0], 2, 2, c.shape[2]) for c in cores]
    return QTTData(ranks, cores, {"kind": "laplace", "n": n, "eps": eps}), A


# ------------------------------------------ operator norms and preconditioner
def knorm_table() -> dict:
    """Stored spectral norms ||K||_2 of the synthetic operators used by the
    solve workloads, computed by power iteration in the CPU oracle (see
    ``oracle/make_knorm.py``).  Keys are "d{d}_r{rmax}_s{seed}"."""
    path = os.path.join(_DATA, "knorm.json")
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        return json.load(fh)


def knorm_key(d: int, rmax: int, seed: int) -> str:
    return f"d{d}_r{rmax}_s{seed}"


def scaled_operator(d: int, rmax: int, seed: int, target: float = 0.5,
                    sigma: float | None = None) -> QTTData:
    """synthetic_operator scaled so that ||K||_2 = target, using the stored
    norm (or the one given)."""
    K = synthetic_operator(d, rmax, seed)
    if sigma is None:
        tab = knorm_table()
        key = knorm_key(d, rmax, seed)
        if key not in tab:
            raise KeyError(f"no stored ||K||_2 for {key}; run oracle/make_knorm.py")
        sigma = tab[key]["sigma"]
    out = K.scaled(target / sigma)
    out.meta.update({"knorm_target": target, "knorm_unscaled": sigma})
    return out


def _core_product(A: QTTData, B: QTTData) -> QTTData:
    """Core-wise product A B (ranks multiply); set-up only."""
    cores = []
    for a, b in zip(A.cores, B.cores):
        # c[(p,q), i, j, (s,t)] = sum_l a[p,i,l,s] b[q,l,j,t]
        c = np.einsum("pils,qljt->pqijst", a, b)
        pa, qa = a.shape[0], b.shape[0]
        sa, tb = a.shape[3], b.shape[3]
        cores.append(c.reshape(pa * qa, 2, 2, sa * tb))
    ranks = [A.ranks[k] * B.ranks[k] for k in range(A.d + 1)]
    return QTTData(ranks, cores)


def _core_sum(terms) -> QTTData:
    """sum of operators (list of (coef, QTTData)) by rank concatenation."""
    d = terms[0][1].d
    ranks = [1] + [sum(t.ranks[k] for _, t in terms) for k in range(1, d)] + [1]
    cores = []
    for k in range(d):
        c = np.zeros((ranks[k], 2, 2, ranks[k + 1]))
        ro = co = 0
        for coef, t in terms:
            g = t.cores[k] * (coef if k == d - 1 else 1.0)
            ra, rb = g.shape[0], g.shape[3]
            r0 = ro if k > 0 else 0
            c0 = co if k < d - 1 else 0
            c[r0:r0 + ra, :, :, c0:c0 + rb] += g
            ro += ra if k > 0 else 0
            co += rb if k < d - 1 else 0
        cores.append(c)
    return QTTData(ranks, cores)


def neumann_preconditioner_unrounded(K: QTTData) -> QTTData:
    """I - K + K^2 as an exact QTT (rank 1 + r + r^2)."""
    if K.d == 1:
        I2 = np.eye(2)
        k = K.cores[0][0, :, :, 0]
        return QTTData([1, 1], [(I2 - k + k @ k).reshape(1, 2, 2, 1)])
    K2 = _core_product(K, K)
    return _core_sum([(1.0, identity(K.d)), (-1.0, K), (1.0, K2)])


def tt_round(op: QTTData, eps: float) -> QTTData:
    """TT rounding (Oseledets): right-to-left QR orthogonalisation, then a
    left-to-right sweep of truncated SVDs with the Algorithm 1 threshold
    eps ||A||_F / sqrt(d-1)."""
    d = op.d
    cores = [np.asarray(c, dtype=np.float64).reshape(c.shape[0], 4, c.shape[3]).copy()
             for c in op.cores]
    ranks = list(op.ranks)
    # right-to-left orthogonalisation: core k becomes row-orthonormal
    for k in range(d - 1, 0, -1):
        ra, n, rb = cores[k].shape
        M = cores[k].reshape(ra, n * rb)
        Q, R = np.linalg.qr(M.T)  # M^T = Q R  =>  M = R^T Q^T
        rnew = Q.shape[1]
        cores[k] = Q.T.reshape(rnew, n, rb)
        pa, pn, _ = cores[k - 1].shape
        cores[k - 1] = (cores[k - 1].reshape(pa * pn, -1) @ R.T).reshape(pa, pn, rnew)
        ranks[k] = rnew
    norm = np.linalg.norm(cores[0].ravel())
    delta = eps * norm / math.sqrt(max(d - 1, 1))
    for k in range(d - 1):
        ra, n, rb = cores[k].shape
        U, S, Vt = np.linalg.svd(cores[k].reshape(ra * n, rb), full_matrices=False)
        tail = np.sqrt(np.cumsum((S ** 2)[::-1]))[::-1]
        r = len(S)
        for cand in range(1, len(S) + 1):
            rest = tail[cand] if cand < len(S) else 0.0
            if rest <= delta:
                r = cand
                break
        cores[k] = U[:, :r].reshape(ra, n, r)
        SV = S[:r, None] * Vt[:r]
        _, nn, rc = cores[k + 1].shape
        cores[k + 1] = (SV @ cores[k + 1].reshape(rb, nn * rc)).reshape(r, nn, rc)
        ranks[k + 1] = r
    out = [c.reshape(c.shape[0], 2, 2, c.shape[2]) for c in cores]
    return QTTData(ranks, out, dict(op.meta, rounded_eps=eps))


def neumann_preconditioner(K: QTTData, eps: float = 1e-4) -> QTTData:
    """P = round(I - K + K^2, eps): approximate inverse of I + K for
    ||K|| < 1 (error operator -K^3 before rounding)."""
    P = tt_round(neumann_preconditioner_unrounded(K), eps)
    P.meta.update({"kind": "neumann_preconditioner", "eps": eps})
    return P


# ------------------------------------------------------- workload draws
def batched_workload(count: int = 256, seed: int = 4, d_range=(12, 20),
                     r_range=(16, 40), rhs_range=(1, 32)):
    """Uneven batch: per operator d, r_max, nrhs drawn uniformly (inclusive),
    then its cores and right-hand sides from per-operator seeds."""
    rng = np.random.default_rng(seed)
    items = []
    for n in range(count):
        d = int(rng.integers(d_range[0], d_range[1] + 1))
        rmax = int(rng.integers(r_range[0], r_range[1] + 1))
        nrhs = int(rng.integers(rhs_range[0], rhs_range[1] + 1))
        items.append({"d": d, "rmax": rmax, "nrhs": nrhs,
                      "op_seed": 1000003 * (seed + 1) + 2 * n,
                      "rhs_seed": 1000003 * (seed + 1) + 2 * n + 1})
    return items


def serving_trace(count: int, rate: float, seed: int = 5, d_range=(14, 22),
                  rhs_range=(1, 16)):
    """Poisson arrivals (exponential gaps, mean 1/rate seconds) of solve
    requests; per request d, nrhs and the seed of its right-hand sides."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for n in range(count):
        t += float(rng.exponential(1.0 / rate))
        d = int(rng.integers(d_range[0], d_range[1] + 1))
        nrhs = int(rng.integers(rhs_range[0], rhs_range[1] + 1))
        reqs.append({"id": n, "arrival": t, "d": d, "nrhs": nrhs,
                     "rhs_seed": 5000011 * (seed + 1) + n})
    return reqs
