"""Seeded synthetic inputs for the QTT apply and solves.

This module is the only code that both the CUDA path and the CPU oracle
consume.  It produces seeded data -- QTT cores, dense matrices, right-hand
sides, workload draws -- and holds none of the method's arithmetic: the
compression of a dense matrix (Algorithm 1), TT rounding and the core-wise
products and sums that form a preconditioner are done by each side with its
own code (the library's GPU entry points, or the oracle).

Recipes (all draws from ``numpy.random.default_rng(seed)``, PCG64, which gives
the same stream on every platform):

* ``laplace_volume_dense`` -- the dense second-kind volume operator
  A = I + h^3 K on a uniform n x n x n grid, h = 1/n, K(x, y) =
  1/(4 pi |x - y|) for x != y and 0 on the diagonal (punctured trapezoid
  rule, Sec. 5.2), points in Morton order (bit 3l + c of the index is bit l
  of coordinate c); its QTT form comes from Algorithm 1 at eps = 1e-8.
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
# The .qtt operator file (header: magic "QTT1", version, d, element type,
# core layout, reserved -- little-endian uint32 -- then d + 1 uint32 ranks
# and the FP64 cores in QTTData's order).  The library reads and writes the
# same format; this is an independent numpy version for the generators.
_QTT_MAGIC = b"QTT1"


def save_qtt(path: str, data: QTTData) -> None:
    head = np.array([1, data.d, 0, 0, 0], dtype="<u4").tobytes()
    body = np.asarray(data.ranks, dtype="<u4").tobytes() + b"".join(
        np.ascontiguousarray(c, dtype="<f8").tobytes() for c in data.cores)
    with open(path, "wb") as f:
        f.write(_QTT_MAGIC + head + body)


def load_qtt(path: str) -> QTTData:
    raw = open(path, "rb").read()
    if raw[:4] != _QTT_MAGIC or len(raw) < 24:
        raise ValueError(f"{path}: not a .qtt file")
    version, d, etype, layout, _ = np.frombuffer(raw, dtype="<u4", count=5, offset=4)
    if version != 1 or etype != 0 or layout != 0:
        raise ValueError(f"{path}: unsupported .qtt version, element type or layout")
    ranks = [int(r) for r in np.frombuffer(raw, dtype="<u4", count=d + 1, offset=24)]
    off = 24 + 4 * (d + 1)
    cores = []
    for k in range(d):
        n = 4 * ranks[k] * ranks[k + 1]
        cores.append(np.frombuffer(raw, dtype="<f8", count=n, offset=off)
                     .reshape(ranks[k], 2, 2, ranks[k + 1]).astype(np.float64))
        off += 8 * n
    if off != len(raw):
        raise ValueError(f"{path}: length does not match the ranks")
    return QTTData(ranks, cores, {"kind": "file", "path": path})


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


def general_cores(m, n, rmax: int, seed: int):
    """Cores of a QTT matrix with general mode sizes (m_k x n_k modes):
    ranks min(prod of the mode products on either side, rmax), entries
    i.i.d. N(0, 1 / (r_k n_k)) so that every step keeps the intermediate's
    size of order one.  Core k has shape (r_k, m_k, n_k, r_{k+1})."""
    rng = np.random.default_rng(seed)
    d = len(m)
    ranks = [1]
    for k in range(1, d):
        left = int(np.prod([m[l] * n[l] for l in range(k)]))
        right = int(np.prod([m[l] * n[l] for l in range(k, d)]))
        ranks.append(min(rmax, left, right))
    ranks.append(1)
    return [rng.standard_normal((ranks[k], m[k], n[k], ranks[k + 1])) / math.sqrt(ranks[k] * n[k])
            for k in range(d)]


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
