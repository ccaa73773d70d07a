"""QTT oracle: plain FP64 CPU reference for the QTT matrix x dense-vector
product and the solves built on it.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never links or calls it, and the two share no code: the only thing
both sides read is the seeded input data from
``paper_1511_06029_gb300.inputs``.

The arithmetic lives in ``qtt_oracle.c`` (plain C, compiled with
``-ffp-contract=off`` so that every multiply and add rounds separately, the
same on x86-64 and aarch64).  This module only marshals numpy arrays.

An operator is any object with ``.ranks`` (list of d+1 ints, ends equal to 1)
and ``.cores`` (list of d float64 arrays shaped (r_k, 2, 2, r_{k+1}), index
order [alpha_k][row bit i][column bit j][alpha_{k+1}]).  Vectors are numpy
arrays of shape (N,) or (nrhs, N); element t of a vector is indexed least
significant bit first, bit k belonging to core k (Sec. 2.1 and 2.4 of the
paper: Matlab reshape order, finest level first).

Function -> passage it follows:
  apply, apply_ld   y = A x from the TT entry formula (Sec. 2.2, eq.
                    TTdeccores; Sec. 3.1 matrix tensorisation), cores
                    contracted last-to-first (Algorithm 2 runs first-to-last)
  dense             A(i, j) as the chain of slice products (same passages)
  entries           single A(i, j), same formula, for full-size samples
  dense_matvec      brute-force O(N^2) product
  transpose         A^T: row and column bit swapped in every core
  tt_sum            A + B by rank concatenation (Corollary 1, Sec. 3.3)
  tt_product        A B core by core (Sec. 4.2, compressed product)
  solve_direct      x = P f (Tables 1-2 "Solve": inverse applied to dense RHS)
  solve_refine      x <- x + P (f - A x)  (mixed-precision refinement)
  solve_gmres       right-preconditioned GMRES(m) (Sec. 5.3: QTT inverse of
                    the preconditioned system used inside GMRES)
  power_norm        ||K||_2 by power iteration on K^T K
  vec_full          dense vector of a QTT vector (Sec. 2.2 entry formula)
  apply_tt          compressed matrix-vector product c = A b, QTT vector in
                    and out (Sec. 4.2, compressed product equation)
  tt_round          TT rounding with the Algorithm 1 threshold per unfolding
                    (orthogonalisation, then truncated SVDs; numpy QR/SVD)
  tt_svd            QTT decomposition of a dense matrix, Algorithm 1 step by
                    step (truncated SVD of each unfolding; numpy SVD)
  apply_general     y = A x with m_k x n_k modes (Sec. 3.1 tensorisation),
                    rectangular operators included
  local_frames,     the inversion's local system (appendix on local linear
  local_apply       systems): interfaces Psi_{k-1}, Phi_k by their
                    recursions, and the three-core product Psi G_k Phi W_k
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qtt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libqtt_oracle.so")
_lock = threading.Lock()
_lib = None

QO_OK, QO_EINVAL, QO_ENOMEM, QO_ENOTCONV = 0, 1, 2, 4


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle's C source into a shared library (plain gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            I, L, P = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
            D = ctypes.c_double
            sig = {
                "qo_apply": [I, P, P, L, P, L, P, L, I],
                "qo_apply_ld": [I, P, P, L, P, L, P, L, I],
                "qo_dense": [I, P, P, P],
                "qo_dense_matvec": [L, P, L, P, L, P, L],
                "qo_transpose": [I, P, P, P],
                "qo_sum": [I, P, P, P, P, P, P],
                "qo_product": [I, P, P, P, P, P, P],
                "qo_solve_direct": [I, P, P, L, P, P, I],
                "qo_solve_refine": [I, D, P, P, P, P, L, P, P, D, I, P, P, I],
                "qo_solve_gmres": [I, D, P, P, P, P, L, P, P, D, I, I, P, P, I],
                "qo_power_norm": [I, P, P, P, I, D, P, P, I],
                "qo_num_params": [I, P],
                "qo_entries": [I, P, P, L, P, P, P],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            _lib = lib
    return _lib


def _check(st: int, what: str):
    if st == QO_OK:
        return
    names = {QO_EINVAL: "invalid argument", QO_ENOMEM: "out of memory",
             QO_ENOTCONV: "not converged"}
    raise OracleError(f"oracle {what}: {names.get(st, st)}")


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _flat(op):
    ranks = np.ascontiguousarray(np.asarray(op.ranks, dtype=np.int32))
    d = len(ranks) - 1
    for k, c in enumerate(op.cores):
        if c.shape != (ranks[k], 2, 2, ranks[k + 1]):
            raise OracleError(f"core {k} has shape {c.shape}, expected "
                              f"{(ranks[k], 2, 2, ranks[k + 1])}")
    flat = np.ascontiguousarray(
        np.concatenate([np.asarray(c, dtype=np.float64).ravel() for c in op.cores]))
    return d, ranks, flat


class Op:
    """Minimal operator container for results built by the oracle."""

    def __init__(self, ranks, cores):
        self.ranks = [int(v) for v in ranks]
        self.cores = cores

    @property
    def d(self):
        return len(self.ranks) - 1


def _unflat(ranks, flat):
    cores, off = [], 0
    for k in range(len(ranks) - 1):
        n = 4 * ranks[k] * ranks[k + 1]
        cores.append(flat[off:off + n].reshape(ranks[k], 2, 2, ranks[k + 1]).copy())
        off += n
    return Op(ranks, cores)


def _as_block(x, N):
    x = np.asarray(x, dtype=np.float64)
    single = x.ndim == 1
    xb = np.ascontiguousarray(x.reshape(1, -1) if single else x)
    if xb.shape[1] != N:
        raise OracleError(f"vector length {xb.shape[1]} != N = {N}")
    return xb, single


def apply(op, x, threads: int = 0, long_double: bool = False) -> np.ndarray:
    """y = A x (FP64; ``long_double=True`` carries the sweep in long double)."""
    lib = _load()
    d, ranks, flat = _flat(op)
    N = 1 << d
    xb, single = _as_block(x, N)
    y = np.empty_like(xb)
    fn = lib.qo_apply_ld if long_double else lib.qo_apply
    _check(fn(d, _ptr(ranks), _ptr(flat), xb.shape[0], _ptr(xb), N, _ptr(y), N,
              threads), "apply")
    return y[0] if single else y


def dense(op) -> np.ndarray:
    """Dense N x N reconstruction (d <= 13)."""
    lib = _load()
    d, ranks, flat = _flat(op)
    N = 1 << d
    A = np.empty((N, N), dtype=np.float64)
    _check(lib.qo_dense(d, _ptr(ranks), _ptr(flat), _ptr(A)), "dense")
    return A


def entries(op, I, J) -> np.ndarray:
    """A(I[n], J[n]) for index arrays I, J (entry formula, O(d r^2) each)."""
    lib = _load()
    d, ranks, flat = _flat(op)
    I = np.ascontiguousarray(I, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    out = np.empty(I.shape[0], dtype=np.float64)
    _check(lib.qo_entries(d, _ptr(ranks), _ptr(flat), I.shape[0], _ptr(I), _ptr(J),
                          _ptr(out)), "entries")
    return out


def dense_matvec(A, x) -> np.ndarray:
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    N = A.shape[0]
    xb, single = _as_block(x, N)
    y = np.empty_like(xb)
    _check(lib.qo_dense_matvec(N, _ptr(A), xb.shape[0], _ptr(xb), N, _ptr(y), N),
           "dense_matvec")
    return y[0] if single else y


def transpose(op) -> Op:
    lib = _load()
    d, ranks, flat = _flat(op)
    out = np.empty_like(flat)
    _check(lib.qo_transpose(d, _ptr(ranks), _ptr(flat), _ptr(out)), "transpose")
    return _unflat(list(ranks), out)


def tt_sum(A, B) -> Op:
    lib = _load()
    d, ra, fa = _flat(A)
    d2, rb, fb = _flat(B)
    if d != d2:
        raise OracleError("sum of operators with different d")
    rc = np.zeros(d + 1, dtype=np.int32)
    rcl = [1] + [int(ra[k] + rb[k]) for k in range(1, d)] + [1]
    n = sum(4 * rcl[k] * rcl[k + 1] for k in range(d))
    out = np.zeros(n, dtype=np.float64)
    _check(lib.qo_sum(d, _ptr(ra), _ptr(fa), _ptr(rb), _ptr(fb), _ptr(rc), _ptr(out)),
           "sum")
    return _unflat(list(rc), out)


def tt_product(A, B) -> Op:
    lib = _load()
    d, ra, fa = _flat(A)
    d2, rb, fb = _flat(B)
    if d != d2:
        raise OracleError("product of operators with different d")
    rc = np.zeros(d + 1, dtype=np.int32)
    rcl = [int(ra[k] * rb[k]) for k in range(d + 1)]
    n = sum(4 * rcl[k] * rcl[k + 1] for k in range(d))
    out = np.zeros(n, dtype=np.float64)
    _check(lib.qo_product(d, _ptr(ra), _ptr(fa), _ptr(rb), _ptr(fb), _ptr(rc), _ptr(out)),
           "product")
    return _unflat(list(rc), out)


def solve_direct(P, f, threads: int = 0) -> np.ndarray:
    return apply(P, f, threads=threads)


def _solve_common(K, P, f):
    d = len(K.ranks) - 1 if K is not None else len(P.ranks) - 1
    N = 1 << d
    fb, single = _as_block(f, N)
    if K is not None:
        _, rk, gk = _flat(K)
    else:
        rk, gk = np.ones(d + 1, dtype=np.int32), None
    if P is not None:
        _, rp, gp = _flat(P)
    else:
        rp, gp = np.ones(d + 1, dtype=np.int32), None
    return d, N, fb, single, rk, gk, rp, gp


def _gptr(g):
    return None if g is None else _ptr(g)


def solve_refine(K, P, f, a: float = 1.0, tol: float = 1e-13,
                 max_iter: int = 200, threads: int = 0, raise_on_fail=True):
    """Refinement for (a I + K) x = f: x_0 = P f, x <- x + P (f - A x).
    Returns (x, iters, relres)."""
    lib = _load()
    d, N, fb, single, rk, gk, rp, gp = _solve_common(K, P, f)
    x = np.zeros_like(fb)
    nr = fb.shape[0]
    iters = np.zeros(nr, dtype=np.int32)
    rel = np.zeros(nr, dtype=np.float64)
    st = lib.qo_solve_refine(d, a, _ptr(rk), _gptr(gk), _ptr(rp), _gptr(gp), nr,
                             _ptr(fb), _ptr(x), tol, max_iter, _ptr(iters), _ptr(rel),
                             threads)
    if st != QO_ENOTCONV or raise_on_fail:
        _check(st, "refine")
    return (x[0] if single else x), iters, rel


def solve_gmres(K, P, f, a: float = 1.0, tol: float = 1e-13, restart: int = 30,
                max_iter: int = 500, threads: int = 0, raise_on_fail=True):
    """Right-preconditioned GMRES(restart) for (a I + K) x = f, x_0 = 0.
    Returns (x, iters, relres)."""
    lib = _load()
    d, N, fb, single, rk, gk, rp, gp = _solve_common(K, P, f)
    x = np.zeros_like(fb)
    nr = fb.shape[0]
    iters = np.zeros(nr, dtype=np.int32)
    rel = np.zeros(nr, dtype=np.float64)
    st = lib.qo_solve_gmres(d, a, _ptr(rk), _gptr(gk), _ptr(rp), _gptr(gp), nr,
                            _ptr(fb), _ptr(x), tol, restart, max_iter, _ptr(iters),
                            _ptr(rel), threads)
    if st != QO_ENOTCONV or raise_on_fail:
        _check(st, "gmres")
    return (x[0] if single else x), iters, rel


def power_norm(op, v0, max_iter: int = 100, rtol: float = 1e-6, threads: int = 0):
    """||A||_2 estimate by power iteration on A^T A from v0.
    Returns (sigma, iterations)."""
    lib = _load()
    d, ranks, flat = _flat(op)
    v0 = np.ascontiguousarray(v0, dtype=np.float64)
    sigma = ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    _check(lib.qo_power_norm(d, _ptr(ranks), _ptr(flat), _ptr(v0), max_iter, rtol,
                             ctypes.byref(sigma), ctypes.byref(it), threads),
           "power_norm")
    return sigma.value, it.value


# ------------------------------------------------- compressed vectors (numpy)
# A QTT vector has .ranks (s_0 = s_d = 1) and .cores shaped (s_k, 2, s_{k+1}),
# element t = G_1[:, t_1, :] ... G_d[:, t_d, :] with t_k bit k of t (least
# significant first, as for the operators).

class Vec:
    """Minimal QTT-vector container for results built by the oracle."""

    def __init__(self, ranks, cores):
        self.ranks = [int(v) for v in ranks]
        self.cores = cores

    @property
    def d(self):
        return len(self.ranks) - 1


def vec_full(v) -> np.ndarray:
    """Dense vector of a QTT vector from the entry formula (Sec. 2.2):
    contracted last core first; the row index of the running block is the
    already-placed low bits."""
    d = len(v.ranks) - 1
    # block[t_high, alpha]: entries over the bits k..d-1, for rank alpha_k
    block = np.asarray(v.cores[d - 1], dtype=np.float64)[:, :, 0].T  # (2, s_{d-1})
    for k in range(d - 2, -1, -1):
        G = np.asarray(v.cores[k], dtype=np.float64)  # (s_k, 2, s_{k+1})
        # new index = t_k + 2 * t_high: bit k is the least significant here
        nb = np.einsum("aib,hb->hia", G, block)  # (high, t_k, s_k)
        block = nb.reshape(-1, G.shape[0])
    return block[:, 0]


def apply_tt(A, v) -> Vec:
    """Compressed matrix-vector product c = A b (Sec. 4.2, the compressed
    product equation): core k of c is, for every merged rank pair, the sum
    over j_k of A's core slice (alpha_{k-1}, i_k j_k, alpha_k) times b's
    (beta_{k-1}, j_k, beta_k); the pair (alpha, beta) becomes one rank index
    alpha s + beta, so the ranks multiply."""
    d = len(A.ranks) - 1
    if len(v.ranks) - 1 != d:
        raise OracleError("operator and vector have different d")
    cores = []
    for k in range(d):
        GA = np.asarray(A.cores[k], dtype=np.float64)  # (r, 2 i, 2 j, r')
        Gb = np.asarray(v.cores[k], dtype=np.float64)  # (s, 2 j, s')
        C = np.einsum("aijc,bje->abice", GA, Gb)
        r, s, _, rc, se = C.shape
        cores.append(C.reshape(r * s, 2, rc * se))
    return Vec([a * b for a, b in zip(A.ranks, v.ranks)], cores)


def tt_round(t, eps: float):
    """TT rounding of an operator or a vector: left-to-right QR
    orthogonalisation, then right-to-left truncated SVDs, each keeping the
    smallest rank whose discarded singular values have 2-norm <= eps
    ||t||_F / sqrt(d-1) (the threshold of Algorithm 1), so that
    ||t - round(t)||_F <= eps ||t||_F.  Returns the same kind of object."""
    d = len(t.ranks) - 1
    is_op = np.asarray(t.cores[0]).ndim == 4
    cores = [np.asarray(c, dtype=np.float64).reshape(c.shape[0], -1, c.shape[-1]).copy()
             for c in t.cores]
    # left-to-right: cores 0 .. d-2 become left-orthonormal
    for k in range(d - 1):
        ra, n, rb = cores[k].shape
        Q, R = np.linalg.qr(cores[k].reshape(ra * n, rb))
        cores[k] = Q.reshape(ra, n, Q.shape[1])
        nxt = cores[k + 1]
        cores[k + 1] = np.einsum("ab,bnc->anc", R, nxt)
    delta = eps * np.linalg.norm(cores[d - 1]) / np.sqrt(max(d - 1, 1))
    # right-to-left: truncate the unfolding between cores k-1 and k
    for k in range(d - 1, 0, -1):
        ra, n, rb = cores[k].shape
        U, S, Vt = np.linalg.svd(cores[k].reshape(ra, n * rb), full_matrices=False)
        keep = len(S)
        while keep > 1 and np.sqrt(np.sum(S[keep - 1:] ** 2)) <= delta:
            keep -= 1
        cores[k] = Vt[:keep].reshape(keep, n, rb)
        cores[k - 1] = np.einsum("pna,ab->pnb", cores[k - 1], U[:, :keep] * S[:keep])
    ranks = [1] + [c.shape[2] for c in cores[:-1]] + [1]
    if is_op:
        return Op(ranks, [c.reshape(c.shape[0], 2, 2, c.shape[2]) for c in cores])
    return Vec(ranks, cores)


def tt_svd(A: np.ndarray, eps: float) -> Op:
    """QTT decomposition of a dense 2^d x 2^d matrix by Algorithm 1: the
    tensor's modes are the bit pairs (i_k, j_k), k = 0 .. d-1 (index order
    of Sec. 2.1, least significant bit first); each unfolding M_k is split
    by a truncated SVD keeping the smallest rank whose discarded singular
    values have 2-norm <= eps ||A||_F / sqrt(d-1); U_k becomes core k and
    S_k V_k^T the next unfolding.  ||A - A_tt||_F <= eps ||A||_F."""
    A = np.asarray(A, dtype=np.float64)
    N = A.shape[0]
    d = int(round(np.log2(N)))
    if A.shape != (N, N) or (1 << d) != N:
        raise OracleError("tt_svd needs a 2^d x 2^d matrix")
    # A[i, j] with i = sum_k i_k 2^k: C-order axes (i_{d-1} .. i_0, j_{d-1} .. j_0)
    T = A.reshape([2] * (2 * d))
    order = []
    for k in range(d):
        order += [d - 1 - k, 2 * d - 1 - k]          # (i_k, j_k), k = 0 first
    T = np.transpose(T, order)
    delta = eps * np.linalg.norm(A) / np.sqrt(max(d - 1, 1))
    cores, ranks = [], [1]
    M = T.reshape(4, -1)                             # first unfolding, r_0 = 1
    for k in range(d - 1):
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
        keep = len(S)
        while keep > 1 and np.sqrt(np.sum(S[keep - 1:] ** 2)) <= delta:
            keep -= 1
        cores.append(U[:, :keep].reshape(ranks[-1], 2, 2, keep))
        ranks.append(keep)
        M = (S[:keep, None] * Vt[:keep]).reshape(keep * 4, -1)
    cores.append(M.reshape(ranks[-1], 2, 2, 1))
    ranks.append(1)
    return Op(ranks, cores)


def apply_general(cores, x) -> np.ndarray:
    """y = A x for a QTT-format matrix with general mode sizes (Sec. 3.1's
    tensorisation with m_k x n_k modes; rectangular when prod m != prod n).
    cores[k] has shape (r_k, m_k, n_k, r_{k+1}); x has shape (prod n,) or
    (nrhs, prod n) with column index j = sum_k j_k prod_{l<k} n_l (first mode
    fastest, as for the binary case); y's row index likewise.  The sweep
    runs core 0 first, keeping (unused column modes, produced row modes,
    rank) as the state."""
    G = [np.asarray(c, dtype=np.float64) for c in cores]
    x = np.asarray(x, dtype=np.float64)
    single = x.ndim == 1
    X = x.reshape(1, -1) if single else x
    m = [g.shape[1] for g in G]
    n = [g.shape[2] for g in G]
    if X.shape[1] != int(np.prod(n)):
        raise OracleError("x length != prod n_k")
    R = X.shape[0]
    # Z[rhs, remaining high column modes, n_k, produced rows, alpha_k]
    Z = X.reshape(R, -1, n[0], 1, 1)
    for k, g in enumerate(G):
        Y = np.einsum("rhjla,aijb->rhilb", Z, g)        # (R, high, m_k, low, r')
        Y = Y.reshape(R, Y.shape[1], m[k] * Y.shape[3], g.shape[3])
        if k + 1 < len(G):
            Z = Y.reshape(R, Y.shape[1] // n[k + 1], n[k + 1], Y.shape[2], g.shape[3])
        else:
            Z = Y
    y = Z.reshape(R, -1)
    return y[0] if single else y


# ------------------------------------- local system of the inversion sweeps
# For the inversion A X = I with X in QTT form (cores W_k(gamma, j, p,
# gamma'), row bit j, column bit p), fixing every core of X but W_k leaves the
# reduced system P^T (I (x) A) P vec(W_k) = P^T vec(I) (appendix on the local
# linear systems).  Its left-hand side is a three-core QTT matrix-vector
# product with the interfaces Psi_{k-1} (cores before k) and Phi_k (cores
# after k).

def local_frames(G_cores, W_cores, k):
    """(Psi_{k-1}, Phi_k) of the appendix's local-system formula, built by
    their recursions: Psi over cores 0 .. k-1 from Psi = 1, Phi over cores
    d-1 .. k+1 from Phi = 1.  Index order [alpha (A's rank), beta (the
    projected X), gamma (the applied X)]."""
    G = [np.asarray(c, dtype=np.float64) for c in G_cores]
    W = [np.asarray(c, dtype=np.float64) for c in W_cores]
    psi = np.ones((1, 1, 1))
    for l in range(k):
        psi = np.einsum("abc,bipB,aijA,cjpC->ABC", psi, W[l], G[l], W[l])
    phi = np.ones((1, 1, 1))
    for l in range(len(G) - 1, k, -1):
        phi = np.einsum("bipB,aijA,cjpC,ABC->abc", W[l], G[l], W[l], phi)
    return psi, phi


def local_apply(psi, Gk, phi, Wk) -> np.ndarray:
    """The local system's left-hand side applied to W_k: the sum over
    alpha, gamma and j of Psi_{k-1} G_k Phi_k W_k, indexed (beta_{k-1}, i_k,
    p_k, beta_k) -- the appendix's three-core QTT matrix-vector product."""
    return np.einsum("abc,aijA,ABC,cjpC->bipB", psi, np.asarray(Gk, dtype=np.float64), phi,
                     np.asarray(Wk, dtype=np.float64))
