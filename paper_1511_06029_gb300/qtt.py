"""Python binding of libqtt (ctypes; argument marshalling only).

Every step of the apply and the solves runs in the library's CUDA kernels;
this module converts torch tensors to pointers, sizes and streams.  There is
no CPU fallback: if ``libqtt.so`` has not been built, or no GPU is present,
the calls raise.

Names follow the C-ABI in ``include/qtt.h``:

    op = Operator(data, packs=("bf16",))   # qtt_create (data: ranks + cores)
    y  = op.apply(x, compute="f64")        # qtt_apply
    r  = op.residual(f, x, a=1.0)          # qtt_residual
    x, info = solve(K, P, f, kind="gmres") # qtt_solve
    op.close()                             # qtt_destroy
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqtt.so")

QTT_OK, QTT_ERR_INVALID_ARG, QTT_ERR_OOM, QTT_ERR_CUDA = 0, 1, 2, 3
QTT_ERR_NOT_CONVERGED, QTT_ERR_TIMEOUT, QTT_ERR_UNSUPPORTED = 4, 5, 6
QTT_ERR_CHECK = 7
DTYPES = {"f64": 0, "f32": 1, "tf32": 2, "bf16": 3}
PACKS = {"f32": 1 << 1, "tf32": 1 << 2, "bf16": 1 << 3}
SOLVE_KINDS = {"direct": 0, "gmres": 1, "refine": 2}

# Every function the header declares, with its ctypes signature.
_I, _U, _L, _D, _P = ctypes.c_int, ctypes.c_uint, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
SIGNATURES = {
    "qtt_create": (_I, [ctypes.POINTER(_P), _I, _P, _P, _U, _P]),
    "qtt_create_flat": (_I, [ctypes.POINTER(_P), _I, _P, _P, _U, _P]),
    "qtt_destroy": (_I, [_P]),
    "qtt_op_d": (_I, [_P]),
    "qtt_op_rank": (_I, [_P, _I]),
    "qtt_op_flops": (_D, [_P]),
    "qtt_apply": (_I, [_P, _P, _P, _L, _L, _I, _I, _P]),
    "qtt_apply_host": (_I, [_P, _P, _P, _L, _L, _I, _I, _L, _P]),
    "qtt_residual": (_I, [_P, _D, _P, _P, _P, _L, _L, _P]),
    "qtt_apply_noalloc": (_I, [_P, _P, _P, _L, _L, _P]),
    "qtt_apply_tt_size": (_I, [_P, _P, ctypes.POINTER(_L)]),
    "qtt_apply_tt": (_I, [_P, _P, _P, _P, _P]),
    "qtt_selftest_wait": (_I, [_D, _P]),
    "qtt_set_scratch_limit": (_I, [ctypes.c_size_t]),
    "qtt_scratch_stats": (_I, [ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                               ctypes.POINTER(ctypes.c_size_t)]),
    "qtt_plan_create": (_I, [ctypes.POINTER(_P), _P, _P, _P, _L, _L, _I, _I]),
    "qtt_plan_run": (_I, [_P, _P]),
    "qtt_plan_destroy": (_I, [_P]),
    "qtt_solve": (_I, [_P, _P, _P, _P, _L, _L, _P, _P, _P]),
    "qtt_gcreate": (_I, [ctypes.POINTER(_P), _I, _P, _P, _P, _P, _P]),
    "qtt_gapply": (_I, [_P, _P, _P, _L, _L, _L, _I, _P]),
    "qtt_gdestroy": (_I, [_P]),
    "qtt_gop_rows": (_L, [_P]),
    "qtt_gop_cols": (_L, [_P]),
    "qtt_gop_flops": (_D, [_P, _I]),
    "qtt_tt_round": (_I, [_I, _P, _I, _P, _D, _P, _P, _P]),
    "qtt_apply_autotune": (_I, [_P, _L, _I, _I, _P, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "qtt_apply_set_plan": (_I, [_P, _I, _I]),
    "qtt_apply_get_plan": (_I, [_P, _I, ctypes.POINTER(_I)]),
    "qtt_tt_svd": (_I, [_I, _P, _D, _P, _P, _L, ctypes.POINTER(_L), _P]),
    "qtt_local_apply": (_I, [_I, _I, _I, _I, _P, _P, _P, _P, _P, _L, _P]),
    "qtt_op_product": (_I, [_P, _P, _P, _L, _P, _P]),
    "qtt_tt_sum": (_I, [_I, _I, _I, _P, _P, _P, _P, _P, _L, _P]),
    "qtt_status_string": (ctypes.c_char_p, [_I]),
    "qtt_last_error": (ctypes.c_char_p, []),
    "qtt_kernel_launches": (ctypes.c_uint64, []),
    "qtt_sync_status": (_I, [_P]),
    "qtt_batch_create": (_I, [ctypes.POINTER(_P), _I, _P, _P, _P, _P, _P, _I, ctypes.c_size_t, _P]),
    "qtt_batch_run": (_I, [_P, _P]),
    "qtt_batch_run_host": (_I, [_P, _P, _P, _P]),
    "qtt_batch_status": (_I, [_P, _P]),
    "qtt_batch_selftest_timeout": (_I, [_P, _D, _P]),
    "qtt_batch_set_variant": (_I, [_P, _I, _P]),
    "qtt_batch_autotune": (_I, [_P, _I, _P, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "qtt_batch_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                            ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_size_t)]),
    "qtt_batch_direct_ops": (_I, [_P, ctypes.POINTER(_I)]),
    "qtt_checked_build": (_I, []),
    "qtt_check_selftest": (_I, [_P]),
    "qtt_write_file": (_I, [ctypes.c_char_p, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "qtt_read_file": (_I, [ctypes.c_char_p, ctypes.POINTER(_I), ctypes.POINTER(_I), _I,
                           ctypes.POINTER(_D), ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "qtt_batch_destroy": (_I, [_P]),
    "qtt_server_create": (_I, [ctypes.POINTER(_P), _I, ctypes.c_size_t, _P]),
    "qtt_server_submit": (_I, [_P, _P, _P, _P, _P, _L, ctypes.POINTER(_L)]),
    "qtt_server_poll": (_I, [_P, _L, _I, ctypes.POINTER(_I), _P, ctypes.POINTER(_D),
                             ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "qtt_server_stats": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I),
                              ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                              ctypes.POINTER(_I)]),
    "qtt_server_destroy": (_I, [_P]),
    "qtt_server_submit_apply": (_I, [_P, _P, _P, _P, _L, _I, ctypes.POINTER(_L)]),
    "qtt_server_ticks": (_I, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
}


class QTTError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str = ""):
        self.status = status
        super().__init__(f"{where}: status {status} ({msg})")


class SolveParams(ctypes.Structure):
    _fields_ = [("kind", _I), ("a", _D), ("tol", _D), ("restart", _I),
                ("max_iter", _I), ("precond_compute", _I), ("inner_iters", _I)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", _I), ("rel_residual", _D), ("status", _I)]


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load libqtt.so and bind every declared symbol (raises if missing)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise QTTError(-1, "load_library",
                               f"{path} not built; run `python -m paper_1511_06029_gb300.build`")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(st: int, where: str):
    if st != QTT_OK:
        lib = load_library()
        msg = lib.qtt_last_error().decode() or lib.qtt_status_string(st).decode()
        raise QTTError(st, where, msg)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise QTTError(-1, "libqtt", "a CUDA device is required (no CPU fallback)")
    return torch


def _stream_handle(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


_TORCH_DTYPE = {"f64": "float64", "f32": "float32", "tf32": "float32", "bf16": "bfloat16"}


def _io_name(t) -> str:
    torch = _torch()
    m = {torch.float64: "f64", torch.float32: "f32", torch.bfloat16: "bf16"}
    if t.dtype not in m:
        raise QTTError(QTT_ERR_INVALID_ARG, "libqtt", f"unsupported tensor dtype {t.dtype}")
    return m[t.dtype]


def _block(t, N, what, host=False):
    """(nrhs, N) view with unit inner stride -> (nrhs, ld)."""
    if t.is_cuda == host:
        raise QTTError(QTT_ERR_INVALID_ARG, what,
                       "tensor must be in host memory" if host else "tensor must be on the GPU")
    if t.dim() == 1:
        if t.shape[0] != N or t.stride(0) != 1:
            raise QTTError(QTT_ERR_INVALID_ARG, what, "bad vector shape/stride")
        return 1, N
    if t.dim() != 2 or t.shape[1] != N or t.stride(1) != 1:
        raise QTTError(QTT_ERR_INVALID_ARG, what, f"expected (nrhs, {N}) with unit stride")
    if t.shape[0] > 1 and t.stride(0) < N:
        raise QTTError(QTT_ERR_INVALID_ARG, what, "rows overlap (row stride < N)")
    return t.shape[0], (t.stride(0) if t.shape[0] > 1 else N)


class Plan:
    """One apply recorded as a CUDA graph (qtt_plan_*): x and out are fixed,
    their contents are read and written at every run()."""

    def __init__(self, op, x, out, compute="f64"):
        nrhs, ld = _block(x, op.N, "qtt_plan_create")
        n2, ld2 = _block(out, op.N, "qtt_plan_create")
        if n2 != nrhs or ld2 != ld or out.dtype != x.dtype:
            raise QTTError(QTT_ERR_INVALID_ARG, "qtt_plan_create", "out shape/stride/dtype mismatch")
        self.op, self.x, self.out = op, x, out  # keep the operator and buffers alive
        h = _P()
        _check(load_library().qtt_plan_create(ctypes.byref(h), op.handle,
                                              ctypes.c_void_p(x.data_ptr()),
                                              ctypes.c_void_p(out.data_ptr()), nrhs, ld,
                                              DTYPES[_io_name(x)], DTYPES[compute]),
               "qtt_plan_create")
        self.handle = h

    def run(self, stream=None):
        _check(load_library().qtt_plan_run(self.handle, _stream_handle(stream)), "qtt_plan_run")
        return self.out

    def close(self):
        if getattr(self, "handle", None):
            load_library().qtt_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Operator:
    """A QTT matrix resident on the GPU (qtt_create / qtt_destroy)."""

    def __init__(self, data, packs=(), stream=None):
        lib = load_library()
        _torch()
        ranks = np.ascontiguousarray(np.asarray(data.ranks, dtype=np.int32))
        d = len(ranks) - 1
        cores = [np.ascontiguousarray(c, dtype=np.float64) for c in data.cores]
        flat = np.ascontiguousarray(np.concatenate([c.ravel() for c in cores]))
        mask = 0
        for p in packs:
            mask |= PACKS[p]
        h = ctypes.c_void_p()
        ptrs = (ctypes.c_void_p * d)(*[c.ctypes.data for c in cores])
        _check(lib.qtt_create(ctypes.byref(h), d, ranks.ctypes.data_as(_P),
                              ctypes.cast(ptrs, _P), mask, _stream_handle(stream)),
               "qtt_create")
        self._h = h
        self.d = d
        self.N = 1 << d
        self.ranks = [int(v) for v in ranks]
        self.packs = tuple(packs)
        self._flat = flat

    def host_cores_flat(self):
        """The FP64 cores given at creation, back to back (host copy)."""
        return self._flat

    @property
    def handle(self):
        if self._h is None:
            raise QTTError(QTT_ERR_INVALID_ARG, "Operator", "operator was closed")
        return self._h

    def flops(self, nrhs: int = 1) -> float:
        return load_library().qtt_op_flops(self.handle) * nrhs

    def apply(self, x, out=None, compute: str = "f64", stream=None):
        """y = A x on the GPU (qtt_apply).  x: (N,) or (nrhs, N) CUDA tensor of
        float64 / float32 / bfloat16; y has the same dtype and shape."""
        torch = _torch()
        nrhs, ld = _block(x, self.N, "qtt_apply")
        if out is None:
            out = torch.empty_like(x, memory_format=torch.contiguous_format)
        n2, ld2 = _block(out, self.N, "qtt_apply")
        if n2 != nrhs or out.dtype != x.dtype:
            raise QTTError(QTT_ERR_INVALID_ARG, "qtt_apply", "out shape/dtype mismatch")
        if ld2 != ld:
            raise QTTError(QTT_ERR_INVALID_ARG, "qtt_apply", "x and out need the same row stride")
        io = _io_name(x)
        _check(load_library().qtt_apply(self.handle, ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), nrhs, ld,
                                        DTYPES[io], DTYPES[compute], _stream_handle(stream)),
               "qtt_apply")
        return out

    def apply_host(self, x, out=None, compute: str = "f64", chunk: int = 0, stream=None):
        """y = A x with x and y in host memory (qtt_apply_host): the copies to
        and from the device are part of the call, overlapped with the applies
        chunk by chunk.  x: (N,) or (nrhs, N) CPU tensor of float64 / float32 /
        bfloat16, best page-locked (x.pin_memory()); y has the same dtype and
        shape (a page-locked tensor is made when `out` is not given).  The call
        returns once the work is queued on `stream`; synchronise the stream
        before reading y."""
        torch = _torch()
        nrhs, ld = _block(x, self.N, "qtt_apply_host", host=True)
        if out is None:
            out = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
        n2, ld2 = _block(out, self.N, "qtt_apply_host", host=True)
        if n2 != nrhs or out.dtype != x.dtype:
            raise QTTError(QTT_ERR_INVALID_ARG, "qtt_apply_host", "out shape/dtype mismatch")
        if ld2 != ld:
            raise QTTError(QTT_ERR_INVALID_ARG, "qtt_apply_host",
                           "x and out need the same row stride")
        io = _io_name(x)
        _check(load_library().qtt_apply_host(self.handle, ctypes.c_void_p(x.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr()), nrhs, ld,
                                             DTYPES[io], DTYPES[compute], int(chunk),
                                             _stream_handle(stream)),
               "qtt_apply_host")
        return out

    def apply_tt(self, b_ranks, b_cores, out=None, stream=None):
        """Compressed product c = A b for a QTT vector b (qtt_apply_tt).
        b_ranks: d + 1 ints; b_cores: CUDA float64 tensor of b's cores back to
        back (core k [s_k][2][s_{k+1}]).  Returns (c_ranks, c_cores) with
        c_cores a CUDA float64 tensor of c's cores back to back (core k
        [r_k s_k][2][r_{k+1} s_{k+1}]), written into `out` when given."""
        torch = _torch()
        lib = load_library()
        br = np.ascontiguousarray(np.asarray(b_ranks, dtype=np.int32))
        if br.shape != (self.d + 1,):
            raise QTTError(QTT_ERR_INVALID_ARG, "qtt_apply_tt", "b_ranks needs d + 1 entries")
        if not (b_cores.is_cuda and b_cores.dtype == torch.float64 and b_cores.is_contiguous()):
            raise QTTError(QTT_ERR_INVALID_ARG, "qtt_apply_tt",
                           "b_cores must be a contiguous CUDA float64 tensor")
        need = sum(2 * int(br[k]) * int(br[k + 1]) for k in range(self.d))
        if b_cores.numel() != need:
            raise QTTError(QTT_ERR_INVALID_ARG, "qtt_apply_tt", f"b_cores needs {need} elements")
        n = ctypes.c_int64(0)
        _check(lib.qtt_apply_tt_size(self.handle, br.ctypes.data_as(_P), ctypes.byref(n)),
               "qtt_apply_tt_size")
        if out is None:
            out = torch.empty(n.value, dtype=torch.float64, device=b_cores.device)
        elif not (out.is_cuda and out.dtype == torch.float64 and out.is_contiguous()
                  and out.numel() == n.value):
            raise QTTError(QTT_ERR_INVALID_ARG, "qtt_apply_tt",
                           f"out must be a contiguous CUDA float64 tensor of {n.value} elements")
        _check(lib.qtt_apply_tt(self.handle, br.ctypes.data_as(_P),
                                ctypes.c_void_p(b_cores.data_ptr()),
                                ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
               "qtt_apply_tt")
        return [a * int(b) for a, b in zip(self.ranks, br)], out

    def autotune(self, nrhs: int, compute: str = "bf16", reps: int = 2, cache=None, stream=None):
        """Pick the fastest fusion plan for applies of nrhs right-hand sides in
        `compute` (qtt_apply_autotune).  With `cache` (a JSON path; default
        $QTT_PLAN_CACHE when set) a plan found earlier for the same d, ranks,
        nrhs and arithmetic is reused instead of timed, and a new choice is
        stored.  Returns (plan code, seconds per apply or None if cached)."""
        import json
        import zlib
        cache = cache or os.environ.get("QTT_PLAN_CACHE")
        key = (f"d{self.d}_r{zlib.crc32(np.asarray(self.ranks, dtype=np.int32).tobytes()):08x}"
               f"_n{int(nrhs)}_{compute}")
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as fh:
                table = json.load(fh)
        if key in table:
            _check(load_library().qtt_apply_set_plan(self.handle, DTYPES[compute],
                                                     int(table[key]["plan"])),
                   "qtt_apply_set_plan")
            return int(table[key]["plan"]), None
        plan, sec = ctypes.c_int(0), ctypes.c_double(0.0)
        _check(load_library().qtt_apply_autotune(self.handle, int(nrhs), DTYPES[compute], int(reps),
                                                 _stream_handle(stream), ctypes.byref(plan),
                                                 ctypes.byref(sec)), "qtt_apply_autotune")
        if cache:
            table[key] = {"plan": plan.value, "seconds": sec.value}
            tmp = cache + f".tmp{os.getpid()}"
            os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
            with open(tmp, "w") as fh:
                json.dump(table, fh, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return plan.value, sec.value

    def set_plan(self, compute: str, plan: int):
        _check(load_library().qtt_apply_set_plan(self.handle, DTYPES[compute], int(plan)),
               "qtt_apply_set_plan")

    def get_plan(self, compute: str) -> int:
        v = ctypes.c_int(0)
        _check(load_library().qtt_apply_get_plan(self.handle, DTYPES[compute], ctypes.byref(v)),
               "qtt_apply_get_plan")
        return v.value

    def plan(self, x, out, compute: str = "f64"):
        """Record y = A x for these two tensors as a CUDA graph (qtt_plan_create);
        Plan.run() replays it on whatever x holds at that time."""
        return Plan(self, x, out, compute)

    def residual(self, f, x, a: float = 1.0, out=None, stream=None):
        """r = f - (a x + K x) in FP64 (qtt_residual)."""
        torch = _torch()
        nrhs, ld = _block(f, self.N, "qtt_residual")
        if out is None:
            out = torch.empty_like(f)
        for t in (x, out):
            n2, ld2 = _block(t, self.N, "qtt_residual")
            if n2 != nrhs or ld2 != ld or t.dtype != torch.float64:
                raise QTTError(QTT_ERR_INVALID_ARG, "qtt_residual", "shape/stride/dtype mismatch")
        _check(load_library().qtt_residual(self.handle, a, ctypes.c_void_p(f.data_ptr()),
                                           ctypes.c_void_p(x.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), nrhs, ld,
                                           _stream_handle(stream)), "qtt_residual")
        return out

    def close(self):
        if self._h is not None:
            load_library().qtt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _dev_f64(t, what):
    torch = _torch()
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise QTTError(QTT_ERR_INVALID_ARG, what, "expected a contiguous CUDA float64 tensor")
    return ctypes.c_void_p(t.data_ptr())


def tt_round(ranks, n, cores, eps, out=None, stream=None):
    """TT rounding on the GPU (qtt_tt_round).  cores: CUDA float64 tensor of
    the cores back to back, core k [r_k][n][r_{k+1}] (n = 2 for a QTT vector,
    4 for a binary QTT matrix).  Returns (new ranks, tensor of the rounded
    cores back to back)."""
    torch = _torch()
    r = np.ascontiguousarray(np.asarray(ranks, dtype=np.int32))
    d = len(r) - 1
    need = sum(int(r[k]) * n * int(r[k + 1]) for k in range(d))
    if cores.numel() != need:
        raise QTTError(QTT_ERR_INVALID_ARG, "qtt_tt_round", f"cores need {need} elements")
    if out is None:
        out = torch.empty_like(cores)
    ro = np.zeros(d + 1, dtype=np.int32)
    _check(load_library().qtt_tt_round(d, r.ctypes.data_as(_P), int(n),
                                       _dev_f64(cores, "qtt_tt_round"), float(eps),
                                       ro.ctypes.data_as(_P), _dev_f64(out, "qtt_tt_round"),
                                       _stream_handle(stream)), "qtt_tt_round")
    size = sum(int(ro[k]) * n * int(ro[k + 1]) for k in range(d))
    return [int(v) for v in ro], out[:size]


def tt_svd(A, eps, stream=None):
    """Algorithm 1 on the GPU (qtt_tt_svd): A a CUDA float64 (2^d, 2^d)
    tensor.  Returns (ranks, cores back to back as a CUDA tensor, each core
    [r_k][2 i][2 j][r_{k+1}])."""
    torch = _torch()
    N = A.shape[0]
    d = int(N).bit_length() - 1
    if A.dim() != 2 or A.shape[1] != N or (1 << d) != N:
        raise QTTError(QTT_ERR_INVALID_ARG, "qtt_tt_svd", "A must be 2^d x 2^d")
    lib = load_library()
    ro = np.zeros(d + 1, dtype=np.int32)
    need = ctypes.c_int64(0)
    # first call sizes the output (nothing is written), second fills it
    cap = 4 * sum(min(4 ** k, 4 ** (d - k)) * min(4 ** (k + 1), 4 ** (d - k - 1)) for k in range(d))
    cap = min(cap, 1 << 26)
    out = torch.empty(cap, dtype=torch.float64, device=A.device)
    st = lib.qtt_tt_svd(d, _dev_f64(A, "qtt_tt_svd"), float(eps), ro.ctypes.data_as(_P),
                        ctypes.c_void_p(out.data_ptr()), cap, ctypes.byref(need),
                        _stream_handle(stream))
    if st == QTT_ERR_INVALID_ARG and need.value > cap:
        out = torch.empty(need.value, dtype=torch.float64, device=A.device)
        st = lib.qtt_tt_svd(d, _dev_f64(A, "qtt_tt_svd"), float(eps), ro.ctypes.data_as(_P),
                            ctypes.c_void_p(out.data_ptr()), need.value, ctypes.byref(need),
                            _stream_handle(stream))
    _check(st, "qtt_tt_svd")
    return [int(v) for v in ro], out[:need.value]


def op_product(A, B, stream=None):
    """C = A B core by core on the GPU (qtt_op_product).  Returns (ranks, CUDA
    float64 tensor of C's cores back to back, [r][2][2][r'] each)."""
    torch = _torch()
    if A.d != B.d:
        raise QTTError(QTT_ERR_INVALID_ARG, "qtt_op_product", "operators differ in d")
    rc = [a * b for a, b in zip(A.ranks, B.ranks)]
    n = 4 * sum(rc[k] * rc[k + 1] for k in range(A.d))
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    ro = np.zeros(A.d + 1, dtype=np.int32)
    _check(load_library().qtt_op_product(A.handle, B.handle, ctypes.c_void_p(out.data_ptr()), n,
                                         ro.ctypes.data_as(_P), _stream_handle(stream)),
           "qtt_op_product")
    return [int(v) for v in ro], out


def tt_sum(terms, n, stream=None):
    """sum_t c_t T_t on the GPU (qtt_tt_sum).  terms: list of (coef, ranks,
    CUDA float64 cores back to back); n entries per mode.  Returns (ranks,
    cores)."""
    torch = _torch()
    d = len(terms[0][1]) - 1
    rk = [np.ascontiguousarray(np.asarray(r, dtype=np.int32)) for _, r, _ in terms]
    R = [1] + [sum(int(r[k]) for r in rk) for k in range(1, d)] + [1]
    size = sum(n * R[k] * R[k + 1] for k in range(d))
    out = torch.empty(size, dtype=torch.float64, device="cuda")
    T = len(terms)
    rptr = (_P * T)(*[r.ctypes.data_as(_P) for r in rk])
    cptr = (_P * T)(*[_dev_f64(c, "qtt_tt_sum").value for _, _, c in terms])
    coef = (ctypes.c_double * T)(*[float(c) for c, _, _ in terms])
    ro = np.zeros(d + 1, dtype=np.int32)
    _check(load_library().qtt_tt_sum(d, int(n), T, ctypes.cast(rptr, _P), ctypes.cast(cptr, _P),
                                     ctypes.cast(coef, _P), ro.ctypes.data_as(_P),
                                     ctypes.c_void_p(out.data_ptr()), size,
                                     _stream_handle(stream)), "qtt_tt_sum")
    return [int(v) for v in ro], out


def neumann_preconditioner(K, eps, stream=None):
    """P = round(I - K + K^2, eps) built on the GPU from the operator K
    (qtt_op_product, qtt_tt_sum, qtt_tt_round).  Returns (ranks, host list
    of cores shaped (r, 2, 2, r'))."""
    torch = _torch()
    d = K.d
    r2, k2 = op_product(K, K, stream)
    kflat = torch.from_numpy(np.ascontiguousarray(K.host_cores_flat())).cuda()
    ident = torch.from_numpy(np.tile(np.eye(2).ravel(), d)).cuda()
    rs, s = tt_sum([(1.0, [1] * (d + 1), ident), (-1.0, K.ranks, kflat), (1.0, r2, k2)], 4, stream)
    rp, p = tt_round(rs, 4, s, eps, stream=stream)
    host = p.cpu().numpy()
    cores, off = [], 0
    for k in range(d):
        sz = 4 * rp[k] * rp[k + 1]
        cores.append(host[off:off + sz].reshape(rp[k], 2, 2, rp[k + 1]))
        off += sz
    return rp, cores


def local_apply(psi, G, phi, W, out=None, stream=None):
    """The inversion's local-system product (qtt_local_apply): psi (ra, rx,
    rx), G (ra, 2, 2, ra2), phi (ra2, rx2, rx2), W (nvec, rx, 2, 2, rx2) or
    (rx, 2, 2, rx2); CUDA float64.  Returns y shaped like W."""
    torch = _torch()
    ra, rx = psi.shape[0], psi.shape[1]
    ra2, rx2 = phi.shape[0], phi.shape[1]
    if (psi.shape != (ra, rx, rx) or G.shape != (ra, 2, 2, ra2) or phi.shape != (ra2, rx2, rx2)
            or W.shape[-4:] != (rx, 2, 2, rx2)):
        raise QTTError(QTT_ERR_INVALID_ARG, "qtt_local_apply", "inconsistent shapes")
    nvec = 1 if W.dim() == 4 else W.shape[0]
    if out is None:
        out = torch.empty_like(W)
    _check(load_library().qtt_local_apply(ra, ra2, rx, rx2, _dev_f64(psi, "psi"), _dev_f64(G, "G"),
                                          _dev_f64(phi, "phi"), _dev_f64(W, "W"),
                                          _dev_f64(out, "y"), nvec, _stream_handle(stream)),
           "qtt_local_apply")
    return out


class GeneralOperator:
    """A QTT matrix with m_k x n_k modes (qtt_gcreate / qtt_gdestroy).
    cores[k]: array shaped (r_k, m_k, n_k, r_{k+1}); rectangular when
    prod m != prod n."""

    def __init__(self, cores, stream=None):
        lib = load_library()
        _torch()
        cores = [np.ascontiguousarray(c, dtype=np.float64) for c in cores]
        d = len(cores)
        ranks = np.array([1] + [c.shape[3] for c in cores], dtype=np.int32)
        m = np.array([c.shape[1] for c in cores], dtype=np.int32)
        n = np.array([c.shape[2] for c in cores], dtype=np.int32)
        for k, c in enumerate(cores):
            if c.ndim != 4 or c.shape[0] != ranks[k]:
                raise QTTError(QTT_ERR_INVALID_ARG, "qtt_gcreate", f"core {k} has shape {c.shape}")
        flat = np.ascontiguousarray(np.concatenate([c.ravel() for c in cores]))
        h = ctypes.c_void_p()
        _check(lib.qtt_gcreate(ctypes.byref(h), d, ranks.ctypes.data_as(_P), m.ctypes.data_as(_P),
                               n.ctypes.data_as(_P), flat.ctypes.data_as(_P),
                               _stream_handle(stream)), "qtt_gcreate")
        self._h = h
        self.d = d
        self.ranks = [int(v) for v in ranks]
        self.m, self.n = [int(v) for v in m], [int(v) for v in n]
        self.rows = int(lib.qtt_gop_rows(h))
        self.cols = int(lib.qtt_gop_cols(h))

    def flops(self, nrhs: int = 1, transpose: bool = False) -> float:
        return load_library().qtt_gop_flops(self._h, 1 if transpose else 0) * nrhs

    def apply(self, x, out=None, transpose: bool = False, stream=None):
        """y = A x (or A^T x): x a CUDA float64 tensor (len,) or (nrhs, len)."""
        torch = _torch()
        nin, nout = (self.rows, self.cols) if transpose else (self.cols, self.rows)
        nrhs, ldx = _block(x, nin, "qtt_gapply")
        if out is None:
            out = torch.empty((nout,) if x.dim() == 1 else (nrhs, nout), dtype=torch.float64,
                              device=x.device)
        n2, ldy = _block(out, nout, "qtt_gapply")
        if n2 != nrhs or x.dtype != torch.float64 or out.dtype != torch.float64:
            raise QTTError(QTT_ERR_INVALID_ARG, "qtt_gapply", "shape/dtype mismatch")
        _check(load_library().qtt_gapply(self._h, ctypes.c_void_p(x.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), nrhs, ldx, ldy,
                                         1 if transpose else 0, _stream_handle(stream)),
               "qtt_gapply")
        return out

    def close(self):
        if self._h is not None:
            load_library().qtt_gdestroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(K, P, f, kind: str = "gmres", a: float = 1.0, tol: float = 1e-10,
          restart: int = 30, max_iter: int = 300, precond_compute: str = "f64",
          inner_iters: int = 0, out=None, stream=None, raise_on_fail: bool = True):
    """Solve (a I + K) x = f (qtt_solve).  Returns (x, info) with info a list
    of (iters, rel_residual, status) per right-hand side."""
    torch = _torch()
    N = (K or P).N
    nrhs, ld = _block(f, N, "qtt_solve")
    if out is None:
        out = torch.empty_like(f)
    prm = SolveParams(SOLVE_KINDS[kind], a, tol, restart, max_iter, DTYPES[precond_compute],
                      inner_iters)
    info = (SolveInfo * nrhs)()
    st = load_library().qtt_solve(K.handle if K is not None else None,
                                  P.handle if P is not None else None,
                                  ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  nrhs, ld, ctypes.byref(prm), info, _stream_handle(stream))
    if st != QTT_OK and (st != QTT_ERR_NOT_CONVERGED or raise_on_fail):
        _check(st, "qtt_solve")
    return out, [(i.iters, i.rel_residual, i.status) for i in info]


class Batch:
    """Many uneven operators applied in one persistent launch per memory wave,
    replayed from a CUDA graph (qtt_batch_*).  xs/ys: lists of FP32 CUDA
    tensors shaped (nrhs_i, N_i); they stay bound to the batch."""

    def __init__(self, ops, xs, ys, compute="f32", mem_budget=0, stream=None):
        lib = load_library()
        n = len(ops)
        if not (n == len(xs) == len(ys)) or n == 0:
            raise QTTError(QTT_ERR_INVALID_ARG, "Batch", "ops, xs, ys must have equal length")
        nrhs, lds = [], []
        for op, x, y in zip(ops, xs, ys):
            nr, ld = _block(x, op.N, "qtt_batch_create")
            nr2, ld2 = _block(y, op.N, "qtt_batch_create")
            if nr != nr2 or ld != ld2 or x.dtype != y.dtype:
                raise QTTError(QTT_ERR_INVALID_ARG, "qtt_batch_create", "x/y mismatch")
            nrhs.append(nr)
            lds.append(ld)
        self._keep = (list(ops), list(xs), list(ys))
        arr = lambda vals, ct: (ct * n)(*vals)
        h = ctypes.c_void_p()
        _check(lib.qtt_batch_create(ctypes.byref(h), n,
                                    ctypes.cast(arr([o.handle for o in ops], _P), _P),
                                    ctypes.cast(arr(nrhs, ctypes.c_int64), _P),
                                    ctypes.cast(arr([x.data_ptr() for x in xs], _P), _P),
                                    ctypes.cast(arr([y.data_ptr() for y in ys], _P), _P),
                                    ctypes.cast(arr(lds, ctypes.c_int64), _P),
                                    DTYPES[compute], mem_budget, _stream_handle(stream)),
               "qtt_batch_create")
        self._h = h

    def run(self, stream=None):
        _check(load_library().qtt_batch_run(self._h, _stream_handle(stream)), "qtt_batch_run")

    def run_host(self, xs_host, ys_host, stream=None):
        """The run with every operator's vectors in host memory
        (qtt_batch_run_host): xs_host / ys_host are lists of contiguous FP32
        CPU tensors shaped like the batch's xs / ys, best page-locked; the
        copies overlap the run.  Returns once queued on `stream`."""
        torch = _torch()
        ops, xs, _ = self._keep
        if not (len(xs_host) == len(ys_host) == len(ops)):
            raise QTTError(QTT_ERR_INVALID_ARG, "qtt_batch_run_host", "one x and y per operator")
        for x, xh, yh in zip(xs, xs_host, ys_host):
            for t in (xh, yh):
                if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() \
                        or t.numel() != x.numel():
                    raise QTTError(QTT_ERR_INVALID_ARG, "qtt_batch_run_host",
                                   "host vectors: contiguous FP32 CPU tensors of nrhs x N")
        n = len(ops)
        xp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in xs_host])
        yp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in ys_host])
        self._host_keep = (xs_host, ys_host)
        _check(load_library().qtt_batch_run_host(self._h, ctypes.cast(xp, _P), ctypes.cast(yp, _P),
                                                 _stream_handle(stream)), "qtt_batch_run_host")

    def status(self, stream=None):
        _check(load_library().qtt_batch_status(self._h, _stream_handle(stream)), "qtt_batch_status")

    def selftest_timeout(self, seconds, stream=None):
        """Run the first wave with a withheld dependency (qtt_batch_selftest_timeout);
        the next status() raises QTT_ERR_TIMEOUT."""
        _check(load_library().qtt_batch_selftest_timeout(self._h, float(seconds),
                                                         _stream_handle(stream)),
               "qtt_batch_selftest_timeout")

    def set_variant(self, v, stream=None):
        _check(load_library().qtt_batch_set_variant(self._h, v, _stream_handle(stream)),
               "qtt_batch_set_variant")

    def autotune(self, reps=2, stream=None):
        v, t = ctypes.c_int(0), ctypes.c_double(0.0)
        _check(load_library().qtt_batch_autotune(self._h, reps, _stream_handle(stream),
                                                 ctypes.byref(v), ctypes.byref(t)),
               "qtt_batch_autotune")
        return v.value, t.value

    def info(self):
        w, v, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        f, sb = ctypes.c_double(), ctypes.c_size_t()
        _check(load_library().qtt_batch_info(self._h, ctypes.byref(w), ctypes.byref(v),
                                             ctypes.byref(g), ctypes.byref(f), ctypes.byref(sb)),
               "qtt_batch_info")
        t = ctypes.c_int()
        _check(load_library().qtt_batch_direct_ops(self._h, ctypes.byref(t)),
               "qtt_batch_direct_ops")
        return {"waves": w.value, "variant": v.value, "grid": g.value, "flops": f.value,
                "scratch_bytes": sb.value, "direct_ops": t.value}

    def close(self):
        if self._h is not None:
            load_library().qtt_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching solve and apply server (qtt_server_*).  submit()
    and submit_apply() take host numpy arrays (nrhs, N) float64; the result
    lands in the returned array when poll()/wait() reports the request
    done."""

    def __init__(self, slots=4, mem_budget=0, kind="gmres", a=1.0, tol=1e-10, restart=30,
                 max_iter=300, precond_compute="bf16", inner_iters=0):
        lib = load_library()
        _torch()
        self.prm = SolveParams(SOLVE_KINDS[kind], a, tol, restart, max_iter,
                               DTYPES[precond_compute], inner_iters)
        h = ctypes.c_void_p()
        _check(lib.qtt_server_create(ctypes.byref(h), slots, mem_budget, ctypes.byref(self.prm)),
               "qtt_server_create")
        self._h = h
        self._live = {}

    def submit(self, K, P, f):
        f = np.ascontiguousarray(np.atleast_2d(np.asarray(f, dtype=np.float64)))
        x = np.empty_like(f)
        rid = ctypes.c_int64()
        _check(load_library().qtt_server_submit(
            self._h, K.handle if K is not None else None, P.handle if P is not None else None,
            f.ctypes.data_as(_P), x.ctypes.data_as(_P), f.shape[0], ctypes.byref(rid)),
            "qtt_server_submit")
        self._live[rid.value] = (f, x)
        return rid.value

    def submit_apply(self, A, x, compute="f64"):
        """y = A x as a served request (host arrays (nrhs, N) float64)."""
        x = np.ascontiguousarray(np.atleast_2d(np.asarray(x, dtype=np.float64)))
        y = np.empty_like(x)
        rid = ctypes.c_int64()
        _check(load_library().qtt_server_submit_apply(
            self._h, A.handle, x.ctypes.data_as(_P), y.ctypes.data_as(_P), x.shape[0],
            DTYPES[compute], ctypes.byref(rid)), "qtt_server_submit_apply")
        self._live[rid.value] = (x, y)
        return rid.value

    def ticks(self):
        """(ticks run, grouped launches issued) so far (qtt_server_ticks)."""
        t, g = ctypes.c_uint64(), ctypes.c_uint64()
        _check(load_library().qtt_server_ticks(self._h, ctypes.byref(t), ctypes.byref(g)),
               "qtt_server_ticks")
        return t.value, g.value

    def poll(self, rid, wait=False):
        """None while running; else (x, info, (t_submit, t_admit, t_finish))."""
        f, x = self._live[rid]
        done = ctypes.c_int()
        info = (SolveInfo * f.shape[0])()
        ts, ta, tf = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        st = load_library().qtt_server_poll(self._h, rid, 1 if wait else 0, ctypes.byref(done),
                                            info, ctypes.byref(ts), ctypes.byref(ta),
                                            ctypes.byref(tf))
        if not done.value:
            _check(st, "qtt_server_poll")
            return None
        del self._live[rid]
        _check(st, "qtt_server_poll")
        return x, [(i.iters, i.rel_residual, i.status) for i in info], (ts.value, ta.value, tf.value)

    def wait(self, rid):
        return self.poll(rid, wait=True)

    def stats(self):
        p, r, pi = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        iu, piu = ctypes.c_size_t(), ctypes.c_size_t()
        _check(load_library().qtt_server_stats(self._h, ctypes.byref(p), ctypes.byref(r),
                                               ctypes.byref(iu), ctypes.byref(piu),
                                               ctypes.byref(pi)), "qtt_server_stats")
        return {"pending": p.value, "running": r.value, "in_use": iu.value,
                "peak_in_use": piu.value, "peak_running": pi.value}

    def close(self):
        if self._h is not None:
            load_library().qtt_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_launches() -> int:
    """Kernels the library has launched so far (qtt_kernel_launches)."""
    return int(load_library().qtt_kernel_launches())


def write_file(path: str, ranks, cores) -> None:
    """Write an operator (ranks[0..d], cores[k] shaped (r_k, 2, 2, r_{k+1}))
    as a .qtt file (qtt_write_file)."""
    ranks = [int(r) for r in ranks]
    flat = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.float64).ravel()
                                                for c in cores]))
    rk = (ctypes.c_int * len(ranks))(*ranks)
    _check(load_library().qtt_write_file(os.fsencode(path), len(ranks) - 1, rk,
                                         flat.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "qtt_write_file")


def read_file(path: str):
    """Read a .qtt file (qtt_read_file): returns (ranks, cores), cores[k]
    shaped (r_k, 2, 2, r_{k+1})."""
    lib = load_library()
    d, n = ctypes.c_int(), ctypes.c_int64()
    _check(lib.qtt_read_file(os.fsencode(path), ctypes.byref(d), None, 0, None, 0,
                             ctypes.byref(n)), "qtt_read_file")
    rk = (ctypes.c_int * (d.value + 1))()
    flat = np.empty(n.value, dtype=np.float64)
    _check(lib.qtt_read_file(os.fsencode(path), ctypes.byref(d), rk, d.value + 1,
                             flat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n.value,
                             ctypes.byref(n)), "qtt_read_file")
    ranks = list(rk)
    cores, o = [], 0
    for k in range(d.value):
        sz = 4 * ranks[k] * ranks[k + 1]
        cores.append(flat[o:o + sz].reshape(ranks[k], 2, 2, ranks[k + 1]).copy())
        o += sz
    return ranks, cores


def selftest_wait(seconds: float, stream=None):
    """Launch a kernel whose bounded device wait runs out after `seconds`
    (qtt_selftest_wait); the next sync_status() raises QTT_ERR_TIMEOUT."""
    _check(load_library().qtt_selftest_wait(float(seconds), _stream_handle(stream)),
           "qtt_selftest_wait")


def set_scratch_limit(nbytes: int):
    """Cap the library's scratch at `nbytes` (0 = no cap; qtt_set_scratch_limit)."""
    _check(load_library().qtt_set_scratch_limit(int(nbytes)), "qtt_set_scratch_limit")


def scratch_stats():
    """{'in_use', 'pool_reserved', 'pool_used'} in bytes (qtt_scratch_stats)."""
    a, b, c = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(load_library().qtt_scratch_stats(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "qtt_scratch_stats")
    return {"in_use": a.value, "pool_reserved": b.value, "pool_used": c.value}


def sync_status(stream=None):
    _check(load_library().qtt_sync_status(_stream_handle(stream)), "qtt_sync_status")
