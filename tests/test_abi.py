"""The C-ABI library builds, loads and exports every symbol that
include/qtt.h declares; argument validation that needs no GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(qtt_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1511_06029_gb300 import build, qtt
    build.build()
    return qtt.load_library()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("qtt_create", "qtt_apply", "qtt_solve", "qtt_destroy",
                     "qtt_status_string", "qtt_sync_status"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1511_06029_gb300 import qtt
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert name in qtt.SIGNATURES, f"binding lacks {name}"


def test_status_strings(lib):
    for s in range(7):
        assert lib.qtt_status_string(s)
    assert lib.qtt_status_string(99) == b"unknown status"


def test_create_rejects_bad_arguments_without_gpu(lib):
    from paper_1511_06029_gb300 import qtt
    h = ctypes.c_void_p()
    cores = np.zeros(64, dtype=np.float64)
    P = ctypes.c_void_p

    def create(d, ranks, mask=0):
        r = np.asarray(ranks, dtype=np.int32)
        return lib.qtt_create_flat(ctypes.byref(h), d, r.ctypes.data_as(P),
                                   cores.ctypes.data_as(P), mask, None)

    assert create(0, [1]) == qtt.QTT_ERR_INVALID_ARG
    assert create(31, [1] * 32) == qtt.QTT_ERR_INVALID_ARG
    assert create(2, [2, 1, 1]) == qtt.QTT_ERR_INVALID_ARG
    assert create(2, [1, 0, 1]) == qtt.QTT_ERR_INVALID_ARG
    assert create(2, [1, 5000, 1]) == qtt.QTT_ERR_INVALID_ARG
    assert create(2, [1, 2, 1], mask=1 << 9) == qtt.QTT_ERR_INVALID_ARG
    assert h.value is None
    assert lib.qtt_create(None, 2, None, None, 0, None) == qtt.QTT_ERR_INVALID_ARG
    assert b"out" in lib.qtt_last_error()
    # the per-core form: a NULL core pointer is refused before anything is read
    r = np.asarray([1, 2, 1], dtype=np.int32)
    ptrs = (ctypes.c_void_p * 2)(cores.ctypes.data, None)
    assert lib.qtt_create(ctypes.byref(h), 2, r.ctypes.data_as(P), ctypes.cast(ptrs, P), 0,
                          None) == qtt.QTT_ERR_INVALID_ARG
    assert b"NULL core" in lib.qtt_last_error() and h.value is None


def test_apply_rejects_null_operator(lib):
    from paper_1511_06029_gb300 import qtt
    assert lib.qtt_apply(None, None, None, 1, 4, 0, 0, None) == qtt.QTT_ERR_INVALID_ARG
    assert lib.qtt_destroy(None) == qtt.QTT_OK
    assert lib.qtt_op_d(None) == -1
    import ctypes
    n = ctypes.c_int64(-1)
    assert lib.qtt_apply_tt_size(None, None, ctypes.byref(n)) == qtt.QTT_ERR_INVALID_ARG
    assert lib.qtt_apply_tt(None, None, None, None, None) == qtt.QTT_ERR_INVALID_ARG
    assert lib.qtt_batch_run_host(None, None, None, None) == qtt.QTT_ERR_INVALID_ARG
    assert lib.qtt_apply_host(None, None, None, 1, 4, 0, 0, 0, None) == qtt.QTT_ERR_INVALID_ARG


def test_normal_build_is_not_the_checked_build():
    """The normal library reports itself unchecked and refuses the checked
    build's self-test (host-side, no device work)."""
    from paper_1511_06029_gb300 import qtt
    lib = qtt.load_library()
    assert lib.qtt_checked_build() == 0
    assert lib.qtt_check_selftest(None) == qtt.QTT_ERR_UNSUPPORTED
