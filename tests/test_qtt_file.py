"""The .qtt operator file: the library's writer and reader (C, host-only) and
the generator's numpy writer and reader agree bit for bit in both
directions, an operator read back applies exactly as the original (oracle),
and malformed files are refused with a status, not a crash."""
import struct

import numpy as np
import pytest

import oracle
from paper_1511_06029_gb300 import inputs


@pytest.fixture(scope="module")
def qtt():
    from paper_1511_06029_gb300 import build, qtt as q
    build.build()
    q.load_library()
    return q


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def _awkward(seed):
    """Random ranks and cores, with -0.0, a subnormal, +-inf and a NaN payload
    planted so that the round trip must keep every bit."""
    data = inputs.random_cores(6, [1, 3, 5, 2, 7, 4, 1], seed)
    c = data.cores[2].reshape(-1)
    c[:5] = [-0.0, 5e-324, np.inf, -np.inf, np.frombuffer(struct.pack("<Q", 0x7FF800000000ABCD),
                                                          dtype=np.float64)[0]]
    return data


def test_library_writer_numpy_reader(qtt, tmp_path):
    data = _awkward(1)
    p = str(tmp_path / "a.qtt")
    qtt.write_file(p, data.ranks, data.cores)
    back = inputs.load_qtt(p)
    assert back.ranks == data.ranks
    for a, b in zip(data.cores, back.cores):
        assert a.shape == b.shape and np.array_equal(_bits(a), _bits(b))


def test_numpy_writer_library_reader(qtt, tmp_path):
    data = _awkward(2)
    p = str(tmp_path / "b.qtt")
    inputs.save_qtt(p, data)
    ranks, cores = qtt.read_file(p)
    assert ranks == data.ranks
    for a, b in zip(data.cores, cores):
        assert a.shape == b.shape and np.array_equal(_bits(a), _bits(b))
    # the two writers produce the same bytes
    q = str(tmp_path / "c.qtt")
    qtt.write_file(q, data.ranks, data.cores)
    assert open(p, "rb").read() == open(q, "rb").read()


def test_operator_from_file_applies_identically(tmp_path):
    data = inputs.synthetic_operator(9, 6, 3)
    p = str(tmp_path / "op.qtt")
    inputs.save_qtt(p, data)
    back = inputs.load_qtt(p)
    x = inputs.gaussian_rhs(data.N, 2, 4)
    assert np.array_equal(oracle.apply(back, x), oracle.apply(data, x))


def _status(qtt, path, ranks_cap=64, cores_cap=1 << 20):
    import ctypes
    lib = qtt.load_library()
    d, n = ctypes.c_int(), ctypes.c_int64()
    rk = (ctypes.c_int * 64)()
    buf = np.zeros(1 << 20)
    return lib.qtt_read_file(path.encode(), ctypes.byref(d), rk, ranks_cap,
                             buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), cores_cap,
                             ctypes.byref(n))


def test_malformed_files_are_refused(qtt, tmp_path):
    data = inputs.random_cores(4, [1, 2, 3, 2, 1], 5)
    good = str(tmp_path / "good.qtt")
    inputs.save_qtt(good, data)
    raw = open(good, "rb").read()
    assert _status(qtt, good) == qtt.QTT_OK

    def variant(name, content):
        p = str(tmp_path / name)
        open(p, "wb").write(content)
        return p

    bad_magic = variant("magic.qtt", b"QTX1" + raw[4:])
    version = variant("version.qtt", raw[:4] + struct.pack("<I", 2) + raw[8:])
    etype = variant("etype.qtt", raw[:12] + struct.pack("<I", 1) + raw[16:])
    truncated = variant("trunc.qtt", raw[:-8])
    longer = variant("long.qtt", raw + b"\0" * 8)
    rank0 = variant("rank0.qtt", raw[:24] + struct.pack("<I", 2) + raw[28:])
    dzero = variant("d0.qtt", raw[:8] + struct.pack("<I", 0) + raw[12:])
    for p in (bad_magic, truncated, longer, rank0, dzero, str(tmp_path / "missing.qtt")):
        assert _status(qtt, p) == qtt.QTT_ERR_INVALID_ARG, p
    for p in (version, etype):
        assert _status(qtt, p) == qtt.QTT_ERR_UNSUPPORTED, p
    # buffers too small
    assert _status(qtt, good, ranks_cap=3) == qtt.QTT_ERR_INVALID_ARG
    assert _status(qtt, good, cores_cap=10) == qtt.QTT_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        inputs.load_qtt(truncated)
    # the writer refuses invalid ranks
    with pytest.raises(qtt.QTTError) as e:
        qtt.write_file(str(tmp_path / "w.qtt"), [2, 3, 1], [np.zeros((2, 2, 2, 3)),
                                                           np.zeros((3, 2, 2, 1))])
    assert e.value.status == qtt.QTT_ERR_INVALID_ARG
