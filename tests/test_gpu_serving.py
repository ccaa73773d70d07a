"""Solve server: continuous admission by slots and device memory, overlap on
the device, and every request's result the same alone and in the mix."""
import time

import numpy as np
import pytest

import oracle
from paper_1511_06029_gb300 import inputs
from conftest import rel_l2, neumann

pytestmark = pytest.mark.gpu

GPU_TOL = 3e-11


@pytest.fixture(scope="module")
def qtt():
    from paper_1511_06029_gb300 import build, qtt as q
    build.build()
    q.load_library()
    return q


@pytest.fixture(scope="module")
def operators(qtt):
    ops = {}
    for d in (8, 9, 10):
        K = inputs.scaled_operator(d, 8, 7000 + d)
        P = neumann(oracle, K, 1e-4)
        ops[d] = (K, P, qtt.Operator(K), qtt.Operator(P, packs=("bf16",)))
    yield ops
    for _, _, Kg, Pg in ops.values():
        Kg.close()
        Pg.close()


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        d = int(rng.integers(8, 11))
        nrhs = int(rng.integers(1, 4))
        out.append((d, inputs.gaussian_rhs(1 << d, nrhs, 900 + i)))
    return out


def test_mix_equals_alone_and_oracle(qtt, operators):
    reqs = _requests(14, 1)
    # alone: one slot, one request at a time
    alone = qtt.Server(slots=1, kind="gmres", tol=GPU_TOL, precond_compute="bf16")
    xs_alone = []
    for d, f in reqs:
        _, _, Kg, Pg = operators[d]
        xs_alone.append(alone.wait(alone.submit(Kg, Pg, f))[0])
    alone.close()
    # mix: four slots, a budget that holds only some requests at a time, all
    # submitted at once so they queue, get admitted as others finish, overlap
    mix = qtt.Server(slots=4, mem_budget=400 << 20, kind="gmres", tol=GPU_TOL,
                     precond_compute="bf16")
    ids = [mix.submit(operators[d][2], operators[d][3], f) for d, f in reqs]
    results = [mix.wait(i) for i in ids]
    st = mix.stats()
    mix.close()
    assert st["peak_running"] >= 2
    for (d, f), xa, (x, info, (ts, ta, tf)) in zip(reqs, xs_alone, results):
        assert np.array_equal(x, xa)  # bitwise: the arithmetic is the request's own
        assert ts <= ta <= tf
        assert all(s == qtt.QTT_OK and r <= GPU_TOL for _, r, s in info)
        K, P = operators[d][0], operators[d][1]
        xo, _, _ = oracle.solve_gmres(K, P, f, a=1.0, tol=1e-13, restart=30)
        assert rel_l2(x, xo) <= 1e-10


def test_admission_by_memory(qtt, operators):
    _, _, Kg, Pg = operators[10]
    f = inputs.gaussian_rhs(1 << 10, 3, 5)
    # a budget below one request's estimate is rejected at submission
    tiny = qtt.Server(slots=2, mem_budget=1 << 20, kind="gmres", tol=GPU_TOL)
    with pytest.raises(qtt.QTTError) as e:
        tiny.submit(Kg, Pg, f)
    assert e.value.status == qtt.QTT_ERR_OOM
    tiny.close()
    # a budget for exactly one request at a time serialises admission
    one = qtt.Server(slots=4, mem_budget=(64 << 20) + (8 << 20), kind="gmres", tol=GPU_TOL,
                     precond_compute="bf16")
    ids = [one.submit(Kg, Pg, f) for _ in range(3)]
    res = [one.wait(i) for i in ids]
    assert one.stats()["peak_running"] == 1
    one.close()
    # admissions happen in order, each after the previous finished
    times = [r[2] for r in res]
    for a, b in zip(times, times[1:]):
        assert b[1] >= a[2]


def test_poll_before_done_and_unknown_id(qtt, operators):
    _, _, Kg, Pg = operators[9]
    S = qtt.Server(slots=1, kind="gmres", tol=GPU_TOL, precond_compute="bf16")
    rid = S.submit(Kg, Pg, inputs.gaussian_rhs(1 << 9, 2, 6))
    t0 = time.time()
    while S.poll(rid) is None:
        assert time.time() - t0 < 60
        time.sleep(0.001)
    with pytest.raises(qtt.QTTError):
        import ctypes
        done = ctypes.c_int()
        qtt._check(qtt.load_library().qtt_server_poll(S._h, rid, 0, ctypes.byref(done), None,
                                                      None, None, None), "poll")
    S.close()
