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


def test_served_solves_are_bitwise_qtt_solve(qtt, operators):
    """The tick scheduler runs qtt_solve's arithmetic: a GMRES request with a
    BF16 preconditioner and one inner step, and a refinement request, give
    bitwise the x that qtt_solve gives for the same inputs."""
    import torch
    for kind, pc, inner in (("gmres", "bf16", 1), ("refine", "f64", 0)):
        for d in (9, 10):
            K, P, Kg, Pg = operators[d]
            f = inputs.gaussian_rhs(1 << d, 2, 40 + d)
            S = qtt.Server(slots=2, kind=kind, tol=GPU_TOL, precond_compute=pc,
                           inner_iters=inner)
            Kp = qtt.Operator(K, packs=("bf16",)) if inner else Kg
            x, info, _ = S.wait(S.submit(Kp, Pg, f))
            S.close()
            xs, infos = qtt.solve(Kp, Pg, torch.from_numpy(f).cuda(), kind=kind, tol=GPU_TOL,
                                  precond_compute=pc, inner_iters=inner)
            assert np.array_equal(x, xs.cpu().numpy()), (kind, d)
            assert [i[0] for i in info] == [i[0] for i in infos]
            if inner:
                Kp.close()


def test_apply_requests_share_grouped_launches(qtt, operators):
    """Six FP64 apply requests of d = 8, 9, 10 submitted together: each is
    bitwise qtt_apply's, and their 54 core steps ran in far fewer grouped
    launches (one launch per core step index, shared by every request that
    has that step).  Then applies, a BF16 apply and solves in one mix: the
    FP64 applies bitwise, the BF16 apply within the BF16 bound of the
    oracle, the solves converged."""
    import torch
    S = qtt.Server(slots=8, kind="gmres", tol=GPU_TOL, precond_compute="bf16")
    ds = (8, 9, 10, 10, 9, 8)
    xs = [inputs.gaussian_rhs(1 << d, 1 + i % 3, 300 + i) for i, d in enumerate(ds)]
    ids = [S.submit_apply(operators[d][2], x) for d, x in zip(ds, xs)]
    ys = [S.wait(i)[0] for i in ids]
    ticks, grouped = S.ticks()
    S.close()
    for d, x, y in zip(ds, xs, ys):
        assert np.array_equal(y, operators[d][2].apply(torch.from_numpy(x).cuda()).cpu().numpy())
    assert grouped < sum(ds) and ticks <= len(ds)

    S = qtt.Server(slots=8, kind="gmres", tol=GPU_TOL, precond_compute="bf16")
    jobs = []
    for i, d in enumerate(ds):
        jobs.append(("apply", d, xs[i], S.submit_apply(operators[d][2], xs[i])))
    for d in (9, 10):
        f = inputs.gaussian_rhs(1 << d, 2, 400 + d)
        jobs.append(("solve", d, f, S.submit(operators[d][2], operators[d][3], f)))
    xb = inputs.gaussian_rhs(1 << 10, 2, 500)
    Kb = qtt.Operator(operators[10][0], packs=("bf16",))
    jobs.append(("apply_bf16", 10, xb, S.submit_apply(Kb, xb, compute="bf16")))
    out = [(kind, d, x, S.wait(rid)) for kind, d, x, rid in jobs]
    S.close()
    for kind, d, x, (y, info, _) in out:
        K, P, Kg, Pg = operators[d]
        if kind == "apply":
            ref = Kg.apply(torch.from_numpy(x).cuda()).cpu().numpy()
            assert np.array_equal(y, ref)
        elif kind == "apply_bf16":
            assert rel_l2(y, oracle.apply(K, x)) <= 3 * np.sqrt(d) * 2.0 ** -8
        else:
            assert all(s == qtt.QTT_OK and r <= GPU_TOL for _, r, s in info)
            xo, _, _ = oracle.solve_gmres(K, P, x, a=1.0, tol=1e-13, restart=30)
            assert rel_l2(y, xo) <= 1e-10
    Kb.close()
