"""qtt_solve (DIRECT, GMRES, REFINE) on the GPU against the oracle's solves.

With ||K||_2 = 0.5 the condition number of I + K is at most 3, so a GPU
residual tolerance of 3e-11 bounds the solution error by 1e-10 relative; the
oracle solves to 1e-13.  Solutions are compared, not iterates (different
orthogonalisations give different iterates)."""
import numpy as np
import pytest

import oracle
from paper_1511_06029_gb300 import inputs
from conftest import rel_l2, neumann, neumann_unrounded

pytestmark = pytest.mark.gpu

GPU_TOL = 3e-11
SOL_TOL = 1e-10


@pytest.fixture(scope="module")
def qtt():
    from paper_1511_06029_gb300 import build, qtt as q
    build.build()
    q.load_library()
    return q


def _problem(d):
    K = inputs.scaled_operator(d, 8, 7000 + d)
    P = neumann(oracle, K, 1e-4)
    return K, P


def _gpu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("d,nrhs", [(8, 1), (10, 3), (12, 2)])
def test_gmres_fp64_with_p(qtt, d, nrhs):
    K, P = _problem(d)
    f = inputs.gaussian_rhs(K.N, nrhs, 11)
    xo, ito, _ = oracle.solve_gmres(K, P, f, a=1.0, tol=1e-13, restart=30)
    Kg, Pg = qtt.Operator(K), qtt.Operator(P)
    x, info = qtt.solve(Kg, Pg, _gpu(f), kind="gmres", tol=GPU_TOL, restart=30)
    x = x.cpu().numpy()
    assert rel_l2(x, xo) <= SOL_TOL
    for (it, rel, st), f_c, x_c in zip(info, f, x):
        assert st == qtt.QTT_OK and rel <= GPU_TOL
        # true residual checked independently with the oracle's apply
        r = f_c - (x_c + oracle.apply(K, x_c))
        assert np.linalg.norm(r) <= 1.01 * GPU_TOL * np.linalg.norm(f_c)
    Kg.close(), Pg.close()


def test_gmres_unpreconditioned(qtt):
    K, _ = _problem(9)
    f = inputs.gaussian_rhs(K.N, 2, 12)
    xo, _, _ = oracle.solve_gmres(K, None, f, a=1.0, tol=1e-13, restart=30)
    Kg = qtt.Operator(K)
    x, info = qtt.solve(Kg, None, _gpu(f), kind="gmres", tol=GPU_TOL, restart=10, max_iter=500)
    assert rel_l2(x.cpu().numpy(), xo) <= SOL_TOL
    Kg.close()


@pytest.mark.parametrize("pc", ["bf16", "tf32", "f32"])
def test_gmres_low_precision_preconditioner(qtt, pc):
    """P applied in BF16/TF32/FP32; the FP64 residual and Arnoldi keep the
    solution at 1e-10."""
    K, P = _problem(11)
    f = inputs.gaussian_rhs(K.N, 2, 13)
    xo, _, _ = oracle.solve_gmres(K, P, f, a=1.0, tol=1e-13, restart=30)
    Kg, Pg = qtt.Operator(K), qtt.Operator(P, packs=(pc,))
    x, info = qtt.solve(Kg, Pg, _gpu(f), kind="gmres", tol=GPU_TOL, restart=30,
                        precond_compute=pc)
    assert rel_l2(x.cpu().numpy(), xo) <= SOL_TOL
    assert all(st == qtt.QTT_OK for _, _, st in info)
    Kg.close(), Pg.close()


@pytest.mark.parametrize("pc", ["f64", "bf16"])
def test_refine(qtt, pc):
    K, P = _problem(10)
    f = inputs.gaussian_rhs(K.N, 2, 14)
    xo, _, _ = oracle.solve_refine(K, P, f, a=1.0, tol=1e-13)
    Kg = qtt.Operator(K)
    Pg = qtt.Operator(P, packs=(() if pc == "f64" else (pc,)))
    x, info = qtt.solve(Kg, Pg, _gpu(f), kind="refine", tol=GPU_TOL, max_iter=200,
                        precond_compute=pc)
    assert rel_l2(x.cpu().numpy(), xo) <= SOL_TOL
    assert all(st == qtt.QTT_OK for _, _, st in info)
    Kg.close(), Pg.close()


def test_refine_contraction_pin(qtt):
    """Unrounded P = I - K + K^2 in FP64: the error operator is -K^3, so the
    number of refinement steps to 1e-12 is at most ceil(12 / -log10 0.125)
    plus the initial apply and one step of slack."""
    K = inputs.scaled_operator(8, 8, 7008)
    P = neumann_unrounded(oracle, K)
    f = inputs.gaussian_rhs(K.N, 1, 15)
    Kg, Pg = qtt.Operator(K), qtt.Operator(P)
    x, info = qtt.solve(Kg, Pg, _gpu(f), kind="refine", tol=1e-12, max_iter=100)
    assert info[0][0] <= int(np.ceil(12 / -np.log10(0.125))) + 2
    Kg.close(), Pg.close()


def test_direct(qtt):
    K, P = _problem(9)
    f = inputs.gaussian_rhs(K.N, 2, 16)
    Kg, Pg = qtt.Operator(K), qtt.Operator(P)
    x, info = qtt.solve(Kg, Pg, _gpu(f), kind="direct")
    xo = oracle.solve_direct(P, f)
    assert rel_l2(x.cpu().numpy(), xo) <= 1e-12
    for (it, rel, st), f_c, x_c in zip(info, f, xo):
        r = f_c - (x_c + oracle.apply(K, x_c))
        assert abs(rel - np.linalg.norm(r) / np.linalg.norm(f_c)) <= 1e-9 * rel
    Kg.close(), Pg.close()


def test_not_converged_is_reported(qtt):
    K, P = _problem(8)
    f = inputs.gaussian_rhs(K.N, 1, 17)
    Kg = qtt.Operator(K)
    with pytest.raises(qtt.QTTError) as e:
        qtt.solve(Kg, None, _gpu(f), kind="refine", tol=1e-14, max_iter=1)
    assert e.value.status == qtt.QTT_ERR_NOT_CONVERGED
    x, info = qtt.solve(Kg, None, _gpu(f), kind="gmres", tol=1e-14, max_iter=2,
                        raise_on_fail=False)
    assert info[0][2] == qtt.QTT_ERR_NOT_CONVERGED and info[0][0] == 2
    Kg.close()


def test_zero_rhs_and_leading_dimension(qtt):
    import torch
    K, P = _problem(9)
    N = K.N
    f = np.zeros((3, N + 40))
    f[1, :N] = inputs.gaussian_rhs(N, 1, 18)[0]
    ft = _gpu(f)[:, :N]
    xt = torch.full((3, N + 40), 5.0, dtype=torch.float64, device="cuda")[:, :N]
    Kg, Pg = qtt.Operator(K), qtt.Operator(P)
    for kind in ("gmres", "refine"):
        x, info = qtt.solve(Kg, Pg, ft, kind=kind, tol=GPU_TOL, out=xt)
        xs = x.cpu().numpy()
        assert np.array_equal(xs[0], np.zeros(N)) and np.array_equal(xs[2], np.zeros(N))
        xo, _, _ = oracle.solve_gmres(K, P, f[1, :N], a=1.0, tol=1e-13)
        assert rel_l2(xs[1], xo) <= SOL_TOL
        pad = xt.as_strided((3, N + 40), (N + 40, 1)).cpu().numpy()[:, N:]
        assert np.all(pad == 5.0)
    Kg.close(), Pg.close()


def test_run_to_run_bitwise(qtt):
    """Deterministic reductions: the same solve twice gives identical bits."""
    K, P = _problem(10)
    f = _gpu(inputs.gaussian_rhs(K.N, 3, 19))
    Kg, Pg = qtt.Operator(K), qtt.Operator(P, packs=("bf16",))
    x1, _ = qtt.solve(Kg, Pg, f, kind="gmres", tol=GPU_TOL, precond_compute="bf16")
    x2, _ = qtt.solve(Kg, Pg, f, kind="gmres", tol=GPU_TOL, precond_compute="bf16")
    assert bool((x1 == x2).all())
    Kg.close(), Pg.close()


@pytest.mark.parametrize("pc,inner", [("bf16", 6), ("tf32", 4), ("f64", 3)])
def test_refine_inner_iterations(qtt, pc, inner):
    """Mixed-precision refinement without P: the correction is `inner`
    Richardson steps z <- r - K z with K in low precision; only the residual
    and the update are FP64.  Reaches the 1e-10 solution error."""
    K, _ = _problem(11)
    f = inputs.gaussian_rhs(K.N, 3, 20)
    xo, _, _ = oracle.solve_gmres(K, None, f, a=1.0, tol=1e-13)
    Kg = qtt.Operator(K, packs=(() if pc == "f64" else (pc,)))
    x, info = qtt.solve(Kg, None, _gpu(f), kind="refine", tol=GPU_TOL, max_iter=60,
                        precond_compute=pc, inner_iters=inner)
    assert rel_l2(x.cpu().numpy(), xo) <= SOL_TOL
    assert all(st == qtt.QTT_OK for _, _, st in info)
    Kg.close()


def test_refine_inner_needs_packed_k(qtt):
    K, _ = _problem(8)
    Kg = qtt.Operator(K)
    f = _gpu(inputs.gaussian_rhs(K.N, 1, 21))
    with pytest.raises(qtt.QTTError) as e:
        qtt.solve(Kg, None, f, kind="refine", precond_compute="bf16", inner_iters=2)
    assert e.value.status == qtt.QTT_ERR_INVALID_ARG
    Kg.close()
