"""The inversion's local-system product on the GPU (qtt_local_apply) against
the oracle's local_apply (pinned by <X_e, A X> with dense matrices), with
the interfaces Psi, Phi built by the oracle's recursions."""
import numpy as np
import pytest

import oracle
from paper_1511_06029_gb300 import inputs
from conftest import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qtt():
    from paper_1511_06029_gb300 import build, qtt as q
    build.build()
    q.load_library()
    return q


def _x_cores(d, rmax, seed):
    rng = np.random.default_rng(seed)
    ranks = [min(4 ** k, 4 ** (d - k), rmax) for k in range(d + 1)]
    return [rng.standard_normal((ranks[k], 2, 2, ranks[k + 1])) / np.sqrt(2 * ranks[k])
            for k in range(d)]


@pytest.mark.parametrize("d,ra,rx", [(4, 3, 5), (6, 8, 12), (7, 16, 20)])
def test_local_apply_every_core(qtt, d, ra, rx):
    import torch
    G = inputs.synthetic_operator(d, ra, 3 + d).cores
    W = _x_cores(d, rx, 9 + d)
    for k in range(d):
        psi, phi = oracle.local_frames(G, W, k)
        ref = oracle.local_apply(psi, G[k], phi, W[k])
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
        y = qtt.local_apply(dev(psi), dev(G[k]), dev(phi), dev(W[k])).cpu().numpy()
        assert y.shape == ref.shape
        assert rel_l2(y, ref) <= 1e-13, k


def test_local_apply_batched(qtt):
    """Operator ranks 6/8, X ranks 12/10, five vectors W in one call (the
    oracle's four-operand sum runs over every index combination, so the
    ranks stay small)."""
    import torch
    rng = np.random.default_rng(4)
    ra, ra2, rx, rx2, nv = 6, 8, 12, 10, 5
    psi = rng.standard_normal((ra, rx, rx))
    G = rng.standard_normal((ra, 2, 2, ra2))
    phi = rng.standard_normal((ra2, rx2, rx2))
    W = rng.standard_normal((nv, rx, 2, 2, rx2))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    y = qtt.local_apply(dev(psi), dev(G), dev(phi), dev(W)).cpu().numpy()
    for v in range(nv):
        assert rel_l2(y[v], oracle.local_apply(psi, G, phi, W[v])) <= 1e-13


def test_local_apply_rejects_bad_shapes(qtt):
    import torch
    z = lambda *s: torch.zeros(s, dtype=torch.float64, device="cuda")
    with pytest.raises(qtt.QTTError):
        qtt.local_apply(z(2, 3, 3), z(2, 2, 2, 4), z(4, 5, 5), z(3, 2, 2, 6))
