import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def rel_l2(a, b):
    import numpy as np
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


# ------------------------------------------- operators built by the oracle
# The seeded generator only provides data; operators that need the method's
# compression tools are built here with the oracle (test infrastructure).
def laplace_qtt(oracle, n: int = 8, eps: float = 1e-8):
    """The n^3 Laplace volume operator (Sec. 5.2) compressed by the oracle's
    Algorithm 1 at eps.  Returns (QTTData, dense A)."""
    from paper_1511_06029_gb300 import inputs
    A = inputs.laplace_volume_dense(n)
    T = oracle.tt_svd(A, eps)
    return inputs.QTTData(list(T.ranks), list(T.cores), {"kind": "laplace", "n": n,
                                                          "eps": eps}), A


def neumann_unrounded(oracle, K):
    """I - K + K^2 as an exact QTT (ranks 1 + r + r^2) from the oracle's sum
    and product."""
    from paper_1511_06029_gb300 import inputs
    S = oracle.tt_sum(oracle.tt_sum(inputs.identity(K.d), K.scaled(-1.0)),
                      oracle.tt_product(K, K))
    return inputs.QTTData(list(S.ranks), list(S.cores), {"kind": "neumann_unrounded"})


def neumann(oracle, K, eps: float = 1e-4):
    """P = round(I - K + K^2, eps) by the oracle's TT rounding."""
    from paper_1511_06029_gb300 import inputs
    P = oracle.tt_round(neumann_unrounded(oracle, K), eps)
    return inputs.QTTData(list(P.ranks), list(P.cores), {"kind": "neumann", "eps": eps})
