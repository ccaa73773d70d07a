"""Multi-step launches against one launch per step.

The head kernel (steps 0 .. m-1 in registers, ranks <= 8) and the tail
kernel (the last steps, ranks <= 8, writing y; plain loads below 128 low
positions, TMA-staged tiles from there) follow the one-step kernel's
numerics step by step, so their result must be bitwise the unfused one in
every reduced precision and for every input and output type.  The
unfused reference runs in a child process with QTT_NO_FUSION=1 (the switch
is read once per process); one child computes every case.

The cases of the staged tail kernel (2^(d-m) >= 256) run both sides with
QTT_NO_TENSOR_CORES=1: unfused, the tail's steps of rank >= 4 would
otherwise go to the BF16 tensor-core single-step kernel, whose FP32 sums
run in another order (so a rare BF16 rounding differs at a million
outputs), and a fused run would take tensor-core step pairs."""
import itertools
import os
import pickle
import subprocess
import sys

import numpy as np
import pytest

from paper_1511_06029_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TORCH = {"f64": "float64", "f32": "float32", "bf16": "bfloat16"}

CASES = [
    ([1, 2, 4, 8, 6, 1], 3),        # head of 3 steps, tail of 2
    ([1, 3, 5, 7, 2, 1], 2),        # uneven ranks, padded core widths
    ([1, 2, 4, 1], 4),              # head of 2 steps, last step single (d = 3)
    ([1, 8, 8, 8, 8, 8, 1], 1),     # rank 8 everywhere: head of 3, tail of 3
    ([1, 2, 16, 4, 1], 2),          # r_2 > 8: no head (m would be 1)
    ([1, 2, 4, 8, 12, 12, 8, 4, 2, 1], 2),   # head, three single steps, tail of 3
    ([1, 4, 8, 12, 6, 3, 1], 3),    # head of 2, two single steps, tail of 2
]
# 2^(d-m) >= 128 low positions: the staged (TMA) tail kernel; both
# sides without tensor cores
STAGED = [
    ([1, 2, 4, 8, 8, 8, 8, 8, 8, 8, 4, 2, 1], 2),       # d = 12, tail 8-4-2-1
    ([1, 2, 4, 8, 8, 8, 8, 8, 12, 8, 6, 1], 3),         # d = 11, tail of 2
    ([1, 4, 8, 8, 8, 8, 8, 8, 8, 8, 7, 3, 1], 1),       # d = 12, tail 8-7-3-1
    ([1, 2, 4] + [8] * 12 + [8, 4, 2, 1], 16),          # d = 18: the stage ring wraps
]
NPLAIN = len(CASES)
CASES = CASES + STAGED
GRID = list(itertools.product(range(len(CASES)), ["f32", "tf32", "bf16"], ["f64", "f32", "bf16"]))
PLAIN = [i for i, g in enumerate(GRID) if g[0] < NPLAIN]
NO_TC = [i for i, g in enumerate(GRID) if g[0] >= NPLAIN]

CHILD = r"""
import pickle, sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1511_06029_gb300 import inputs, qtt
specs = pickle.load(open(sys.argv[2], "rb"))
outs = []
for sp in specs:
    data = inputs.QTTData(sp["ranks"], sp["cores"])
    op = qtt.Operator(data, packs=(sp["compute"],))
    x = torch.from_numpy(sp["x"]).cuda().to(getattr(torch, sp["io"]))
    outs.append(op.apply(x, compute=sp["compute"]).double().cpu().numpy())
    op.close()
pickle.dump(outs, open(sys.argv[3], "wb"))
"""


def _spec(case, compute, io):
    ranks, nrhs = CASES[case]
    d = len(ranks) - 1
    data = inputs.random_cores(d, ranks, sum(ranks) + nrhs)
    x = inputs.gaussian_rhs(data.N, nrhs, d)
    return {"ranks": ranks, "cores": data.cores, "x": x, "compute": compute, "io": TORCH[io]}


@pytest.fixture(scope="module")
def qtt():
    from paper_1511_06029_gb300 import build, qtt as q
    build.build()
    q.load_library()
    return q


def _run_child(tmp, name, idxs, env_extra):
    spec, out = tmp / (name + "_specs.pkl"), tmp / (name + ".pkl")
    pickle.dump([_spec(*GRID[i]) for i in idxs], open(spec, "wb"))
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(spec), str(out)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    return dict(zip(idxs, pickle.load(open(out, "rb"))))


@pytest.fixture(scope="module")
def unfused(tmp_path_factory):
    d = tmp_path_factory.mktemp("fusion")
    ref = _run_child(d, "unfused", PLAIN, {"QTT_NO_FUSION": "1"})
    ref.update(_run_child(d, "unfused_no_tc", NO_TC,
                          {"QTT_NO_FUSION": "1", "QTT_NO_TENSOR_CORES": "1"}))
    return ref


@pytest.fixture(scope="module")
def fused_no_tc(tmp_path_factory):
    return _run_child(tmp_path_factory.mktemp("fusion_no_tc"), "fused_no_tc", NO_TC,
                      {"QTT_NO_TENSOR_CORES": "1"})


@pytest.mark.parametrize("idx", PLAIN)
def test_head_is_bitwise_the_unfused_sweep(qtt, unfused, idx):
    import torch
    sp = _spec(*GRID[idx])
    data = inputs.QTTData(sp["ranks"], sp["cores"])
    op = qtt.Operator(data, packs=(sp["compute"],))
    x = torch.from_numpy(sp["x"]).cuda().to(getattr(torch, sp["io"]))
    fused = op.apply(x, compute=sp["compute"]).double().cpu().numpy()
    op.close()
    assert np.array_equal(fused.view(np.uint64), unfused[idx].view(np.uint64))


@pytest.mark.parametrize("idx", NO_TC)
def test_staged_tail_is_bitwise_the_unfused_sweep(qtt, unfused, fused_no_tc, idx):
    a, b = fused_no_tc[idx], unfused[idx]
    assert a.shape == b.shape and np.array_equal(a.view(np.uint64), b.view(np.uint64))
