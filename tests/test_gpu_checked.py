"""The checked build (libqtt_checked.so, -DQTT_CHECKED): the hot-path kernels
check the indices they derive (right-hand side, position pair, rank block,
TMA box coordinates, batch work item) and clamp and record an out-of-range
one instead of touching memory out of bounds.

Run in a child process that loads the checked library: the FP64 steps (both
forms), the FP32 staged step, the head and tail kernels, the BF16 and TF32
tensor-core pairs and a batch all run clean (no site recorded) and match the
oracle; the self-test kernel, which derives one index out of its range on
purpose, makes the next qtt_sync_status return QTT_ERR_CHECK, and the one
after that is clean again."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import math, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
from paper_1511_06029_gb300 import build, inputs, qtt
import oracle
from conftest import rel_l2
lib = qtt.load_library(build.LIB_CHECKED)
assert lib.qtt_checked_build() == 1
U = {"f64": 1e-12, "f32": 4 * 2.0 ** -24, "tf32": 4 * 2.0 ** -11, "bf16": 4 * 2.0 ** -8}
cases = [(12, 16, 3, "f64"), (9, 8, 2, "f64"), (12, 16, 2, "f32"), (13, 32, 2, "tf32"),
         (12, 16, 2, "bf16")]
for d, r, nrhs, comp in cases:
    data = inputs.synthetic_operator(d, r, d + r)
    x = inputs.gaussian_rhs(data.N, nrhs, d)
    op = qtt.Operator(data, packs=(() if comp == "f64" else (comp,)))
    dt = {"f64": torch.float64, "f32": torch.float32, "tf32": torch.float32,
          "bf16": torch.bfloat16}[comp]
    xd = torch.from_numpy(x).cuda().to(dt)
    y = op.apply(xd, compute=comp).double().cpu().numpy()
    assert lib.qtt_sync_status(None) == qtt.QTT_OK, (d, r, comp, qtt.load_library().qtt_last_error())
    ref = oracle.apply(data, xd.double().cpu().numpy())
    bound = U[comp] * (1 if comp == "f64" else math.sqrt(d))
    assert rel_l2(y, ref) <= bound, (d, r, comp, rel_l2(y, ref))
    op.close()
# a batch (FP32 waves)
items = inputs.batched_workload(count=6, seed=3, d_range=(6, 10), r_range=(4, 24),
                                rhs_range=(1, 3))
datas, ops, xs, ys = [], [], [], []
for it in items:
    data = inputs.synthetic_operator(it["d"], it["rmax"], it["op_seed"])
    datas.append(data)
    ops.append(qtt.Operator(data, packs=("f32",)))
    xs.append(torch.from_numpy(inputs.gaussian_rhs(data.N, it["nrhs"], it["rhs_seed"])
                               .astype(np.float32)).cuda())
    ys.append(torch.empty_like(xs[-1]))
B = qtt.Batch(ops, xs, ys, compute="f32")
B.run()
B.status()
assert lib.qtt_sync_status(None) == qtt.QTT_OK
for data, x, y in zip(datas, xs, ys):
    ref = oracle.apply(data, x.double().cpu().numpy())
    assert rel_l2(y.double().cpu().numpy(), ref) <= 4 * math.sqrt(data.d) * 2.0 ** -24
B.close()
for o in ops:
    o.close()
# the self-test: one index out of range on purpose, reported once
assert lib.qtt_check_selftest(None) == qtt.QTT_OK
assert lib.qtt_sync_status(None) == qtt.QTT_ERR_CHECK
assert b"site 501" in lib.qtt_last_error()
assert lib.qtt_sync_status(None) == qtt.QTT_OK
print("checked ok")
"""


def test_checked_build_runs_clean_and_reports():
    from paper_1511_06029_gb300 import build
    build.build(checked=True)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and "checked ok" in r.stdout, (r.stdout[-2000:], r.stderr[-3000:])
