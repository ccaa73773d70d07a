"""The benchmark's contract on the CPU: the reference arm (the FP64 oracle on
the host cores) prints one well-formed JSON line, rank 0 alone prints under
a two-process launch, and the replica aggregation (max over ranks, whole-job
value) over two gloo ranks."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

# a short oracle sample (seconds of CPU work per step)
ENV = dict(os.environ, QTT_REF_STEP_S="0.3", CUDA_VISIBLE_DEVICES="")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _json_lines(text):
    return [json.loads(l) for l in text.splitlines() if l.startswith("{")]


def _check_reference_line(line, n_gpus):
    assert line["impl"] == "reference"
    assert line["metric"] == "QTT-apply GFLOP/s" and line["unit"] == "GFLOP/s"
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["n_gpus"] == n_gpus and line["steps"] == 1 and line["warmup"] == 3
    assert line["higher_is_better"] is True and line["scaling"] == "weak"
    assert line["vs_baseline"] is None and line["data"] == "synthetic"
    assert line["dtype"] == "f64" and line["config"]["workload"] == "apply_f64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert "diagonal block" in cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=ENV, capture_output=True,
                       text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_reference_line(lines[0], 1)


def test_reference_arm_under_two_ranks_prints_on_rank_0_only():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, env=ENV, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_reference_line(lines[0], 2)


def _replica_rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_local = [2.0, 3.0][rank]          # rank 1 is the slower one
    t_max = bench.max_over_ranks(dist, t_local, "cpu")
    value = bench.job_value(10.0, 4, world, t_max)
    out.put((rank, t_max, value))
    dist.destroy_process_group()


def test_replica_aggregation_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    import bench
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest time; value = all ranks' work / that time
    assert got == [(0, 3.0, 10.0 * 4 * 2 / 3.0), (1, 3.0, 10.0 * 4 * 2 / 3.0)]
    assert bench.max_over_ranks(None, 1.5, "cpu") == 1.5
    assert bench.job_value(10.0, 4, 1, 2.0) == 20.0


class _Apply:
    def __init__(self, data, nrhs, compute="bf16"):
        self.data, self.nrhs, self.compute = data, nrhs, compute


def test_bf16_byte_model_matches_the_launch_lists():
    """The BF16 roofline's byte model (bench.ApplyRun.fused_bytes) mirrors the
    library's dispatch: its launch groups are those of the ncu launch lists
    of the BF16 applies (d = 21, r <= 48, 64 RHS: 10 launches; d = 24,
    r <= 32, 1 RHS: 12 launches), and at d = 21 its bytes agree with the
    summed DRAM counters (163.31 GB measured; the 268 MB planes do not fit
    in L2) to 1 %."""
    import bench
    from paper_1511_06029_gb300 import inputs
    run = _Apply(inputs.synthetic_operator(21, 48, 3), 64)
    fb, plan = bench.ApplyRun.fused_bytes(run)
    assert plan == [(0, 1, 2), (3,), (4, 5), (6, 7), (8, 9), (10, 11), (12, 13), (14, 15),
                    (16, 17), (18, 19, 20)]
    assert abs(fb - 163.31e9) <= 0.01 * 163.31e9
    run = _Apply(inputs.synthetic_operator(24, 32, 2), 1)
    _, plan = bench.ApplyRun.fused_bytes(run)
    assert plan == [(0, 1, 2), (3,), (4, 5), (6, 7), (8, 9), (10, 11), (12, 13), (14, 15),
                    (16, 17), (18, 19), (20,), (21, 22, 23)]


def test_tf32_byte_model_matches_the_launch_list():
    """The TF32 tensor-core pairing in the byte model mirrors the library's
    dispatch: the d = 24, r <= 32 TF32 apply is the head kernel, nine
    tcgen05 pairs from bit 3 and the tail kernel (11 launches in its ncu
    launch list), 4-byte elements."""
    import bench
    from paper_1511_06029_gb300 import inputs
    data = inputs.synthetic_operator(24, 32, 2)
    fb, plan = bench.ApplyRun.fused_bytes(_Apply(data, 1, "tf32"))
    assert plan == [(0, 1, 2), (3, 4), (5, 6), (7, 8), (9, 10), (11, 12), (13, 14), (15, 16),
                    (17, 18), (19, 20), (21, 22, 23)]
    r = data.ranks
    groups = [(0, 3), (3, 5), (5, 7), (7, 9), (9, 11), (11, 13), (13, 15), (15, 17), (17, 19),
              (19, 21), (21, 24)]
    assert fb == sum(r[a] + r[b] for a, b in groups) * data.N * 4
