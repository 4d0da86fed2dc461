"""The benchmark's multi-rank host logic on CPU ranks (gloo, world size 2; no GPU): rank discovery
from the launcher's environment, the slowest-rank reduction of the timings, the whole-job value,
and the reference arm under torchrun, where rank 0 alone works and prints one line."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench as b
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ws_, rank_, local_ = b.dist_env()
        t = b.max_over_ranks(10.0 + 5.0 * rank_, ws_, torch.device("cpu"))
        q.put((rank_, ws_, local_, t))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_time_reaches_every_rank():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 2, 0, 15.0), (1, 2, 1, 15.0)]


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.25, 1, None) == 3.25


def test_whole_job_value_counts_every_rank():
    # 64 chains x 13 substeps per rank, 5 steps in 2 s: 2080 substeps/s per rank
    assert bench.job_value(64 * 13, 1, 5, 2.0) == pytest.approx(2080.0)
    assert bench.job_value(64 * 13, 4, 5, 2.0) == pytest.approx(4 * 2080.0)


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
