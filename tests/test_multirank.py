"""The multi-rank host logic of bench.py on CPU ranks (gloo, world size 2): each rank
reverses its own box, so the job's rate is the boxes of all ranks over the slowest
rank's time, and the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # rank r's own timings: rank 1 is the slow one in the step time, rank 0 end to end
        ms, e2e = (100.0, 0.30) if rank == 0 else (140.0, 0.20)
        ms_max, e2e_max = bench.max_over_ranks(ms, e2e, ws, torch.device("cpu"))
        v, ve = bench.whole_job_rates(ws, 1000, ms_max, e2e_max)
        q.put((rank, ms_max, e2e_max, v, ve))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, e2e, v, ve in out:
        assert ms == 140.0 and e2e == 0.30
        assert v == pytest.approx(2 * 1000 / 0.140)
        assert ve == pytest.approx(2 * 1000 / 0.30)


def test_reference_arm_runs_on_rank_0_only():
    """A non-zero rank of the reference arm exits 0 without work or output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "vortex64", "--steps", "1", "--warmup", "1"],
                       env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
