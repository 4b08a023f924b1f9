"""The multi-rank path on CPU (gloo, world size 2): the replicas share no
data, the only collective is the max-over-ranks timing reduction, and only
rank 0 reports; the reference arm's other ranks exit without work."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_setup("gloo")
    # rank r "took" r + 1.5 seconds for its replica of 1000 cells
    t = bench.max_over_ranks(r + 1.5, w, "cpu")
    out.put((r, w, t, bench.whole_job_rate(1000, 30, w, t)))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_with_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, *_ in res] == [0, 1]
    for r, w, t, rate in res:
        assert w == 2 and t == 2.5                      # the slowest rank's time on every rank
        assert rate == pytest.approx(1000 * 30 * 2 / 2.5)   # all ranks' work over that time


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "sod400", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
