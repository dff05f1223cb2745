"""The multi-GPU path of the benchmark is replicas only (every rank an
independent instance, no collective on the data path): its host logic --
per-rank seeds, max-over-ranks timing, whole-job rate, the reference arm on
rank 0 only -- on two gloo ranks on the CPU."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        tot = bench.max_over_ranks([1.0 + rank, 10.0 - rank], "cpu")
        dist.barrier()
        out[rank] = (tot, bench.replica_seed(rank), bench.whole_job_rate(world, 5, tot[0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_count_every_solve():
    mp = torch.multiprocessing.get_context("spawn")
    with mp.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [mp.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == [2.0, 10.0]          # slowest rank of each total
    assert res[0][1] != res[1][1]                          # independent instances
    assert res[0][2] == res[1][2] == 2 * 5 / 2.0           # all ranks' solves over the max time


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.5, 1.0], "cpu") == [3.5, 1.0]
    assert bench.whole_job_rate(1, 10, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"], env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
