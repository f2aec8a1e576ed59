"""The multi-rank host logic of bench.py on CPU: world size 2 over gloo.

A solve is not sharded (replicas only); what N > 1 adds is the timing
aggregation (maximum over ranks, whole-job throughput), the per-rank replica
seeds and rank 0 alone printing.  These run here without a GPU."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    sys.path.insert(0, ROOT)
    import bench
    # rank 1 is the slower one: 3.0 s against 2.0 s for 10 steps of 1,000 bodies
    value, slowest = bench.job_throughput(2.0 + rank, 1000, 10, ws)
    q.put((rank, value, slowest, bench.replica_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_throughput_takes_the_slowest_rank_and_counts_every_replica():
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
    for rank, value, slowest, seed in res:
        assert slowest == 3.0
        assert value == pytest.approx(2 * 1000 * 10 / 3.0)
    assert [r[3] for r in res] == [0, 1]  # distinct replicas


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(2.0, 1000, 10, 1) == (5000.0, 2.0)


def test_reference_arm_prints_only_on_rank_zero():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert "{" not in r.stdout
