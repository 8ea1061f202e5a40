"""The N > 1 path of bench.py on CPU: world-size-2 gloo process groups.

The method does not shard (one solve runs on one GPU), so `bench.py --gpus N`
runs N independent replicas: each rank solves its own copy of the workload,
the job's time is the slowest rank's (an all-reduce MAX of the per-rank times,
the only collective), and the rate counts every replica's stages. The
reference arm runs on rank 0 alone."""
import argparse
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # per-rank elapsed times: the slowest rank sets each entry
        got = bench.max_over_ranks([1.0 + rank, 5.0 - rank, 0.25 * (rank + 1)], world, "cpu")
        dist.barrier()
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [2.0, 5.0, 0.5]


def test_max_over_ranks_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([3.5, 1.25], 1, "cpu") == [3.5, 1.25]


def test_whole_job_rate_counts_every_replica():
    import bench
    # 2 replicas x 10 steps x 4096 stages in 0.05 s
    assert bench.whole_job_rate(4096, 10, 2, 0.05) == pytest.approx(2 * 10 * 4096 / 0.05)
    assert bench.whole_job_rate(4096, 10, 1, 0.05) == pytest.approx(10 * 4096 / 0.05)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench
    args = argparse.Namespace(steps=1, warmup=3, gpus=2)
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""
