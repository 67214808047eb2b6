"""The replicated multi-GPU path of bench.py on CPU: two gloo ranks (no GPU).

With --gpus N every rank runs the whole workload (replicas: the dual ascent of
one QAP does not shard without an all-gather of the O(n^5) Z duals, and the
configurations fit one GPU), the timed region ends at the slowest rank, and the
reported value is N x units / slowest time.  Here two processes report
different times and must agree on the max and on the whole-job rate.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        slowest = bench.rank_max(ms, dist, "cpu")
        rate = bench.whole_job_rate(world, 300, slowest)
        out[rank] = (slowest, rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_and_rate():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    slowest, rate = res[0]
    assert slowest == 150.0
    assert rate == pytest.approx(2 * 300 / 0.150)


def test_single_process_is_identity():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.rank_max(12.5, None, "cpu") == 12.5
    assert bench.whole_job_rate(1, 300, 600.0) == pytest.approx(500.0)
