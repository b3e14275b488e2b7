"""The multi-rank path of bench.py on CPU: ranks run independent replicas
(no data-path collective) and agree, through one all-reduce, on the slowest
rank's time; the whole-job rate counts every rank's steps.  Two gloo ranks."""
import os
import socket
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms_by_rank, queue):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = bench.max_over_ranks(torch, dist, ms_by_rank[rank], world, "cpu")
        rate = bench.whole_job_rate(2.0e9, 10, world, ms)
        queue.put((rank, ms, rate))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    queue = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, [3.0, 5.0], queue)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(queue.get() for _ in range(2))
    want_rate = 2.0e9 * 10 * 2 / (5.0e-3) / 1e9
    assert [g[0] for g in got] == [0, 1]
    for _, ms, rate in got:
        assert ms == 5.0 and abs(rate - want_rate) <= 1e-9 * want_rate


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(torch, None, 7.5, 1, "cpu") == 7.5
    assert bench.whole_job_rate(1.0e9, 4, 1, 2.0) == 1.0e9 * 4 / 2.0e-3 / 1e9
