"""The benchmark's N > 1 arithmetic on CPU ranks (gloo, world size 2): the
time per step is the maximum over the ranks and the whole-job seconds per
frame divides it by the number of ranks (replicas train separate frames)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, spf = bench.aggregate_timing(4.0 + rank, world, "cpu")
    dist.barrier()
    q.put((rank, ms, spf))
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
    for rank, ms, spf in out:
        assert ms == 5.0                       # the slower rank's time
        assert abs(spf - 5.0 * 150 / 1e3 / 2) < 1e-12
