"""The benchmark's multi-rank logic on CPU: two gloo ranks (127.0.0.1), each a
replica with its own time and work; the reported time is the max over ranks
and the work the sum, as the GPU run under torchrun does with NCCL."""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), HSK_BENCH_BACKEND="gloo")
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import bench
    w, r, local, pg = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank) and pg is not None
    dev = torch.device("cpu")
    t = 10.0 + rank * 5.0          # this replica's time
    work = 1000.0 * (rank + 1)     # this replica's windows
    pg.barrier()
    q.put((rank, bench.reduce_max(pg, t, dev), bench.reduce_sum(pg, work, dev)))
    pg.destroy_process_group()


def test_two_gloo_ranks_max_time_sum_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, work in out:
        assert tmax == 15.0 and work == 3000.0, (rank, tmax, work)


def test_single_process_needs_no_group():
    import bench
    w, r, local, pg = bench.dist_setup() if "WORLD_SIZE" not in os.environ else (1, 0, 0, None)
    assert pg is None and w == 1
    assert bench.reduce_max(None, 3.5, None) == 3.5 and bench.reduce_sum(None, 2.0, None) == 2.0
