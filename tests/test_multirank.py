"""The N>1 bench path on CPU: world-size-2 gloo ranks aggregate their replicas' work
(sum) over the slowest rank's time (max), as bench.py does over NCCL."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    units, secs = bench.aggregate(1000.0 * (rank + 1), 2.0 + rank, dist, "cpu")
    results[rank] = (units, secs)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        results = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, results)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in procs)
        # both ranks see the job total: 1000 + 2000 units over the slower rank's 3 s
        assert results[0] == results[1] == (3000.0, 3.0)


def test_single_rank_passthrough():
    import bench

    assert bench.aggregate(5.0, 2.0) == (5.0, 2.0)


def test_rank_failure_is_seen_by_the_host():
    # a rank that raises before the collective makes the job fail on the host side
    ctx = mp.get_context("spawn")
    p = ctx.Process(target=_failing_rank)
    p.start()
    p.join(timeout=60)
    assert p.exitcode != 0


def _failing_rank():
    raise SystemExit(3)
