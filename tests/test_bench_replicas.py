"""Host logic of bench.py's multi-rank (replica) mode on CPU: two gloo ranks
on 127.0.0.1, no GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

WORLD = 2
ROWS, STEPS = 120_000, 4


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        import bench
        # Rank 1 is the slow one: 10 ms against 25 ms.
        ms, value = bench.replica_value(10.0 + 15.0 * rank, ROWS, STEPS, WORLD, "cpu")
        dist.barrier()
        q.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_replica_value_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in range(WORLD))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    assert all(p.exitcode == 0 for p in procs)
    for rank, ms, value in got:
        assert ms == 25.0, rank
        # Whole-job rate: both replicas' rows over the slowest rank's time.
        assert value == pytest.approx(WORLD * ROWS * STEPS / 0.025)


def test_replica_value_single_rank_needs_no_group():
    import bench
    ms, value = bench.replica_value(8.0, ROWS, STEPS, 1, "cpu")
    assert ms == 8.0 and value == pytest.approx(ROWS * STEPS / 0.008)
