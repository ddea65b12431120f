"""Multi-rank logic of bench.py on CPU: two gloo ranks, max-over-ranks timing
and the whole-job throughput formula (replicas, weak scaling)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    w, r, _ = bench.dist_setup("gloo")
    assert (w, r) == (world, rank)
    ms_local = [3.0, 5.0][rank]
    ms = bench.max_over_ranks(ms_local, w)
    bench.barrier(w)
    n = 1000
    value = w * n / (ms * 1e-3) / 1e6
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1]
    ms, value = out[0]
    assert ms == 5.0  # the slowest rank sets the step time
    assert value == pytest.approx(2 * 1000 / 5e-3 / 1e6)


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks(4.5, 1) == 4.5
