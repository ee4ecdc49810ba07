"""The benchmark's multi-GPU mode runs independent replicas (one ring per
rank, no data-path collective); its host logic -- the max-over-ranks timing
and the per-rank seeds -- checked with two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, lr, w = bench.rank_info()
        t = bench.max_over_ranks(1.0 + 2.0 * rank)  # rank 1 is the slow one
        dist.barrier()
        out.put((rank, r, lr, w, t, bench.replica_seed(4, rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[1:4] for x in res] == [(0, 0, 2), (1, 1, 2)]
    assert res[0][4] == res[1][4] == 3.0
    assert res[0][5] != res[1][5]


def test_replica_rings_differ_and_single_rank_is_identity():
    import bench
    from paper_1907_02289_gb300 import synth
    a = synth.ring(1000, bench.replica_seed(4, 0))
    b = synth.ring(1000, bench.replica_seed(4, 1))
    assert not np.array_equal(a["x"], b["x"])
    assert bench.max_over_ranks(2.5) == 2.5
