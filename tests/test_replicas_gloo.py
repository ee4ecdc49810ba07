"""The benchmark's multi-GPU modes: independent replicas (one ring or patch
set per rank) or one patch set split across the ranks by LPT; no data-path
collective in either.  Their host logic -- the max-over-ranks timing, the
sum of the ranks' work, the per-rank seeds and the patch split -- checked
with two gloo ranks on the CPU."""
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


def _shard_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    from paper_1907_02289_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = synth.patch_sizes(64, 3)
        mine, imb = bench.shard_patches(sizes, rank, world)
        work = float(sum(int(sizes[i]) for i in mine))
        total = bench.sum_over_ranks(work)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        out.put((rank, mine, imb, total, gathered))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_the_patches():
    """Both ranks derive the same LPT split on their own: the two halves are
    disjoint, cover all 64 patches, and the summed work is the whole set."""
    import multiprocessing as mp
    from paper_1907_02289_gb300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, m0, i0, t0, g0), (_, m1, i1, t1, g1) = res
    assert g0 == g1 == [m0, m1]
    assert set(m0).isdisjoint(m1) and sorted(m0 + m1) == list(range(64))
    assert i0 == i1 < 1.05
    assert t0 == t1 == float(sum(int(s) for s in synth.patch_sizes(64, 3)))


def test_shard_with_one_rank_takes_every_patch():
    import bench
    from paper_1907_02289_gb300 import synth
    sizes = synth.patch_sizes(64, 3)
    mine, imb = bench.shard_patches(sizes, 0, 1)
    assert mine == list(range(64)) and imb == 1.0
    assert bench.sum_over_ranks(3.5) == 3.5
    with pytest.raises(SystemExit):
        bench.shard_patches(sizes[:3], 0, 4)
