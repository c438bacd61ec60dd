"""Multi-rank frame sharding of the benchmark (weak scaling, no data-path
collective): two gloo ranks on the CPU partition the frames exactly once and
agree on the max-over-ranks timing."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = bench.shard_frames(8 * world, rank, world)
    got = [None] * world
    dist.all_gather_object(got, mine)
    t = torch.tensor([1.0 + rank])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put((got, float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = sorted(i for part in got for i in part)
    assert flat == list(range(8 * world))          # every frame exactly once
    assert len({len(p) for p in got}) == 1          # same work per rank
    assert tmax == 2.0


def test_shard_frames_single_rank():
    assert bench.shard_frames(5, 0, 1) == [0, 1, 2, 3, 4]
