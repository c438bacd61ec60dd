"""Multi-rank paths on the CPU (two gloo ranks): the benchmark's frame
sharding (weak scaling, no data-path collective) partitions the frames exactly
once and agrees on the max-over-ranks timing; a fit whose beams are split over
ranks combines the per-rank fused-MSE adjoints with one all-reduce."""
import os
import socket

import pytest
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


def _mse_worker(rank, world, port, parts, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2208_10295_gb300.torch_api import allreduce_mse
    L, gT, gg, N = parts[rank]
    loss = torch.tensor([L], dtype=torch.float64)
    grad_table = torch.tensor(gT, dtype=torch.float64)
    grad_gain = torch.tensor([gg], dtype=torch.float64)
    total = allreduce_mse(loss, grad_table, grad_gain, torch.tensor([N], dtype=torch.int64))
    q.put((rank, float(loss.item()), grad_table.numpy(), float(grad_gain.item()), float(total.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_mse_adjoint_allreduce(oracle_lib):
    """A batch's beams split over two gloo ranks: each rank's fused-MSE adjoint
    over its own beams (the oracle's, FP64), combined by one all-reduce of the
    count-weighted vector, equals the adjoint of the whole batch."""
    import numpy as np
    import synth
    w = synth.small_terrain(n_cells=24, half=12.0, n_objects=8, n_frames=2, n_az=96)
    T = oracle_lib.build_tables(w.params)
    fwd = oracle_lib.cast(w.scene, w.sensors, w.frames, T, w.seed)
    tgt = oracle_lib.cast(w.scene, w.sensors, w.frames, oracle_lib.build_tables(w.hidden_params), w.seed)
    g = 1.25
    args = lambda s: (fwd.valid[s], fwd.mat[s], fwd.theta_deg[s], fwd.rf[s], T, g, tgt.intensity[s], tgt.valid[s])
    n = fwd.valid.shape[0]
    cut = n // 3   # unequal shares
    parts = [oracle_lib.cast_backward(*args(slice(0, cut))), oracle_lib.cast_backward(*args(slice(cut, n)))]
    parts = [(float(L), np.asarray(gT, np.float64), float(gg), int(N)) for L, gT, gg, N in parts]
    L_all, gT_all, gg_all, N_all = oracle_lib.cast_backward(*args(slice(0, n)))
    assert parts[0][3] > 100 and parts[1][3] > 100 and parts[0][3] + parts[1][3] == N_all
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_mse_worker, args=(r, world, port, parts, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, L, gT, gg, total in got:
        assert total == N_all
        assert L == pytest.approx(L_all, rel=1e-12)
        assert np.allclose(gT, gT_all, rtol=1e-12, atol=1e-15 * np.abs(gT_all).max())
        assert gg == pytest.approx(gg_all, rel=1e-12)
