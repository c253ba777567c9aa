"""The multi-GPU path of bench.py, on the CPU with gloo and world size 2: each
rank renders its own frame (weak scaling; no collective on the data path),
the job time is the slowest rank's and the job's work is the sum of all
ranks' fragments."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import synth
        w, r, _ = bench.dist_env()
        fr = synth.uniform_frame(48, 32, 6.0, 40, seed=bench.rank_seed(7, r))
        t = 1.0 + r                     # rank 1 is the slow one
        tmax = bench.max_over_ranks(t, w)
        work = bench.sum_over_ranks(float(fr.n), w)
        bench.barrier(w)
        q.put((r, fr.n, int(fr.pixel.sum()), tmax, work))
    finally:
        dist.destroy_process_group()


def test_two_rank_weak_scaling_aggregation():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    (r0, n0, h0, t0, w0), (r1, n1, h1, t1, w1) = res
    assert (r0, r1) == (0, 1)
    assert h0 != h1                     # independent frames per rank
    assert t0 == t1 == 2.0              # max over ranks
    assert w0 == w1 == float(n0 + n1)   # whole-job work
