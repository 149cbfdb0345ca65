"""The N > 1 host logic of bench.py on CPU: two gloo ranks, no GPU.

Each rank draws its own batch (weak scaling, no data-path collective); the
step time reported is the maximum over ranks.
"""
import os
import socket

import pytest
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
    import bench
    r, w, lr = bench.dist_env()
    seed = bench.shard_seed(20251010, r)
    m = bench.reduce_max(1.5 + r * 2.0)
    bench.barrier()
    q.put((r, w, lr, seed, m))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, s0, m0), (r1, w1, l1, s1, m1) = out
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert s0 == 20251010 and s1 != s0          # rank 0 keeps the published seed
    assert m0 == m1 == 3.5                      # max over ranks, seen by both


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max(2.25) == 2.25
    assert bench.shard_seed(7, 0) == 7
