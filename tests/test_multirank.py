"""Host logic of the multi-GPU path on CPU with two gloo ranks (no GPU): one
set of source positions is partitioned over the ranks, each rank solves its
share (here with the CPU oracle standing in for the library), the results are
gathered to rank 0 on the host and must equal the one-rank solve of the whole
set bit for bit; the benchmark's timing aggregation takes the slowest rank's
time and the sum of the ranks' updates."""
import math
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_1910_11335_b300 import inputs, shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _small_set():
    return inputs.small_cone(6, 5, 4, n_groups=2, sn_order=2, legendre_order=0, n_sources=5)


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # sharded solve of one source set, gathered on the host
    w = _small_set()
    mine = shard.partition(w.batch, world, rank)
    local = {k: oracle.solve(w, k, tol=0.0, max_iters=3).total for k in mine}
    gathered = shard.gather_to_root(local, world, rank)
    # timing aggregation and the benchmark's partition of its ring
    ms, upd = bench.aggregate(100.0 + 50.0 * rank, 1000 * (rank + 1), world)

    class A:
        workload, sources = "batch96", 32

    wb = bench.make_workload(A, rank)
    out[rank] = {"mine": mine, "gathered": gathered, "ms": ms, "upd": upd,
                 "ring": [s.pos for s in wb.sources]}
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_gather_and_aggregate():
    import oracle
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    w = _small_set()
    assert out[0]["mine"] == [0, 2, 4] and out[1]["mine"] == [1, 3]
    assert out[1]["gathered"] is None
    whole = [oracle.solve(w, k, tol=0.0, max_iters=3).total for k in range(w.batch)]
    got = out[0]["gathered"]
    assert len(got) == w.batch
    for k in range(w.batch):
        assert np.array_equal(got[k], whole[k]), k
    for r in range(world):
        assert out[r]["ms"] == 150.0 and out[r]["upd"] == 3000.0
    # the benchmark's ranks take interleaved positions of one 64-position ring
    ang = sorted(math.atan2(p[0], -p[1]) % (2 * math.pi) for r in range(world) for p in out[r]["ring"])
    assert len(ang) == 64
    assert np.allclose(np.diff(ang), 2 * math.pi / 64, atol=1e-12)


def test_partition_covers_every_source_once():
    for n in (0, 1, 5, 32, 33):
        for world in (1, 2, 3, 8):
            seen = sorted(k for r in range(world) for k in shard.partition(n, world, r))
            assert seen == list(range(n))
