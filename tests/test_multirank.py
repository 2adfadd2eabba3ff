"""Host logic of the multi-GPU (weak scaling) benchmark path on CPU with two
gloo ranks: every rank solves its own batch of source positions, the job's
time is the slowest rank's and its updates the sum over ranks."""
import math
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    from paper_1910_11335_b300 import inputs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, upd = bench.aggregate(100.0 + 50.0 * rank, 1000 * (rank + 1), world)

    class A:
        workload, sources = "batch96", 32

    w = bench.make_workload(A, rank)
    out[rank] = (ms, upd, w.sources[0].pos, w.sources[1].pos)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_rotate_sources():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    for r in range(world):
        ms, upd, p0, p1 = out[r]
        assert ms == 150.0 and upd == 3000.0
    # rank 1's ring is rotated by half a source spacing (2 pi / (32 * 2))
    a0 = math.atan2(out[0][2][0], -out[0][2][1])
    a1 = math.atan2(out[1][2][0], -out[1][2][1])
    assert abs((a1 - a0) - 2 * math.pi / 64) < 1e-12
    assert out[0][3] != out[1][3]
