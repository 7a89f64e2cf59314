"""Multi-GPU is replicas only: each rank runs its own copy of the workload and the
bench takes the slowest rank's time and the sum of the ranks' work.  The host
side of that reduction runs here on two gloo ranks (CPU, 127.0.0.1)."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.reduce_over_ranks(100.0 + 50.0 * rank, 1000 * (rank + 1), dist)
    out[rank] = (t, u)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_reduction_two_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == (150.0, 3000.0) and out[1] == (150.0, 3000.0)


def test_single_rank_passthrough():
    import bench
    assert bench.reduce_over_ranks(12.5, 7) == (12.5, 7.0)
