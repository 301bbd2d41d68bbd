"""The bench's N > 1 aggregation on CPU: two gloo ranks, each with its own units and time; the
job value is all units over the slowest rank's time (weak scaling, one scalar all_reduce)."""
import os

import torch.distributed as dist
import torch.multiprocessing as mp


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    v, s = bench.aggregate(64.0, 1.0 + rank, world, dist)
    q.put((rank, v, s))
    dist.barrier()
    dist.destroy_process_group()


def test_weak_scaling_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, v, s in out:
        assert s == 2.0 and v == 64.0 * 2 / 2.0
