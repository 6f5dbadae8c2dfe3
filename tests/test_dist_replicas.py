"""The N>1 benchmark path (one replica per rank, no collective on the data
path): the slowest rank's time and the sum of the ranks' bisectors make the
whole-job value. Checked with world_size 2 on CPU over gloo."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = [0.25, 0.40][rank]          # each rank's timed seconds
    bis = [1.0e9, 1.2e9][rank]      # each rank's bisectors updated
    bench.barrier(world)
    t_max = bench.reduce_max(t, world)
    total = bench.reduce_sum(bis, world)
    out[rank] = (t_max, total, total / t_max)
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        t_max, total, value = out[r]
        assert t_max == 0.40
        assert total == 2.2e9
        assert abs(value - 2.2e9 / 0.40) < 1.0
