"""World-size-2 gloo test of the multi-rank (replica) host logic of bench.py:
the timing is the slowest rank's, the work is summed, no data-path collective."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r did (r+1) * 1000 pair interactions in (r+1) * 10 ms
    r = bench.replica_rate(local_work=(rank + 1) * 1000.0, local_ms=(rank + 1) * 10.0, dist=dist, device="cpu")
    mx = bench.reduce_over_ranks(rank + 0.5, dist, "max", device="cpu")
    out[rank] = (r["ms"], r["work"], r["rate"], mx)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_rate_two_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, work, rate, mx = res[rank]
        assert ms == 20.0                      # the slowest rank
        assert work == 3000.0                  # summed over ranks
        assert rate == pytest.approx(3000.0 / 0.020)
        assert mx == 1.5


def test_single_process_is_identity():
    import bench
    r = bench.replica_rate(500.0, 5.0, None)
    assert r == {"ms": 5.0, "work": 500.0, "rate": 500.0 / 0.005}
