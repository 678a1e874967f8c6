"""Multi-rank host logic of bench.py on CPU: two gloo ranks (127.0.0.1) combine their timed regions
by taking the maximum and report the whole-job rate of independent shards (weak scaling)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took 10 * (r + 1) ms for the device region and 30 * (r + 1) ms end to end
    slow, rates = bench.combine_ranks([10.0 * (rank + 1), 30.0 * (rank + 1)], units_per_rank=1000.0, steps=5)
    q.put((rank, slow, rates))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, slow, rates in out:
        assert slow == [20.0, 60.0]
        # 2 ranks x 1000 units x 5 steps over the slowest rank's time
        assert rates[0] == pytest.approx(2 * 1000 * 5 / 0.020)
        assert rates[1] == pytest.approx(2 * 1000 * 5 / 0.060)


def test_single_process_is_unchanged():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    slow, rates = bench.combine_ranks([4.0], units_per_rank=10.0, steps=2)
    assert slow == [4.0] and rates[0] == pytest.approx(10.0 * 2 / 0.004)
