"""Angular decomposition across ranks on CPU: gloo ranks (127.0.0.1) each hold a (theta, phi) block of
every shell, redistribute to whole-shell radial slabs, filter their slab and scatter back. The
gathered result must equal the filter of the whole state (the oracle, shell by shell)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _grid(Nr, Nth, Nph):
    from paper_2305_01537_gb300 import workloads as w
    p, k, L = w.field_mix_8()
    return w.Grid(Nr, Nth, Nph, p, k, L)


def _rank(rank, world, port, q, shape, Pth, Pph, mode):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2305_01537_gb300 import workloads as w
        from paper_2305_01537_gb300.angular import AngularFilter
        Nr, Nth, Nph = shape
        g = _grid(Nr, Nth, Nph)
        x = w.random_state(g.shape, seed=31)

        if mode == "oracle":
            import oracle

            def filter_slab(i0, i1, xs):
                y = oracle.filter(xs.numpy(), g.parity, g.kind, g.L, g.r[i0:i1], g.dr_min, g.floor)
                return torch.from_numpy(y)
        elif mode == "identity":
            def filter_slab(i0, i1, xs):
                return xs.clone()
        else:  # radius tag: adds the global radius index, so a misplaced slab shows
            def filter_slab(i0, i1, xs):
                tag = torch.arange(i0, i1, dtype=xs.dtype).view(1, -1, 1, 1)
                return xs + 1000.0 * tag

        af = AngularFilter(Nr, Nth, Nph, g.nvars, Pth, Pph, filter_slab)
        (j0, j1), (k0, k1) = af.block(rank)
        y = af.apply(torch.from_numpy(np.ascontiguousarray(x[:, :, j0:j1, k0:k1])))
        q.put((rank, (j0, j1, k0, k1), y.numpy()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _run(shape, Pth, Pph, mode):
    world = Pth * Pph
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q, shape, Pth, Pph, mode)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    g = _grid(*shape)
    full = np.empty(g.shape)
    seen = np.zeros(shape[1:], dtype=int)
    for _, (j0, j1, k0, k1), y in out:
        full[:, :, j0:j1, k0:k1] = y
        seen[j0:j1, k0:k1] += 1
    assert (seen == 1).all()  # the blocks tile every shell exactly once
    return g, full


@pytest.mark.parametrize("Pth,Pph", [(2, 1), (1, 2), (2, 2), (3, 1)])
def test_matches_whole_state_filter(Pth, Pph):
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2305_01537_gb300 import workloads as w
    shape = (7, 10, 12)  # radii, rows and columns that do not divide evenly
    g, got = _run(shape, Pth, Pph, "oracle")
    x = w.random_state(g.shape, seed=31)
    ref = oracle.filter(x, g.parity, g.kind, g.L, g.r, g.dr_min, g.floor)
    # each shell is filtered on its own, so the slab and the whole state give the same bits
    assert np.array_equal(got, ref)


def test_exchange_is_exact_and_keeps_radii():
    import sys
    sys.path.insert(0, ROOT)
    from paper_2305_01537_gb300 import workloads as w
    shape = (5, 6, 8)
    g, got = _run(shape, 2, 2, "identity")
    x = w.random_state(g.shape, seed=31)
    assert np.array_equal(got, x)
    g, got = _run(shape, 2, 2, "tag")
    tag = 1000.0 * np.arange(shape[0]).reshape(1, -1, 1, 1)
    assert np.array_equal(got, x + tag)


def test_rejects_bad_group_and_shape():
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2305_01537_gb300.angular import AngularFilter, split_range
    assert [split_range(10, 3, i) for i in range(3)] == [(0, 4), (4, 7), (7, 10)]
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(_free_port())
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        with pytest.raises(ValueError):
            AngularFilter(4, 6, 8, 1, 2, 1, lambda a, b, x: x)  # 2 blocks in a group of 1
        af = AngularFilter(4, 6, 8, 1, 1, 1, lambda a, b, x: x)
        with pytest.raises(ValueError):
            af.apply(torch.zeros(1, 4, 6, 7, dtype=torch.float64))
        x = torch.randn(1, 4, 6, 8, dtype=torch.float64)
        assert torch.equal(af.apply(x), x)
    finally:
        dist.destroy_process_group()
