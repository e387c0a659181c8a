"""The multi-rank path on CPU: two gloo ranks shard the thetas, each applies the oracle for its
own thetas, and the gathered results equal a single-process run (no data-path collective)."""
import os
import socket

import numpy as np
import pytest

from paper_2511_03109_gb300 import inputs, sharding


def test_shard_partitions_items():
    items = list(range(23))
    for world in (1, 2, 3, 8):
        parts = [sharding.shard(items, r, world) for r in range(world)]
        flat = sorted(x for p in parts for x in p)
        assert flat == items
        for r, p in enumerate(parts):
            assert all(sharding.owner(x, world) == r for x in p)
    with pytest.raises(ValueError):
        sharding.shard(items, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    from oracle import pmatrix

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    P = inputs.uniform_points(300, 2, 5)
    X = inputs.gaussian_rhs(300, 2, 6)
    thetas = inputs.uniform_thetas([0.1], [1.0], 5, 7)
    M = pmatrix.ParametricMatrix(P, "gauss", [0.1], [1.0], [8], 5, 2, 1.0, 1e-8)
    M.offline()
    mine = sharding.shard(list(range(len(thetas))), rank, world)
    res = {i: M.matvec(M.instantiate(thetas[i]), X) for i in mine}
    gathered = [None] * world
    dist.all_gather_object(gathered, res)
    t = sharding.max_over_ranks(float(rank + 1), dist)
    if rank == 0:
        allres = {}
        for g in gathered:
            allres.update(g)
        out.put((allres, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_match_single_process():
    import torch.multiprocessing as mp

    from oracle import pmatrix

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    allres, tmax = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert tmax == 2.0
    P = inputs.uniform_points(300, 2, 5)
    X = inputs.gaussian_rhs(300, 2, 6)
    thetas = inputs.uniform_thetas([0.1], [1.0], 5, 7)
    M = pmatrix.ParametricMatrix(P, "gauss", [0.1], [1.0], [8], 5, 2, 1.0, 1e-8)
    M.offline()
    assert sorted(allres) == list(range(5))
    for i, th in enumerate(thetas):
        np.testing.assert_allclose(allres[i], M.matvec(M.instantiate(th), X), rtol=0, atol=0)
