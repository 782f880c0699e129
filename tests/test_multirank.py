"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The shifted-COCG columns are independent, so bench.py shards them across ranks with no collective on
the data path: each rank solves its own sample of boundary columns ("weak" scaling), and only the
timing (max over ranks) and the unit count (sum over ranks) are reduced.  This test runs those reductions
and the column sharding in two gloo processes.
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, root, out):
    import sys
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from workloads import small_problem
    p = small_problem(grid=(16, 12, 10), cols=24, seed=5)
    cols = bench.rank_columns(p, rank)
    gathered = [None] * world
    dist.all_gather_object(gathered, [int(c) for c in cols])
    t_max = bench._max_over_ranks(1.0 + rank, world)
    units = bench._sum_over_ranks(float(len(cols)), world)
    out[rank] = (gathered, t_max, units)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_reductions(repo_root):
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, repo_root, out)) for r in range(world)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    g0, tmax0, units0 = out[0]
    g1, tmax1, units1 = out[1]
    assert g0 == g1
    c0, c1 = np.array(g0[0]), np.array(g0[1])
    assert c0.size == c1.size == 24                      # weak scaling: same work per rank
    assert np.unique(c0).size == 24 and np.unique(c1).size == 24
    assert not np.array_equal(c0, c1)                    # ranks solve different columns
    assert tmax0 == tmax1 == 2.0                         # step time = max over ranks
    assert units0 == units1 == 48.0                      # units = sum over ranks
