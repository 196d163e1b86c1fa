"""The multi-process host logic (one process per GPU) on CPU: gloo ranks,
world size 2.  The path shards into independent units, so the only
collectives are the max-over-ranks time and the sum of units after the timed
region; the partition of a batched SVD over ranks is computed by every rank
on its own and must agree, cover every matrix once and stay balanced."""
import ast
import os
import socket

import numpy as np
import pytest

from paper_2202_08361_gb300 import dist as D
from paper_2202_08361_gb300 import workloads


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = D.rank_env()
        assert (w, r, lr) == (world, rank, rank)
        # timing: rank k took 10 + 5k ms for 1000 + k units
        rate, total, ms = D.aggregate_rate(1000 + rank, 10.0 + 5.0 * rank, dist)
        # the batched SVD split, computed independently on each rank
        m, n = workloads.uneven_shapes(count=500)
        parts = D.partition_lpt(D.svd_costs(m, n), world)
        mine = parts[rank]
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        np.save(os.path.join(out_dir, "r%d.npy" % rank),
                np.array([rate, total, ms], dtype=np.float64))
        with open(os.path.join(out_dir, "parts%d.txt" % rank), "w") as f:
            f.write(repr(gathered))
        # each rank draws different 2x2 matrices
        a = workloads.evd_batch(8, False, seed_salt=D.evd_seed_salt(rank))[0]
        allv = [None] * world
        dist.all_gather_object(allv, a.tolist())
        assert allv[0] != allv[1]
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_gloo_world2_reductions_and_partition(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    res = [np.load(tmp_path / ("r%d.npy" % r)) for r in range(world)]
    for r in res:
        total = 1000 + 1001
        assert r[1] == total and r[2] == 15.0
        assert r[0] == pytest.approx(total / 15e-3)
    g0 = (tmp_path / "parts0.txt").read_text()
    g1 = (tmp_path / "parts1.txt").read_text()
    assert g0 == g1  # both ranks computed the same split
    parts = ast.literal_eval(g0)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(500))


def test_partition_lpt_properties():
    m, n = workloads.uneven_shapes(count=10000)
    costs = D.svd_costs(m, n)
    for world in (1, 2, 3, 4, 8):
        parts = D.partition_lpt(costs, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= sum(costs) / world + max(costs)
        assert all(p == sorted(p) for p in parts)
    # by hand: 5 -> r0; 4 -> r1; 3 -> r1 (load 4 < 5); 3 -> r0 (5 < 7);
    # 3 -> r1 (7 < 8)
    assert D.partition_lpt([5, 4, 3, 3, 3], 2) == [[0, 3], [1, 2, 4]]
    assert D.partition_lpt([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        D.partition_lpt([1], 0)


def test_single_process_reductions_are_identity():
    assert D.reduce_max(3.5) == 3.5 and D.reduce_sum(7) == 7
    rate, total, ms = D.aggregate_rate(100, 50.0)
    assert (total, ms) == (100, 50.0) and rate == pytest.approx(2000.0)
    with pytest.raises(ValueError):
        D.aggregate_rate(1, 0.0)
