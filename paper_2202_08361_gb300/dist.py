"""Host-side logic for running the path with one process per GPU.

The batched 2x2 EVDs and the matrices of a batched SVD are independent
problems, so ranks exchange no data on the compute path: each rank takes its
own units, and the only communication is after the timed region, where the
step time becomes the maximum over ranks and the unit count the sum.  The
helpers work with any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
import os


def rank_env():
    """(world_size, rank, local_rank) from the torchrun environment; a plain
    `python` launch is a world of one."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def evd_seed_salt(rank):
    """Each rank draws its own batch of 2x2 matrices (weak scaling: the same
    number per rank, different matrices)."""
    return int(rank)


def partition_lpt(costs, world):
    """Split units with the given costs over `world` ranks, largest first to
    the least-loaded rank (ties: lower index first, lower rank first).

    Returns one ascending index list per rank.  The result depends only on
    `costs` and `world`, so every rank computes the same split on its own.
    The largest load is at most (sum of costs) / world + max cost."""
    world = int(world)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def svd_costs(m, n):
    """Work estimate of one matrix of a batched SVD: m n^2 per sweep."""
    return [int(a) * int(b) * int(b) for a, b in zip(m, n)]


def _reduce(value, op_name, dist, device):
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return float(t.item())


def reduce_max(value, dist=None, device="cpu"):
    """Maximum of `value` over ranks (the identity without a process group)."""
    return _reduce(value, "MAX", dist, device)


def reduce_sum(value, dist=None, device="cpu"):
    """Sum of `value` over ranks (the identity without a process group)."""
    return _reduce(value, "SUM", dist, device)


def aggregate_rate(units, ms, dist=None, device="cpu"):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time.  Returns (units per second, total units, max ms)."""
    total = reduce_sum(units, dist, device)
    ms_max = reduce_max(ms, dist, device)
    if ms_max <= 0.0:
        raise ValueError("non-positive time")
    return total / (ms_max * 1e-3), total, ms_max
