"""Host-side logic for running independent domains on several GPUs (one process per GPU).

The batched workload of Sec. 4.1 is a set of independent domains: they exchange nothing, so
spreading them over ranks needs no data-path collective.  Each rank builds one context over
its own share of the domains; the only communication is the max-over-ranks reduction of the
measured time (and of any scalar the caller wants to combine).
"""
from __future__ import annotations


def shard_domains(cells, world):
    """Assign domains to `world` ranks, balancing the cells each rank advances.

    cells: cell count of each domain (the work of one time step is proportional to it).
    Returns a list of `world` sorted index lists.  Longest-processing-time-first greedy: domains
    in descending size (ties by index) go to the rank with the fewest cells so far (ties by rank),
    so the result is deterministic and the largest rank load exceeds the mean by less than the
    largest single domain.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(cells)), key=lambda d: (-int(cells[d]), d))
    load = [0] * world
    out = [[] for _ in range(world)]
    for d in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(d)
        load[r] += int(cells[d])
    return [sorted(s) for s in out]


def max_over_ranks(value, dist=None, device=None):
    """Largest `value` over all ranks of the default process group (the value itself without one).

    Used for timings: a multi-rank job is as slow as its slowest rank.  `device` is where the
    reduction tensor lives (a CUDA device for NCCL, None = CPU for gloo).
    """
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, dist=None, device=None):
    """Sum of `value` over all ranks (e.g. the cells each rank advanced)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
