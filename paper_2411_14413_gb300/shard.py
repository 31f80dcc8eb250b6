"""Sharding of one transport problem over several processes (one GPU each).

Particles are independent (Sec. "The SIMTRA model": no particle-particle
interaction), so a problem splits into disjoint ticket ranges with no data
exchange during transport.  The one exchange step is the sum of the ranks'
tallies at the end: an integer sum for counts and histograms, so the result
is bit-identical to one process running every ticket, and a floating-point
sum for energy and score.  Timing of a multi-process job is the slowest
rank's time with the work summed over ranks.

Host logic only: works with any torch.distributed backend (NCCL for device
tensors, gloo for host tensors).
"""

from __future__ import annotations


def ticket_shard(n_tickets: int, rank: int, world: int) -> tuple[int, int]:
    """[begin, end) of rank's contiguous share of n_tickets tickets; the shares
    of ranks 0..world-1 partition [0, n_tickets) and differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    if n_tickets < 0:
        raise ValueError("negative ticket count")
    q, r = divmod(int(n_tickets), int(world))
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def run_shard(transport, rank: int, world: int, seed=None, **kw):
    """Transport rank's share of the tickets of `transport` (an api.Transport)
    into its tallies; returns the run statistics."""
    b, e = ticket_shard(int(transport.layout.n_tickets), rank, world)
    return transport.run(seed=seed, ticket_begin=b, ticket_end=e, **kw)


def combine_tallies(tallies: dict, group=None) -> dict:
    """Sum every tally tensor over the ranks of `group` in place (all-reduce);
    the records buffer, if present, is per particle and is left alone."""
    import torch.distributed as dist

    for name in sorted(tallies):
        if name == "records":
            continue
        dist.all_reduce(tallies[name], op=dist.ReduceOp.SUM, group=group)
    return tallies


def reduce_job(time_ms: float, work: list, device=None, group=None) -> tuple[float, list]:
    """(max over ranks of time_ms, per-item sums over ranks of `work`)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(time_ms), [float(w) for w in work]
    t = torch.tensor([float(time_ms)], dtype=torch.float64, device=device)
    w = torch.tensor([float(x) for x in work], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(w, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), [float(x) for x in w.tolist()]
