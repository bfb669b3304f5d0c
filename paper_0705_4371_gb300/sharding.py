"""Multi-GPU layout of the batched form: independent runs are assigned whole
to ranks (no exchange between ranks on the data path); the only collective
is the max over ranks of the timed region.

assign_runs is deterministic, so every rank computes the same assignment
without communicating.
"""


def assign_runs(sites, world):
    """Longest-first greedy assignment of runs (by site count) to `world`
    ranks: each run, largest first (ties: lower index), goes to the rank
    with the fewest sites so far (ties: lower rank).  Returns one sorted
    list of run indices per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    share = [[] for _ in range(world)]
    for r in sorted(range(len(sites)), key=lambda i: (-int(sites[i]), i)):
        k = min(range(world), key=lambda q: (load[q], q))
        share[k].append(r)
        load[k] += int(sites[r])
    return [sorted(s) for s in share]


def max_over_ranks(value, device=None):
    """The largest `value` over the ranks of the default process group (the
    value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
