"""Host-side placement of objects on ranks and the cross-rank reductions of the benchmark.

Objects share no parameters, so a training step over many objects is a set of independent problems: each rank
(one process per GPU) trains its own objects and nothing is exchanged on the data path.  Objects of uneven size are
placed with the longest-processing-time-first rule (each object, largest cost first, goes to the rank with the least
load so far; ties go to the lower rank), whose makespan is at most 4/3 - 1/(3 m) of the optimum (Graham, 1969).
The only collectives are the benchmark's: the maximum of the per-rank step times and sums of per-rank counters.
"""


def lpt_partition(costs, world):
    """Returns one list of object indices per rank (each list in ascending order)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def makespan(costs, parts):
    return max((sum(float(costs[i]) for i in p) for p in parts), default=0.0)


def _reduce(value, op, dist, device):
    import torch

    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(value, dist=None, device="cpu"):
    """Maximum over all ranks (the step time of the slowest rank)."""
    return _reduce(value, None if dist is None else dist.ReduceOp.MAX, dist, device)


def sum_over_ranks(value, dist=None, device="cpu"):
    """Sum over all ranks (samples processed by the whole job)."""
    return _reduce(value, None if dist is None else dist.ReduceOp.SUM, dist, device)
