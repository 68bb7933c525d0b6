"""Multi-GPU host logic: one process per GPU, no collective on the data path.

The method's units are independent where they shard at all: whole meshes of a
batch (each mesh's stencils, steps and adjoint stay inside the mesh), or
whole replicas of one mesh.  A rank works on its own units only; the ranks
meet twice per measurement, at a barrier before the timed region and in one
max-reduction of the timed duration after it (the job is as slow as its
slowest rank).  A single mesh split across GPUs would need a halo exchange
of the stencil cells every stage, which this package does not provide.
"""
from __future__ import annotations


def shard_meshes(cell_counts, world):
    """Whole meshes per rank, balanced by cell count: the largest mesh first
    to the rank with the fewest cells so far (ties to the lower rank), each
    rank's list in the batch order.  Returns one list of mesh indices per
    rank; every mesh appears exactly once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    parts = [[] for _ in range(world)]
    order = sorted(range(len(cell_counts)), key=lambda k: (-int(cell_counts[k]), k))
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(k)
        load[r] += int(cell_counts[k])
    return [sorted(p) for p in parts]


def max_over_ranks(value, dist=None, device=None):
    """The maximum of a per-rank float over the process group (the value
    itself without one)."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, dist=None, device=None):
    """The sum of a per-rank count over the process group."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_per_rank, ms, dist=None, device=None):
    """Units processed by all ranks per second, over the slowest rank's time
    (ms, per rank)."""
    total = sum_over_ranks(units_per_rank, dist, device)
    slowest = max_over_ranks(ms, dist, device)
    return total / (slowest * 1e-3), slowest
