"""One graph's edge networks sharded over ranks (one process per GPU).

The Max-Cut objective of Section 4.1 is a sum over edges, and every edge's
<Z_u Z_v> network is contracted on its own, so a graph shards with no data
exchanged until the end: each rank evaluates its part of the edge networks
(chosen by the library's longest-processing-time partition, identical on
every rank because planning is seeded) and the 1 + 2p partial sums (<C> and
its gradient) are added once in FP64 across ranks.
"""

from __future__ import annotations


def shard(batch, rank: int, world: int, want_grad: bool = True):
    """(this rank's sub-batch or None when it gets no network, the indices of
    its networks in `batch`)."""
    if world <= 1:
        return batch, list(range(len(batch.edges)))
    parts, _ = batch.partition(world, want_grad)
    mine = [i for i, r in enumerate(parts) if r == rank]
    if not mine:
        return None, []
    return batch.subset(mine), mine


def allreduce_sum(values, device=None):
    """The one exchange of a sharded evaluation: the element-wise FP64 sum of
    every rank's partial results (a torch tensor or a sequence), over the
    default process group when one with more than one rank exists (NCCL for
    CUDA tensors, gloo on the CPU)."""
    import torch
    import torch.distributed as dist
    t = values if isinstance(values, torch.Tensor) else torch.tensor(
        list(values), dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t
