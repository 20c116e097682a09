"""Sharding across GPUs (one process per GPU).

Trials are independent (each is one simulated year of the YET), so a run
splits the YET into contiguous trial blocks, one per rank, with no exchange
during the analysis stage.  The one exchange step is for the filters on the
YLT: PML and TVaR are order statistics of all trials, so the ranks' YLT
blocks are gathered (rank order = trial order) before the selection.

Layers are independent too (the Basic Algorithm loops over them), so a
portfolio can instead be split by layer: each rank analyses whole layers
over every trial and selects their PML/TVaR itself, with no exchange at
all until the per-layer results are collected.
"""
from __future__ import annotations


def trial_shard(n_trials: int, world: int, rank: int) -> tuple[int, int]:
    """(first trial, trial count) of `rank`'s block: sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(int(n_trials), world)
    begin = rank * base + min(rank, extra)
    return begin, base + (1 if rank < extra else 0)


def gather_ylt(local, group=None):
    """Concatenate every rank's YLT block in rank order (blocks may differ in
    length).  Works for CPU tensors over gloo and CUDA tensors over NCCL."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n = torch.tensor([local.numel()], dtype=torch.int64, device=local.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    m = max(sizes)
    padded = torch.zeros(m, dtype=local.dtype, device=local.device)
    padded[: local.numel()] = local
    out = torch.empty(world * m, dtype=local.dtype, device=local.device)
    dist.all_gather_into_tensor(out, padded, group=group)
    return torch.cat([out[r * m: r * m + sizes[r]] for r in range(world)])


def layer_shard(work, world: int, rank: int) -> list[int]:
    """Indices of the layers `rank` analyses, balancing the summed `work`
    (e.g. occurrences x ELTs per layer): layers in decreasing work go to the
    least-loaded rank so far (ties to the lowest rank), the same on every
    rank.  Each rank's list is in increasing layer order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    order = sorted(range(len(work)), key=lambda i: (-float(work[i]), i))
    load = [0.0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += float(work[i])
        if r == rank:
            mine.append(i)
    return sorted(mine)


def gather_results(local: dict, n_layers: int, group=None):
    """Collect {layer index: (pml list, tvar list)} from every rank into one
    list indexed by layer (a small all-gather of plain values)."""
    import torch.distributed as dist
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, local, group=group)
    out = [None] * n_layers
    for part in parts:
        for i, v in part.items():
            out[int(i)] = v
    return out
