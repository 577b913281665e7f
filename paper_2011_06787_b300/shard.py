"""Template sharding over ranks, one process per GPU.

Templates are independent in both the filter bank and the coherent scan (a template's
statistic needs only its own SNR of every detector), so a multi-GPU run gives each rank a
contiguous range of templates and exchanges no data.  The only collective is on the host
side of a benchmark: the maximum of the ranks' times and the sum of their work.
"""
from __future__ import annotations

import numpy as np


def template_shards(filter_offsets, world: int):
    """Contiguous template ranges [(lo, hi)] for ranks 0 .. world-1 whose filter counts are
    as equal as template boundaries allow (each cut at the template boundary nearest to r/world
    of the filters); every rank gets at least one template."""
    off = np.asarray(filter_offsets, dtype=np.int64)
    T = off.size - 1
    if world < 1 or world > T:
        raise ValueError(f"cannot split {T} templates over {world} ranks")
    F = int(off[-1])
    cuts = [0]
    for r in range(1, world):
        target = F * r / world
        t = int(np.searchsorted(off, target, side="left"))
        if t > 0 and target - off[t - 1] < off[min(t, T)] - target:
            t -= 1
        t = min(max(t, cuts[-1] + 1), T - (world - r))
        cuts.append(t)
    cuts.append(T)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def reduce_over_ranks(values, op: str = "max"):
    """Element-wise max or sum of a list of numbers over all ranks of the default process
    group; the values themselves when no group is initialised or it has one rank."""
    import torch
    import torch.distributed as dist
    vals = [float(v) for v in values]
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return vals
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor(vals, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op={"max": dist.ReduceOp.MAX, "sum": dist.ReduceOp.SUM}[op])
    return [float(x) for x in t.tolist()]
