"""Template sharding over ranks, one process per GPU.

Templates are independent in both the filter bank and the coherent scan (a template's
statistic needs only its own SNR of every detector), so a multi-GPU run gives each rank a
contiguous range of templates and exchanges no data.  The candidate stage compares templates
of one bank (the largest SNR over the bank per sample, Sec. II.C.1), so shards cut at bank
boundaries keep it local; a bank that must span ranks takes one all-reduce(max) of its
per-sample maxima (bank_max_over_ranks).  The benchmark's own collectives are on the host:
the maximum of the ranks' times and the sum of their work.
"""
from __future__ import annotations

import numpy as np


def template_shards(filter_offsets, world: int, bank_starts=None):
    """Contiguous template ranges [(lo, hi)] for ranks 0 .. world-1 whose filter counts are
    as equal as the allowed cuts permit (each cut at the allowed boundary nearest to r/world of
    the filters); every rank gets at least one template.

    Without bank_starts every template boundary is allowed.  With bank_starts (the first
    template of each bank, ascending, starting at 0) only bank boundaries are: no bank spans two
    ranks, so the per-bank quantities of the candidate stage (the largest SNR over a bank's
    templates per sample, Sec. II.C.1) stay local to one rank.  That needs at least as many
    banks as ranks."""
    off = np.asarray(filter_offsets, dtype=np.int64)
    T = off.size - 1
    if bank_starts is None:
        allowed = np.arange(T + 1)
    else:
        allowed = np.asarray(list(bank_starts) + [T], dtype=np.int64)
        if allowed[0] != 0 or np.any(np.diff(allowed) <= 0) or allowed[-1] != T:
            raise ValueError("bank_starts must start at 0 and increase below the template count")
    n_units = allowed.size - 1
    if world < 1 or world > n_units:
        raise ValueError(f"cannot split {n_units} {'banks' if bank_starts is not None else 'templates'} "
                         f"over {world} ranks")
    F = int(off[-1])
    at = off[allowed]           # filters before each allowed cut
    cuts = [0]                  # indices into allowed
    for r in range(1, world):
        target = F * r / world
        i = int(np.searchsorted(at, target, side="left"))
        if i > 0 and target - at[i - 1] < at[min(i, n_units)] - target:
            i -= 1
        i = min(max(i, cuts[-1] + 1), n_units - (world - r))
        cuts.append(i)
    cuts.append(n_units)
    return [(int(allowed[cuts[r]]), int(allowed[cuts[r + 1]])) for r in range(world)]


def bank_max_over_ranks(m2_local, t_local):
    """Per-sample maximum over a bank whose templates are split over the ranks of the default
    process group (Sec. II.C.1: the largest |z| over the bank's templates decides the
    single-detector candidates).  m2_local [..] float32: each rank's largest FP32 |z|^2 over its
    own templates of the bank per sample (-1 where it has none); t_local [..] int: the global
    index of that template.  Returns (m2, t) over all ranks, the lowest template among equal
    maxima, by one all-reduce(max) of 64-bit keys (the float's bits, which order as the values
    for non-negative floats, above the complement of the template index).  Without a group (or
    with one rank) the local values are returned."""
    import torch
    import torch.distributed as dist
    m2 = np.ascontiguousarray(m2_local, dtype=np.float32)
    t = np.asarray(t_local, dtype=np.int64)
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return m2.copy(), t.copy()
    bits = np.where(m2 >= 0, m2, np.float32(0)).view(np.int32).astype(np.int64)
    key = np.where(m2 >= 0, (bits << 32) | (0xFFFFFFFF - t), -1)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    k = torch.from_numpy(key).to(dev)
    dist.all_reduce(k, op=dist.ReduceOp.MAX)
    k = k.cpu().numpy()
    ok = k >= 0
    m2_out = np.where(ok, ((k >> 32) & 0xFFFFFFFF).astype(np.int64).astype(np.int32).view(np.float32), np.float32(-1))
    t_out = np.where(ok, 0xFFFFFFFF - (k & 0xFFFFFFFF), -1)
    return m2_out.astype(np.float32), t_out.astype(np.int64)


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
