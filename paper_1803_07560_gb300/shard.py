"""Multi-GPU: subvolumes are independent (Sec. 1, 3: the integral over a region
is the sum over its parts), so N ranks take contiguous shards of a job's
subvolumes with no exchange during the integration; the one exchange is an
all-gather of the per-subvolume records, merged in FP64 on the host by the
library's merge."""
from __future__ import annotations

import numpy as np


def shard_range(nsub: int, world: int, rank: int) -> tuple[int, int]:
    """[start, stop) of the subvolumes rank 'rank' of 'world' integrates."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    base, extra = divmod(nsub, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def gather_records(slots, group=None):
    """All ranks' records [*, slot_len], concatenated in rank order.  'slots'
    is a torch tensor on the device the process group uses (CUDA for NCCL,
    CPU for gloo); shards may differ in size."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n = torch.tensor([slots.shape[0]], dtype=torch.int64, device=slots.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    width = slots.shape[1]
    padded = torch.zeros((max(sizes), width), dtype=slots.dtype, device=slots.device)
    padded[:slots.shape[0]] = slots
    parts = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    return np.concatenate([p[:s].cpu().numpy() for p, s in zip(parts, sizes)])


def merge_across_ranks(nx: int, slots, group=None) -> np.ndarray:
    """Totals of the whole job from every rank's records (FP64, host)."""
    from . import merge_host
    return merge_host(nx, gather_records(slots, group))
