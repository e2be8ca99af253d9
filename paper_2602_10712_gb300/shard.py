"""Sharding of independent (design, sun) items across ranks.

The force and torque of every (design, sun direction) item are independent
(Sec. 3.2: F(w, theta) per direction), so N GPUs split the items with no
data-path collective: rank r traces its contiguous slice with the RNG
counter offset sun_base = start, which makes the union of the shards equal
to the unsharded evaluation, and the results are gathered on the host (or
with one all-gather when a process group exists)."""
from __future__ import annotations

import numpy as np


def shard_range(n: int, rank: int, world: int):
    """Contiguous, balanced slice [start, stop) of n items for `rank`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def gather_items(local: np.ndarray, n: int, rank: int, world: int, group=None) -> np.ndarray:
    """All-gather per-rank slices [stop-start, ...] into the full [n, ...]
    array (torch.distributed, any backend; CPU tensors for gloo)."""
    import torch
    import torch.distributed as dist
    if world == 1:
        return np.asarray(local)
    slices = [shard_range(n, r, world) for r in range(world)]
    m = max(b - a for a, b in slices)
    shape = tuple(local.shape[1:])
    pad = np.zeros((m,) + shape, dtype=np.float64)
    pad[:local.shape[0]] = local
    t = torch.from_numpy(pad)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    outs = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(outs, t, group=group)
    full = np.zeros((n,) + shape)
    for r, (a, b) in enumerate(slices):
        full[a:b] = outs[r].cpu().numpy()[:b - a]
    return full
