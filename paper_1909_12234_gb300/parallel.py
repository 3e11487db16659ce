"""Sample sharding across ranks (one process per GPU).

The Hutchinson samples are independent (Eq. 1), so ranks never exchange
field data: each rank solves its own contiguous range of global sample
indices, and only the per-sample values t_j are gathered at the end, in
global sample order, for the statistics (computed on the device by
``qdtrace.trace_stats``).  Works with any torch.distributed backend (NCCL
on GPUs, gloo on CPUs).
"""

import numpy as np


def sample_offset(rank, world, batch, step, base=0):
    """First global sample index of `rank`'s batch number `step` (each batch
    holds `batch` samples; the world processes world * batch per step)."""
    if not (0 <= rank < world) or batch < 1 or step < 0:
        raise ValueError("bad rank/world/batch/step")
    return base + (step * world + rank) * batch


def sample_indices(rank, world, batch, steps, base=0):
    """All global sample indices `rank` processes in `steps` batches."""
    return np.concatenate([np.arange(batch) + sample_offset(rank, world, batch, k, base) for k in range(steps)])


def gather_samples(t_local, idx_local, group=None):
    """Gather per-sample values from every rank and return them sorted by
    global sample index: (indices, values).  Every rank receives the result."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    payload = np.stack([np.asarray(idx_local, dtype=np.float64),
                        np.asarray(t_local).real.astype(np.float64),
                        np.asarray(t_local).imag.astype(np.float64)])
    local = torch.from_numpy(payload).to(dev)
    n = torch.tensor([local.shape[1]], dtype=torch.int64, device=dev)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    width = int(max(s.item() for s in sizes))
    padded = torch.zeros((3, width), dtype=torch.float64, device=dev)
    padded[:, :local.shape[1]] = local
    bufs = [torch.zeros_like(padded) for _ in range(world)]
    dist.all_gather(bufs, padded, group=group)
    parts = [b[:, :int(s.item())].cpu().numpy() for b, s in zip(bufs, sizes)]
    allp = np.concatenate(parts, axis=1)
    order = np.argsort(allp[0], kind="stable")
    idx = allp[0][order].astype(np.int64)
    if len(np.unique(idx)) != len(idx):
        raise ValueError("two ranks processed the same sample index")
    return idx, allp[1][order] + 1j * allp[2][order]
