"""One dataset's all-against-all Best Hits split across processes (one per GPU).

The paper decomposes the comparison phase by data, one query gene -- one row
of Algorithm 2 -- being a unit of work ("Parallel implementation").  Across
GPUs the same holds: every process profiles the same dataset (the index is
replicated), takes one shard of the query genes (``pd_best_hits_shard``) and
computes those rows against every genome; the mutual check of Eq. (9) needs
the rows of both genes of a pair, so the rows are gathered to one process,
assembled into one handle (``pd_hits_import``) and BBH runs there
(``pd_bbh_all``).

This module only moves arrays between processes (``torch.distributed``); the
Best Hits, their assembly and the BBH all run in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import pd


def _backend_device(dist):
    """Tensors for collectives live on the GPU with NCCL, on the host with gloo."""
    import torch
    if dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def gather_pieces(row_ptr, cols, s, root: int = 0):
    """All-gather this process's CSR piece (row_ptr int64 [G+1], cols int32,
    s int32/uint32) and return every process's piece on `root` (None on the
    others).  Pieces are torch tensors on the collective's device."""
    import torch
    import torch.distributed as dist
    dev = _backend_device(dist)
    world, rank = dist.get_world_size(), dist.get_rank()
    rp = torch.as_tensor(row_ptr).to(dev, torch.int64)
    c = torch.as_tensor(cols).to(dev, torch.int32)
    v = torch.as_tensor(np.asarray(s).view(np.int32) if isinstance(s, np.ndarray) else s).to(dev, torch.int32)
    n = torch.tensor([c.numel()], dtype=torch.int64, device=dev)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n)
    sizes = [int(x.item()) for x in sizes]
    cap = max(1, max(sizes))
    pad_c = torch.zeros(cap, dtype=torch.int32, device=dev)
    pad_v = torch.zeros(cap, dtype=torch.int32, device=dev)
    pad_c[:c.numel()] = c
    pad_v[:v.numel()] = v
    all_rp = [torch.zeros_like(rp) for _ in range(world)]
    all_c = [torch.zeros_like(pad_c) for _ in range(world)]
    all_v = [torch.zeros_like(pad_v) for _ in range(world)]
    dist.all_gather(all_rp, rp)
    dist.all_gather(all_c, pad_c)
    dist.all_gather(all_v, pad_v)
    if rank != root:
        return None
    return [(all_rp[r], all_c[r][:sizes[r]], all_v[r][:sizes[r]]) for r in range(world)]


def sharded_best_hits(ctx, prof, rank: int, world: int, on_device=None):
    """This process's shard of the Best Hits as a CSR piece over every gene.
    on_device: a torch device to copy into (device tensors), else host arrays."""
    import torch
    hits = pd.pd_best_hits_shard(ctx, prof, rank, world)
    info = pd.pd_hits_get_info(hits)
    if on_device is None:
        return pd.pd_hits_copy(ctx, hits)
    rp = torch.empty(info.n_rows + 1, dtype=torch.int64, device=on_device)
    cols = torch.empty(max(1, info.n_hits), dtype=torch.int32, device=on_device)
    s = torch.empty(max(1, info.n_hits), dtype=torch.int32, device=on_device)
    n = pd.pd_hits_copy(ctx, hits, rp, cols, s)
    return rp, cols[:n], s[:n]


def sharded_bbh(ctx, prof, root: int = 0):
    """The whole all-against-all result of one dataset computed by every
    process of the default group together: each its shard of the query genes,
    then the pieces gathered and BBH run on `root`.  Returns (hits, bbh)
    handles on root, (None, None) elsewhere."""
    import torch.distributed as dist
    world, rank = dist.get_world_size(), dist.get_rank()
    dev = _backend_device(dist)
    piece = sharded_best_hits(ctx, prof, rank, world, on_device=dev if dev.type == "cuda" else None)
    pieces = gather_pieces(*piece, root=root)
    if pieces is None:
        return None, None
    hits = pd.pd_hits_import(ctx, prof, pieces)
    return hits, pd.pd_bbh_all(ctx, prof, hits)
