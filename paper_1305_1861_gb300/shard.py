"""Key-range sharding across processes (one GPU each) with torch.distributed.

The paper routes every k-mer by its key to one of T consumers, each owning the k-mers of its
share of the key space (Sec. 2.1.5). Across GPUs the same routing needs no exchange of keys:
rank r of a group of N counts only the keys of shard r -- one of N consecutive key ranges of the
library, balanced by window counts (turtle_shard_bounds) -- while reading all the reads. Since the
shards are consecutive ranges in ascending order, rank 0 gets the whole result by concatenating
the shards in rank order; that gather is the only collective, and it moves results, not windows.

This module is marshalling only: the counting runs in libturtle's kernels (turtle_count with
params.shard_index / params.shard_count).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import Params, TURTLE_OK, TurtleError, load, turtle_count

__all__ = ["shard_bounds", "shard_params", "gather_shards", "count_sharded"]


def shard_bounds(part_windows, n_shards: int) -> np.ndarray:
    """Bounds of n_shards consecutive part ranges balanced by window counts (turtle_shard_bounds):
    shard s takes parts [b[s], b[s+1])."""
    w = np.ascontiguousarray(part_windows, dtype=np.uint64)
    out = np.zeros(n_shards + 1, dtype=np.uint32)
    rc = load().turtle_shard_bounds(w.ctypes.data, w.size, n_shards, out.ctypes.data)
    if rc != TURTLE_OK:
        raise TurtleError(rc, "turtle_shard_bounds")
    return out


def shard_params(rank: int, world: int, params: Params | None = None) -> Params:
    """params (or the defaults) restricted to shard `rank` of `world`."""
    p = Params.from_buffer_copy(params) if params is not None else Params.default()
    p.shard_count = world if world > 1 else 0
    p.shard_index = rank if world > 1 else 0
    return p


def _dist():
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        raise RuntimeError("torch.distributed is not initialised")
    return dist


def gather_shards(keys: np.ndarray, counts: np.ndarray, device=None):
    """Send this rank's shard (keys uint64[n] or uint64[n, 2], counts uint32[n]) to rank 0 of the default
    group; rank 0 returns the concatenation in rank order, the other ranks None. device: where the
    messages are staged (CUDA for NCCL; CPU, the default, for gloo)."""
    import torch

    dist = _dist()
    rank, world = dist.get_rank(), dist.get_world_size()
    dev = torch.device(device) if device is not None else torch.device("cpu")
    w = 2 if keys.ndim == 2 else 1
    n = torch.tensor([counts.shape[0], w], dtype=torch.int64, device=dev)
    if rank != 0:
        dist.send(n, 0)
        if counts.shape[0]:
            dist.send(torch.from_numpy(np.ascontiguousarray(keys).view(np.int64).reshape(-1)).to(dev), 0)
            dist.send(torch.from_numpy(np.ascontiguousarray(counts).view(np.int32)).to(dev), 0)
        return None
    parts_k, parts_c = [np.ascontiguousarray(keys)], [np.ascontiguousarray(counts)]
    for r in range(1, world):
        dist.recv(n, r)
        m, wr = int(n[0]), int(n[1])
        if wr != w:
            raise ValueError("rank %d sent %d-word keys, rank 0 holds %d-word keys" % (r, wr, w))
        if m:
            kb = torch.empty(m * w, dtype=torch.int64, device=dev)
            cb = torch.empty(m, dtype=torch.int32, device=dev)
            dist.recv(kb, r)
            dist.recv(cb, r)
            ks = kb.cpu().numpy().view(np.uint64)
            parts_k.append(ks.reshape(m, 2) if w == 2 else ks)
            parts_c.append(cb.cpu().numpy().view(np.uint32))
    return np.concatenate(parts_k, axis=0), np.concatenate(parts_c)


def count_sharded(bases, offsets, k: int, min_count: int = 2, params: Params | None = None, count=None,
                  device=None):
    """Whole-library count split by key range over the ranks of the default group: this rank counts its
    shard (turtle_count with shard params, or `count(bases, offsets, k, min_count, params)` if given),
    rank 0 gathers. Returns (keys, counts, n_windows) on rank 0 and None elsewhere."""
    dist = _dist()
    rank, world = dist.get_rank(), dist.get_world_size()
    p = shard_params(rank, world, params)
    keys, counts, nw = (count or turtle_count)(bases, offsets, k, min_count, p)
    got = gather_shards(np.asarray(keys), np.asarray(counts), device)
    if got is None:
        return None
    return got[0], got[1], nw
