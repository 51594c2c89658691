"""Sharding one database search over several GPUs (one process per GPU).

Every (query, database sequence) pair is independent (Section III, stage (ii)
spreads the database over the coprocessors), so the path shards by database
sequence with a single exchange at the end:

- ``partition``: sequences are dealt to ranks longest first, each to the rank
  holding the fewest residues so far, so every rank gets about the same
  number of DP cells for any query (the paper balances its coprocessors with
  a pool of length-sorted chunks);
- each rank loads its shard (``sw_db_load``) and searches it; its local top-k
  indices are mapped back to global database indices;
- ``merge_top_k`` / ``allgather_top_k``: one all-gather of k (score, global
  index) pairs per rank gives the global top-k under the same order (score
  descending, then index ascending) the single-GPU search uses.

Full score vectors stay on their rank (concatenate by ``global_index`` if a
caller needs them). This module moves data only; the scoring runs in the
CUDA library.
"""
from __future__ import annotations

import heapq

import numpy as np


def partition(offsets, world: int) -> list:
    """Global sequence indices of each rank's shard (ascending within a shard)."""
    off = np.asarray(offsets, dtype=np.uint64)
    lengths = (off[1:] - off[:-1]).astype(np.int64)
    order = np.lexsort((np.arange(lengths.size), -lengths))
    heap = [(0, r) for r in range(world)]
    owner = np.empty(lengths.size, dtype=np.int64)
    for s in order:
        load, r = heapq.heappop(heap)
        owner[s] = r
        heapq.heappush(heap, (load + int(lengths[s]), r))
    return [np.nonzero(owner == r)[0] for r in range(world)]


def shard_arrays(residues, offsets, global_index):
    """(residues, offsets) of the sequences in ``global_index``, in that order."""
    res = np.asarray(residues, dtype=np.uint8)
    off = np.asarray(offsets, dtype=np.uint64)
    gi = np.asarray(global_index, dtype=np.int64)
    lengths = (off[gi + 1] - off[gi]).astype(np.uint64)
    new_off = np.zeros(gi.size + 1, dtype=np.uint64)
    np.cumsum(lengths, out=new_off[1:])
    out = np.empty(int(new_off[-1]), dtype=np.uint8)
    src = off[gi].tolist()
    dst = new_off.tolist()
    for k in range(gi.size):
        out[dst[k]:dst[k + 1]] = res[src[k]:src[k] + (dst[k + 1] - dst[k])]
    return out, new_off


def local_to_global(local_index, global_index):
    """Map a shard's top-k indices (positions in its shard) to global database indices."""
    gi = np.asarray(global_index, dtype=np.uint64)
    return gi[np.asarray(local_index, dtype=np.int64)]


def sharded_top_k(residues, offsets, queries, k: int, search_shard, rank: int, world: int,
                  group=None):
    """The whole sharded search of one database on this rank: take this rank's shard of
    ``partition``, call ``search_shard(shard_residues, shard_offsets, queries, k)`` (which
    returns per query the shard-local top-k scores and indices, ordered as stage (iv)
    orders them), map the indices to global ones and merge over all ranks with one
    all-gather per query. Returns the global top-k (scores, indices) of every query."""
    gi = partition(offsets, world)[rank]
    sres, soff = shard_arrays(residues, offsets, gi)
    local = search_shard(sres, soff, queries, k)
    merged = []
    for ts, ti in local:
        merged.append(allgather_top_k(ts, local_to_global(ti, gi), k, group=group))
    return merged


def merge_top_k(parts, k: int):
    """Global top-k from per-rank lists of (scores int32, global indices uint64)."""
    if not parts:
        return np.zeros(0, np.int32), np.zeros(0, np.uint64)
    s = np.concatenate([np.asarray(p[0], dtype=np.int64) for p in parts])
    i = np.concatenate([np.asarray(p[1], dtype=np.uint64) for p in parts])
    order = np.lexsort((i, -s))[:k]
    return s[order].astype(np.int32), i[order]


def allgather_top_k(local_scores, local_global_index, k: int, group=None):
    """All-gather every rank's local top-k (k pairs) and merge; every rank gets the result."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    kk = min(k, len(local_scores))
    buf = torch.full((k, 2), -1, dtype=torch.int64)
    buf[:kk, 0] = torch.as_tensor(np.asarray(local_scores[:kk], dtype=np.int64))
    buf[:kk, 1] = torch.as_tensor(np.asarray(local_global_index[:kk], dtype=np.int64))
    backend = dist.get_backend(group)
    if backend == "nccl":
        buf = buf.cuda()
    gathered = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(gathered, buf, group=group)
    parts = []
    for g in gathered:
        g = g.cpu().numpy()
        valid = g[:, 1] >= 0
        parts.append((g[valid, 0].astype(np.int32), g[valid, 1].astype(np.uint64)))
    return merge_top_k(parts, k)
