"""Haloes of one catalogue spread over several GPUs (one process per GPU).

Haloes are independent units: the analysis needs no communication while it
runs and no halo is ever split (Sect. 2.2: each process analyses the haloes
whose centres it holds).  Here the units are dealt out by greedy
longest-processing-time (LPT) on the candidate count, the cost proxy of a
halo; the only exchange is a final gather of the fixed-size result records
and the bound lists, on the host.

The compute step is passed in, so the same plumbing serves the GPU path
(ahf.Context.unbind_batch on each rank's device) and host-only tests.
"""
from __future__ import annotations

import heapq

import numpy as np


def lpt_partition(counts, n_ranks):
    """Greedy LPT: haloes in decreasing count order, each to the rank with the
    smallest load so far (ties: lower rank, then lower halo index first).
    Returns one sorted index array per rank."""
    counts = np.asarray(counts, dtype=np.int64)
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(counts)), key=lambda h: (-int(counts[h]), h))
    heap = [(0, r) for r in range(n_ranks)]
    parts = [[] for _ in range(n_ranks)]
    for h in order:
        load, r = heapq.heappop(heap)
        parts[r].append(h)
        heapq.heappush(heap, (load + max(int(counts[h]), 1), r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def loads(counts, parts):
    counts = np.asarray(counts, dtype=np.int64)
    return [int(np.maximum(counts[p], 1).sum()) for p in parts]


def run_sharded(n_halos, counts, compute, rank, world, group=None):
    """Run `compute(halo_indices) -> (records, bound_lists)` on this rank's
    share and gather everything on rank 0.

    records: structured array, one record per halo of the share, in the
    share's order; bound_lists: list of int64 arrays (particle indices).
    Returns (records, bound_lists) for the whole catalogue in halo order on
    rank 0, None elsewhere."""
    parts = lpt_partition(counts, world)
    mine = parts[rank]
    rec, bound = compute(mine)
    if len(rec) != len(mine) or len(bound) != len(mine):
        raise ValueError("compute must return one record and one bound list per halo")
    lengths = np.array([len(b) for b in bound], dtype=np.int64)
    flat = np.concatenate(bound).astype(np.int64) if len(bound) else np.zeros(0, np.int64)
    payload = (mine, rec, lengths, flat)
    if world == 1:
        gathered = [payload]
    else:
        import torch.distributed as dist
        gathered = [None] * world if rank == 0 else None
        dist.gather_object(payload, gathered, dst=0, group=group)
    if rank != 0:
        return None
    out_rec = None
    out_bound = [None] * n_halos
    for idx, r, ln, fl in gathered:
        if out_rec is None:
            out_rec = np.zeros(n_halos, dtype=r.dtype)
        out_rec[idx] = r
        ends = np.cumsum(ln)
        starts = ends - ln
        for k, h in enumerate(idx):
            out_bound[int(h)] = fl[starts[k]:ends[k]]
    if any(b is None for b in out_bound):
        raise RuntimeError("a halo was not covered by any rank")
    return out_rec, out_bound
