"""Partition-sharded build across ranks (one GPU per rank): the divide-and-
conquer build of Section 3.2 with its partitions split over the ranks and its
Shuffle 2 as one all-to-all.

  1. Every rank holds all codes and the same routes (the Map step is cheap next
     to Reduce 1 and gives every rank the same answer).
  2. The partitions are assigned to ranks by longest-processing-time over their
     Reduce-1 work |V_p| |H_p| (the paper balances data skew the same way,
     Section 3.6 (1)): partitions in decreasing work, each to the least loaded
     rank (ties by partition, then rank).
  3. Each rank builds the graph of its own partitions only (route slots of other
     ranks' partitions become -1): for every point, the first k candidates by
     (d, id) among the homes of that rank's partitions -- a partial list.
  4. Shuffle 2: point i is owned by rank i // ceil(N / world); every rank sends
     each owner the partial rows of the owner's points (one all-to-all).
  5. Reduce 2: the owner merges the world partial rows of each of its points.
     The partitions' home sets are disjoint, so the partial lists hold disjoint
     candidates and the first k of their union is exactly the single-GPU row.

Host logic only: the compute steps are library calls (``build_fn`` and
``merge_fn`` default to bdg_build_graph and bdg_merge_lists).
"""
from __future__ import annotations

import numpy as np
import torch


def assign_partitions(home_count, visit_count, world: int) -> np.ndarray:
    """Owner rank of each partition (int64 [m]): longest-processing-time over
    the work |V_p| |H_p|."""
    hc = np.asarray(home_count, np.float64)
    vc = np.asarray(visit_count, np.float64)
    work = hc * vc
    order = np.lexsort((np.arange(work.size), -work))  # decreasing work, then p
    load = np.zeros(world)
    owner = np.empty(work.size, np.int64)
    for p in order:
        r = int(np.argmin(load))  # least loaded; argmin takes the first on ties
        owner[p] = r
        load[r] += work[p]
    return owner


def partition_counts(routes, m: int):
    """(|H_p|, |V_p|) per partition from routes [N, t] (slot 0 = home; -1 =
    no partition); torch tensors on the routes' device."""
    r = routes.long()
    hc = torch.bincount(r[:, 0][r[:, 0] >= 0], minlength=m)
    vc = torch.bincount(r[r >= 0], minlength=m)
    return hc, vc


def rank_routes(routes, owner, rank: int):
    """Routes with every slot naming another rank's partition set to -1."""
    own = torch.as_tensor(owner, device=routes.device) == rank
    keep = (routes >= 0) & own[routes.clamp(min=0).long()]
    return torch.where(keep, routes, torch.full_like(routes, -1)).contiguous()


def point_blocks(n: int, world: int):
    """Owner blocks of points: rank r owns [r * b, min(n, (r + 1) * b)), b =
    ceil(n / world)."""
    b = (n + world - 1) // world
    return [(min(n, r * b), min(n, (r + 1) * b)) for r in range(world)]


def exchange(ids, dists, world: int, rank: int, group=None):
    """Shuffle 2: every rank's partial rows [N, k] -> this rank's block of every
    rank's partial rows, stacked [world, block, k] (all_to_all over the point
    blocks; blocks are padded to one size for the collective)."""
    import torch.distributed as dist
    n, k = ids.shape
    blocks = point_blocks(n, world)
    b = blocks[0][1] - blocks[0][0]
    lo, hi = blocks[rank]

    def padded(x, fill):
        out = torch.full((world * b, k), fill, dtype=x.dtype, device=x.device)
        out[:n] = x
        return out

    pi, pd = padded(ids, -1), padded(dists, 0)
    ri, rd = torch.empty_like(pi), torch.empty_like(pd)
    dist.all_to_all_single(ri, pi, group=group)
    dist.all_to_all_single(rd, pd, group=group)
    return ri.view(world, b, k)[:, : hi - lo], rd.view(world, b, k)[:, : hi - lo]


def _library_build(codes, k, m, t, routes, entry):
    from . import build_graph
    g = build_graph(codes, k, m=m, t=t, routes=routes, entry=entry)
    ids, dists = g.ids.clone(), g.dists.clone()
    g.free()
    return ids, dists


def _library_merge(ids, dists, bits):
    from . import merge_lists
    return merge_lists(ids, dists, bits)


def sharded_build(codes, k: int, m: int, routes, entry, world: int, rank: int, bits: int,
                  group=None, build_fn=None, merge_fn=None):
    """This rank's block of the graph rows: (lo, ids [block, k], dists [block, k]).
    Collective: every rank of the group must call it with the same routes."""
    build_fn = build_fn or _library_build
    merge_fn = merge_fn or (lambda i, d: _library_merge(i, d, bits))
    t = routes.shape[1]
    hc, vc = partition_counts(routes, m)
    owner = assign_partitions(hc.cpu().numpy(), vc.cpu().numpy(), world)
    ids, dists = build_fn(codes, k, m, t, rank_routes(routes, owner, rank), entry)
    pi, pd = exchange(ids, dists, world, rank, group)
    mi, md = merge_fn(pi.contiguous(), pd.contiguous())
    return point_blocks(codes.shape[0], world)[rank][0], mi, md
