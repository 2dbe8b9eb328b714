"""RP-Tuning split over several GPUs by node ranges (one process per GPU).

RP-Tuning rewrites every node's out-list from that node's own list alone
(§3), so the nodes split into contiguous id ranges with no exchange: each
rank tunes the slice of the base graph holding its range (rp_graph_slice ->
rp_tune_batch), and the tuned CSR is the concatenation of the ranks' rows in
range order.  Gathering the slices is optional (a caller may keep the graph
sharded); :func:`gather_slices` does it with one all-gather over a
torch.distributed process group.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import rp_graph_export, rp_graph_free, rp_graph_info, rp_graph_slice, rp_tune_batch


@dataclass
class Slice:
    """Rows lo .. hi-1 of a tuned graph: row_ptr has hi - lo + 1 entries from 0."""
    lo: int
    hi: int
    row_ptr: np.ndarray
    col: np.ndarray


def node_range(rank: int, world: int, n: int) -> tuple[int, int]:
    """Contiguous, balanced range of node ids for `rank` of `world`."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside [0, {world})")
    return n * rank // world, n * (rank + 1) // world


def slice_of(row_ptr: np.ndarray, col: np.ndarray, lo: int, hi: int) -> Slice:
    """Rows lo .. hi-1 of a CSR graph as a Slice."""
    rp = np.asarray(row_ptr[lo:hi + 1], dtype=np.int64)
    return Slice(lo, hi, rp - rp[0], np.ascontiguousarray(col[rp[0]:rp[-1]], dtype=np.int32))


def tune_slices(ctx, base: int, alphas, Rs, rank: int, world: int) -> list:
    """Tune this rank's node range of `base` for every target; one Slice per target."""
    n = rp_graph_info(ctx, base)["n"]
    lo, hi = node_range(rank, world, n)
    part = rp_graph_slice(ctx, base, lo, hi)
    try:
        outs = rp_tune_batch(ctx, part, alphas, Rs)
    finally:
        rp_graph_free(ctx, part)
    slices = []
    for g in outs:
        row_ptr, col = rp_graph_export(ctx, g)
        rp_graph_free(ctx, g)
        slices.append(slice_of(row_ptr, col, lo, hi))
    return slices


def assemble(slices: list, n: int) -> tuple[np.ndarray, np.ndarray]:
    """Concatenate Slices covering 0 .. n-1 (any order) into one CSR graph."""
    slices = sorted(slices, key=lambda s: s.lo)
    at = 0
    for s in slices:
        if s.lo != at or s.hi < s.lo or s.row_ptr.shape != (s.hi - s.lo + 1,):
            raise ValueError(f"slices do not tile 0..{n}: got [{s.lo}, {s.hi}) at {at}")
        at = s.hi
    if at != n:
        raise ValueError(f"slices end at {at}, not {n}")
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    base = 0
    for s in slices:
        row_ptr[s.lo + 1:s.hi + 1] = base + s.row_ptr[1:]
        base += int(s.row_ptr[-1])
    col = np.concatenate([s.col for s in slices]) if slices else np.zeros(0, np.int32)
    return row_ptr, np.ascontiguousarray(col, dtype=np.int32)


def gather_slices(my_slices: list, n: int, group=None) -> list:
    """All-gather every rank's Slices (one list per target) and assemble each
    target's graph on every rank.  Uses torch.distributed (gloo or nccl)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    got = [None] * world
    dist.all_gather_object(got, my_slices, group=group)
    return [assemble([got[r][t] for r in range(world)], n) for t in range(len(my_slices))]
