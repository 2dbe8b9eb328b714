"""RP-Tuning split over several GPUs by node ranges (one process per GPU).

RP-Tuning rewrites every node's out-list from that node's own list alone
(§3), so the nodes split into contiguous id ranges with no exchange: each
rank tunes the slice of the base graph holding its range (rp_graph_slice ->
rp_tune_batch), and the tuned CSR is the concatenation of the ranks' rows in
range order.  Gathering the slices is optional (a caller may keep the graph
sharded); :func:`gather_slices` does it with tensor all-gathers of the row
lengths and column ids over a torch.distributed process group (nccl on the
GPUs, gloo on the host).
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


def allgather_csr(counts, col, n: int, group=None):
    """One target's tuned graph from every rank's part, as torch tensors on the
    device the inputs live on (this rank's GPU under nccl, the host under gloo).

    counts: int64 row lengths of this rank's node range (node_range order);
    col: int32 column ids of those rows.  Three tensor all-gathers: the row
    lengths (padded to the longest range), the slice sizes, the column ids
    (padded to the largest slice).  Returns (row_ptr int64[n+1], col int32).
    """
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = counts.device
    ranges = [node_range(r, world, n) for r in range(world)]
    span = max(hi - lo for lo, hi in ranges)
    cnt = torch.zeros(span, dtype=torch.int64, device=dev)
    cnt[:counts.shape[0]] = counts
    all_cnt = [torch.empty_like(cnt) for _ in range(world)]
    dist.all_gather(all_cnt, cnt, group=group)
    nnz = torch.tensor([col.shape[0]], dtype=torch.int64, device=dev)
    all_nnz = [torch.empty_like(nnz) for _ in range(world)]
    dist.all_gather(all_nnz, nnz, group=group)
    sizes = [int(x.item()) for x in all_nnz]
    pad = torch.full((max(max(sizes), 1),), -1, dtype=torch.int32, device=dev)
    pad[:col.shape[0]] = col
    all_col = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(all_col, pad, group=group)
    lengths = torch.cat([all_cnt[r][:hi - lo] for r, (lo, hi) in enumerate(ranges)])
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    torch.cumsum(lengths, 0, out=row_ptr[1:])
    return row_ptr, torch.cat([all_col[r][:sizes[r]] for r in range(world)])


def gather_slices(my_slices: list, n: int, group=None, device=None) -> list:
    """All-gather every rank's Slices (one list per target) and assemble each
    target's graph on every rank (:func:`allgather_csr` per target, tensors on
    `device`: by default this rank's GPU under nccl, the host under gloo).
    Returns (row_ptr, col) numpy arrays per target."""
    import torch
    import torch.distributed as dist
    if device is None:
        nccl = dist.get_backend(group) == "nccl"
        device = torch.device("cuda", torch.cuda.current_device()) if nccl else torch.device("cpu")
    out = []
    for s in my_slices:
        counts = torch.from_numpy(np.diff(s.row_ptr).astype(np.int64)).to(device)
        col = torch.from_numpy(np.ascontiguousarray(s.col, dtype=np.int32)).to(device)
        row_ptr, col_all = allgather_csr(counts, col, n, group)
        out.append((row_ptr.cpu().numpy(), col_all.cpu().numpy()))
    return out
