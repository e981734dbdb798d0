"""Splitting one self-join (or RS-join) across ranks, and gathering the results.

The size-sorted triangle of window pairs (sets ordered by size, ties by id,
the order the library joins in) is cut into contiguous row bands with about
the same number of window pairs each; rank r joins only the pairs whose later
set lies in its band (bmj_options.row_begin / row_end), over the full
collection, which every rank holds.  The bands' pair lists are disjoint and
their union is the full join, so the only exchange is one gather of the pair
lists at the end, merged into the canonical (a, b) order.

An RS-join splits by R: rank r joins a contiguous range of R's sets (about the
same number of window pairs each) with all of S, and its R ids are offset by
the range's start before the same gather.
"""
from __future__ import annotations

import numpy as np


def sorted_sizes(offsets) -> np.ndarray:
    """Set sizes in the join's size order (ties by original id)."""
    sizes = np.diff(np.asarray(offsets, dtype=np.int64))
    return sizes[np.argsort(sizes, kind="stable")]


def row_window_counts(ssz: np.ndarray, p: int, q: int) -> np.ndarray:
    """Window pairs per sorted row i: i - j0(i), j0(i) = first j with q*s_j >= p*s_i."""
    low = -(-(p * ssz) // q)                       # ceil(p*s/q)
    j0 = np.searchsorted(ssz, low, side="left")
    return np.arange(len(ssz), dtype=np.int64) - j0


def band_split(offsets, p: int, q: int, world: int):
    """[(row_begin, row_end)] for each rank: contiguous, covering every row,
    with about the same number of window pairs each."""
    ssz = sorted_sizes(offsets)
    n = len(ssz)
    if world < 1:
        raise ValueError("world must be >= 1")
    w = row_window_counts(ssz, p, q)
    cum = np.concatenate([[0], np.cumsum(w)])
    total = int(cum[-1])
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        cuts.append(int(np.searchsorted(cum, target, side="left")))
    cuts.append(n)
    cuts = np.maximum.accumulate(np.clip(cuts, 0, n))
    return [(int(cuts[r]), int(cuts[r + 1])) for r in range(world)]


def merge_pairs(parts):
    """Union of disjoint pair lists [(a, b), ...] in the canonical (a, b) order."""
    if not parts:
        return np.zeros(0, np.uint32), np.zeros(0, np.uint32)
    a = np.concatenate([np.asarray(x[0], np.uint32) for x in parts])
    b = np.concatenate([np.asarray(x[1], np.uint32) for x in parts])
    order = np.lexsort((b, a))
    return a[order], b[order]


def gather_pairs(a, b, group=None, dst=None):
    """Gather every rank's pair list as fixed-dtype tensors and merge.

    The counts go first (one all_gather of an int64 each); then every rank's
    pairs travel as int64 keys (a << 32 | b), padded to the largest count, in
    one all_gather (dst None: every rank gets the merged list) or one gather
    to rank dst (the others get None).  Tensors live on the CPU for gloo and
    on the current CUDA device for NCCL.  Each rank's list is sorted and the
    bands are disjoint, so the merge is a stable sort of the concatenated runs.
    """
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    dev = (torch.device("cuda", torch.cuda.current_device())
           if dist.get_backend(group) == "nccl" else torch.device("cpu"))
    a = np.asarray(a, np.uint32).astype(np.int64)
    b = np.asarray(b, np.uint32).astype(np.int64)
    mine = torch.from_numpy((a << 32) | b).to(dev)
    cnt = torch.tensor([mine.numel()], dtype=torch.int64, device=dev)
    counts = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(counts, cnt, group=group)
    counts = [int(c.item()) for c in counts]
    m = max(counts) if counts else 0
    if m == 0:
        empty = (np.zeros(0, np.uint32), np.zeros(0, np.uint32))
        return empty if dst is None or rank == dst else None
    padded = torch.zeros(m, dtype=torch.int64, device=dev)
    padded[:mine.numel()] = mine
    if dst is None:
        bufs = [torch.empty(m, dtype=torch.int64, device=dev) for _ in range(world)]
        dist.all_gather(bufs, padded, group=group)
    else:
        bufs = [torch.empty(m, dtype=torch.int64, device=dev) for _ in range(world)] \
            if rank == dst else None
        dist.gather(padded, bufs, dst=dst, group=group)
        if rank != dst:
            return None
    keys = np.concatenate([bufs[r][:counts[r]].cpu().numpy() for r in range(world)])
    keys = np.sort(keys, kind="stable")
    return (keys >> 32).astype(np.uint32), (keys & 0xffffffff).astype(np.uint32)


def sharded_self_join(offsets, tokens, p: int, q: int, rank: int, world: int, **kw):
    """This rank's band of the join through the C ABI (bmj_self_join)."""
    from . import _bmj
    r0, r1 = band_split(offsets.cpu().numpy() if hasattr(offsets, "cpu") else offsets, p, q, world)[rank]
    return _bmj.bmj_self_join(offsets, tokens, p, q, row_begin=r0, row_end=r1, **kw)


def rs_row_windows(r_offsets, s_offsets, p: int, q: int) -> np.ndarray:
    """Window pairs of every set of R (original order) against S, for the Jaccard
    threshold p/q: the sets of S with ceil(p*x/q) <= size <= floor(q*x/p)."""
    rs = np.diff(np.asarray(r_offsets, dtype=np.int64))
    ss = np.sort(np.diff(np.asarray(s_offsets, dtype=np.int64)))
    low = -(-(p * rs) // q)
    high = (q * rs) // p
    return np.searchsorted(ss, high, side="right") - np.searchsorted(ss, low, side="left")


def rs_split(r_offsets, s_offsets, p: int, q: int, world: int):
    """[(r_begin, r_end)] for each rank: contiguous ranges of R's sets (original
    order) covering R, with about the same number of window pairs each."""
    if world < 1:
        raise ValueError("world must be >= 1")
    w = rs_row_windows(r_offsets, s_offsets, p, q)
    n = len(w)
    cum = np.concatenate([[0], np.cumsum(w)])
    cuts = [0] + [int(np.searchsorted(cum, cum[-1] * r / world, side="left")) for r in range(1, world)]
    cuts.append(n)
    cuts = np.maximum.accumulate(np.clip(cuts, 0, n))
    return [(int(cuts[r]), int(cuts[r + 1])) for r in range(world)]


def rs_part(r_offsets, r_tokens, r0: int, r1: int):
    """The sets [r0, r1) of R as a collection of their own (offsets rebased)."""
    off = np.asarray(r_offsets, dtype=np.int64)
    tok = np.asarray(r_tokens)
    return off[r0:r1 + 1] - off[r0], tok[off[r0]:off[r1]]


def sharded_rs_join(r_offsets, r_tokens, s_offsets, s_tokens, p: int, q: int, rank: int, world: int,
                    **kw):
    """This rank's range of R joined with all of S through the C ABI (bmj_rs_join);
    the R ids it returns are ids of the whole R."""
    from . import _bmj
    r0, r1 = rs_split(r_offsets, s_offsets, p, q, world)[rank]
    po, pt = rs_part(r_offsets, r_tokens, r0, r1)
    a, b, st = _bmj.bmj_rs_join(po, pt, s_offsets, s_tokens, p, q, **kw)
    return (np.asarray(a, np.uint32) + np.uint32(r0)), b, st
