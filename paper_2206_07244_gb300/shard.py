"""Row sharding of C = A * B over several GPUs (one process per GPU).

Output rows are independent (Sec. 2.1, Eq. 2: row i of C needs only row i
of A and the rows of B it references), so the product shards by contiguous
row slabs with B replicated on every GPU and no data exchanged while
multiplying. The slabs are balanced by the prefix sum of the per-row
intermediate-product counts n_prod (Sec. 2.1.2), the work measure of the
method, not by A's non-zeros: on power-law inputs a few rows hold most of
the products. The one exchange is the offset of each rank's part of C's row
pointer: an all-gather of one int64 (the rank's number of entries) and an
exclusive scan over the ranks. Each rank then runs the row-window calls of
the library (spgemm_symbolic with [row_begin, row_end), spgemm_numeric) on
its slab; stitching C on one rank is optional.

Host logic only (numpy and torch.distributed); the multiply itself runs in
the CUDA library on each rank.
"""

from __future__ import annotations

import numpy as np


def nprod_per_row(arpt, acol, brpt) -> np.ndarray:
    """n_prod of every row of C = A * B: the summed lengths of the B rows
    that row i of A references (int64)."""
    arpt = np.asarray(arpt, dtype=np.int64)
    blen = np.diff(np.asarray(brpt, dtype=np.int64))
    cs = np.zeros(arpt[-1] + 1 if arpt.size else 1, dtype=np.int64)
    if acol.size:
        np.cumsum(blen[np.asarray(acol)], out=cs[1:])
    return cs[arpt[1:]] - cs[arpt[:-1]]


def slab_bounds(nprod: np.ndarray, world: int) -> list[tuple[int, int]]:
    """Contiguous row slabs [r0, r1), one per rank, whose products are as
    equal as contiguous cuts allow: cut r of `world` is the first row at
    which the prefix sum of n_prod reaches r / world of the total. Every row
    belongs to exactly one slab; slabs may be empty when a single row holds
    more than a rank's share."""
    nprod = np.asarray(nprod, dtype=np.int64)
    m = nprod.size
    if world <= 1:
        return [(0, m)]
    csum = np.concatenate([[0], np.cumsum(nprod)])
    total = int(csum[-1])
    cuts = [0]
    for r in range(1, world):
        c = int(np.searchsorted(csum, (total * r) // world, side="left"))
        cuts.append(min(max(c, cuts[-1]), m))
    cuts.append(m)
    return list(zip(cuts[:-1], cuts[1:]))


def exclusive_offsets(counts) -> list[int]:
    """Exclusive prefix of per-rank entry counts: where each rank's entries
    start in the stitched C."""
    out, acc = [], 0
    for c in counts:
        out.append(acc)
        acc += int(c)
    return out


def rpt_offset(local_nnz: int, group=None) -> tuple[int, int]:
    """The single exchange of the sharded product: all-gather every rank's
    int64 number of entries and return (this rank's offset into the
    stitched C, the total). Collective over `group` (the default process
    group when None); works with any backend that supports all_gather of
    int64 tensors (nccl, gloo)."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size(group)
    rank = dist.get_rank(group)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    mine = torch.tensor([int(local_nnz)], dtype=torch.int64, device=dev)
    parts = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(ws)]
    dist.all_gather(parts, mine, group=group)
    counts = [int(p.item()) for p in parts]
    return exclusive_offsets(counts)[rank], sum(counts)


def stitch(parts):
    """C from the ranks' parts, in rank order: parts[r] = (local rpt with
    rows_r + 1 entries starting at 0, col, val). The global row pointer is
    each local one shifted by the rank's offset."""
    offs = exclusive_offsets(int(p[0][-1]) for p in parts)
    rpt = [np.zeros(1, dtype=np.int64)]
    for (lr, _, _), off in zip(parts, offs):
        rpt.append(np.asarray(lr[1:], dtype=np.int64) + off)
    col = np.concatenate([np.asarray(p[1]) for p in parts]) if parts else np.zeros(0, np.int32)
    val = np.concatenate([np.asarray(p[2]) for p in parts]) if parts else np.zeros(0)
    return np.concatenate(rpt), col, val
