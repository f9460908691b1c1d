"""Autotuner for the bin configuration of the plain two-phase path.

The paper fixes its bin ranges by experiment (Sec. 5.7; Tables 4 and 5 try
tables 1x/1.2x/1.5x larger than the largest n_prod of a symbolic bin and
1x/1.5x/2x/3x larger than the largest n_nz of a numeric bin). Here the same
choices, plus two that GB300's 227 KB per block opens up, are searched per
workload by timing the library itself:

- ``ratio``: table size / largest row size of each hash bin, per phase;
- ``cut``: the last hash kernel kept in a phase; larger rows go to the
  shared-memory bitmap kernel (whose cost per row grows with the number of
  columns rather than with the row);
- ``lanes_per_brow`` / ``num_lanes_per_brow``: threads per B row in each
  phase, automatic per row or fixed;
- ``bitmap_unroll``: products each bitmap-kernel thread keeps in flight.

The search is coordinate descent from the defaults; each candidate is timed
with CUDA events over a few whole multiplies. The result is a plain dict
(JSON-serialisable) for ``Handle(config)`` or ``bench.py --config``.
"""

from __future__ import annotations

import json
import math

from . import CSR, Handle, kernel_table

SYM_RATIOS = (1.0, 1.2, 1.5)
NUM_RATIOS = (1.0, 1.5, 2.0, 3.0)


def make_config(sym_ratio=1.2, num_ratio=2.0, sym_cut=None, num_cut=None, lanes=0,
                num_lanes=0, unroll=0) -> dict:
    """A bin configuration: hash kernels 0..cut of each phase with ranges
    floor(table / ratio) (capped at the kernel's capacity), then the bitmap
    kernel for everything larger; threads per B row for each phase."""
    cfg = {"lanes_per_brow": int(lanes), "num_lanes_per_brow": int(num_lanes),
           "bitmap_unroll": int(unroll)}
    for key, phase, ratio, cut in (("sym", 0, sym_ratio, sym_cut), ("num", 1, num_ratio, num_cut)):
        table = kernel_table(phase)
        bitmap = len(table) - 1
        last = bitmap - 1 if cut is None else min(int(cut), bitmap - 1)
        kernels, ranges = [], []
        prev = -1
        for k in range(last + 1):
            tpr, blk, tab, cap = table[k]
            r = min(int(math.floor(tab / ratio)), cap)
            if r <= prev:
                continue
            kernels.append(k)
            ranges.append(r)
            prev = r
        kernels.append(bitmap)
        ranges.append(-1)
        cfg[f"{key}_kernel"] = kernels
        cfg[f"{key}_range"] = ranges
    return cfg


def time_config(A: CSR, B: CSR, cfg: dict, reps: int = 3, warmup: int = 1) -> float:
    """Median milliseconds of one whole multiply with this configuration."""
    import torch
    with Handle(cfg) as h:
        for _ in range(warmup):
            C = h.multiply(A, B)
            del C
        times = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            C = h.multiply(A, B)
            e1.record()
            e1.synchronize()
            del C
            times.append(e0.elapsed_time(e1))
        h.status()
    times.sort()
    return times[len(times) // 2]


def tune(A: CSR, B: CSR, reps: int = 3, log=None) -> tuple[dict, list]:
    """Coordinate descent over (num_cut, num_ratio, sym_cut, sym_ratio,
    lanes). Returns (best configuration, [(params, ms), ...])."""
    nsym = len(kernel_table(0)) - 1
    nnum = len(kernel_table(1)) - 1
    params = {"sym_ratio": 1.2, "num_ratio": 2.0, "sym_cut": nsym - 1, "num_cut": nnum - 1,
              "lanes": 0, "num_lanes": 0, "unroll": 0}
    space = {
        "num_cut": list(range(max(0, nnum - 6), nnum)),
        "num_ratio": list(NUM_RATIOS),
        "sym_cut": list(range(max(0, nsym - 5), nsym)),
        "sym_ratio": list(SYM_RATIOS),
        "lanes": [0, 8, 32],
        "num_lanes": [0, 8, 32],
        "unroll": [0, 8],
    }
    seen = {}

    def measure(p):
        key = json.dumps(p, sort_keys=True)
        if key not in seen:
            seen[key] = time_config(A, B, make_config(**p), reps=reps)
            if log:
                log(f"{p} -> {seen[key]:.3f} ms")
        return seen[key]

    best = measure(params)
    for name in ("num_cut", "num_ratio", "sym_cut", "sym_ratio", "lanes", "num_lanes", "unroll"):
        for v in space[name]:
            cand = dict(params, **{name: v})
            t = measure(cand)
            if t < best:
                best, params = t, cand
    history = [(json.loads(k), v) for k, v in seen.items()]
    return make_config(**params), history


# batch kernel variants (lanes per row, table slots): (8, 64), (16, 128), (32, 256)
BATCH_VARIANTS = 3


def time_batch(b, reps: int = 3, warmup: int = 1) -> float:
    """Median wall-clock milliseconds of one batch run (graph launch through
    the synchronising read of the sizes)."""
    import time

    import torch
    for _ in range(warmup):
        b.run()
        b.sync()
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.run()
        b.sync()
        ts.append((time.perf_counter() - t0) * 1e3)
    ts.sort()
    return ts[len(ts) // 2]


def tune_batch(handle: Handle, As, Bs, b_from, reps: int = 3, log=None) -> tuple[dict, list]:
    """Threads per row, table size (the kernel variant) and rows per work item
    of a batch, by exhaustive timing: every variant whose table holds the
    batch's largest row bound, with 1, 2, 4, 8, 16 or 32 row groups' worth of
    rows per item. Returns ({"variant", "tile_rows", "ms"}, history)."""
    from . import SpgemmError
    from .batch import Batch
    hist = []
    best = None
    for variant in range(BATCH_VARIANTS):
        try:
            with Batch(handle, As, Bs, b_from, variant=variant) as b:
                groups_per_block = 256 // b.info()["lanes_per_row"]
        except SpgemmError as e:
            if e.code == -1:     # this table cannot hold the largest row
                continue
            raise
        for mult in (1, 2, 4, 8, 16, 32):
            tile = groups_per_block * mult
            with Batch(handle, As, Bs, b_from, variant=variant, tile_rows=tile) as b:
                ms = time_batch(b, reps)
            rec = {"variant": variant, "tile_rows": tile, "ms": round(ms, 4)}
            hist.append(rec)
            if log:
                log(rec)
            if best is None or ms < best["ms"]:
                best = rec
    return best, hist
