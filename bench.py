"""Benchmark: row-wise SpGEMM C = A*A on GB300, GFLOPS = 2 x intermediate
products / second (the paper's metric, Sec. 6), with the HBM-roofline fraction
of the dominant kernel, the CPU oracle as a baseline and an end-to-end number
through the host-buffer C ABI call.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--impl ours|reference] [--no-e2e] [--no-cpu-baseline]
                    [--no-rerun] [--legs all|none|learned|batched|ablation]

Besides the main line: the numeric phase run again over the kept structure
with new values (spgemm_numeric_values), and the legs: learned sizing vs
plain, 512 Galerkin products batched vs plain calls, and one-access vs
read-then-swap hash probes on the 27-point stencil 128^3.

Default workload: R-MAT n = 2^20, average degree 16 (a=.57, b=c=.19), seed 1,
float64 values uniform in [-1, 1] (about 2.09e10 products, 9.7e9 entries in C,
which needs an int64 row pointer). A step is one whole SpGEMM: n_prod, both
binning steps, symbolic, scan, C allocation and numeric. Inputs are resident
in HBM when the timed region starts; A (193 MB) is larger than L2 and every
step writes about 116 GB of C, so nothing stays L2-resident between steps.

Under torchrun (N > 1) each rank computes a contiguous slab of C's rows
(balanced by the prefix sum of the per-row product counts, B replicated);
the ranks exchange one int64 each (their entry counts, the offsets of their
parts of C.rpt); value = all products / the slowest rank's time.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "SpGEMM GFLOPS (2x intermediate products/s)"

WORKLOADS = {
    "rmat20": ("C = A*A, A = R-MAT n=2^20, degree 16 (a=.57,b=.19,c=.19), seed 1, "
               "float64 U[-1,1]", lambda: W.rmat(20, 16, seed=1)),
    "stencil27_128": ("C = A*A, A = 27-point stencil on 128^3, off-diagonal U[0.5,1.5], "
                      "diagonal 27, seed 3", lambda: W.stencil27(128, seed=3)),
    "laplace2d_64": ("C = A*A, A = 5-point Laplacian on 64x64 (4 / -1)",
                     lambda: W.laplacian_2d(64)),
    "rmat18": ("C = A*A, A = R-MAT n=2^18, degree 16, seed 1",
               lambda: W.rmat(18, 16, seed=1)),
    "rmat16": ("C = A*A, A = R-MAT n=2^16, degree 16, seed 1 (small profiling case)",
               lambda: W.rmat(16, 16, seed=1)),
    "blockdiag20": ("C = A*A, A = random block-diagonal n=2^20, 1024 blocks, mean degree 24, seed 7",
                    lambda: W.block_diagonal(1 << 20, 1024, 24.0, seed=7)),
}

SLOT_NAMES = ([f"sym_bin{j}" for j in range(16)] + [f"num_bin{j}" for j in range(16)]
              + ["nprod", "sym_pass1", "sym_pass2", "num_pass1", "num_pass2", "scan",
                 "features", "mlp_sizes", "copy_rows"])
NSLOTS = len(SLOT_NAMES)


# DRAM traffic of the dominant kernel, from an ncu capture of a row window of
# the workload (dram__bytes_read.sum + dram__bytes_write.sum of that launch),
# scaled to a whole launch by the window's share of the kernel's
# intermediate products. Each entry records the hash of the kernel sources at
# capture time; a kernel changed since then reports no traffic.
TRAFFIC_WINDOWED = {
    # ncu dram__bytes_read.sum + dram__bytes_write.sum of the launch for the
    # row window 4096:8192 (--rows 4096:8192, the timed step's launch),
    # taken with the kernel sources whose hash is sources_sha
    ("rmat20", "num_bitmap_kernel"): {"rows": "4096:8192", "dram_bytes": 16860032000,
                                      "window_products": 635646019, "sources_sha": "b8023f6fa11334ec"},
}
KERNEL_SOURCES = ["paper_2206_07244_gb300/csrc/numeric.cu", "paper_2206_07244_gb300/csrc/common.cuh"]


def kernel_sources_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def op_rates(lib):
    """Rates of the operations a product costs, measured now (spgemm_probe):
    float64 fma, shared-memory float64 accumulation by compare-and-swap,
    float64 L2 reductions scattered (one address per lane) and coalesced (a
    warp's 32 lanes on 32 consecutive doubles), and reductions over 1 GB."""
    import ctypes

    import torch
    from paper_2206_07244_gb300 import _abi
    buf = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
    out = {}
    for name, op, hot, it in (("fp64_fma_gops", 0, 0, 8192), ("smem_cas_fma_gops", 1, 0, 32768),
                              ("smem_cas_fma_hot1024_gops", 1, 1024, 8192),
                              ("smem_cas_fma_hot64_gops", 1, 64, 2048),
                              ("smem_atomicadd_f64_gops", 2, 0, 32768),
                              ("l2_red_scattered_gops", 5, 0, 32768), ("l2_red_coalesced_gops", 7, 0, 65536),
                              ("dram_red_scattered_gops", 6, 0, 4096), ("smem_or_u32_gops", 3, 0, 131072),
                              ("smem_cas_i32_gops", 4, 0, 131072)):
        g = ctypes.c_double()
        _abi.check(lib.spgemm_probe(op, hot, it, ctypes.c_void_p(buf.data_ptr()), buf.numel(),
                                    ctypes.byref(g), None), "spgemm_probe")
        out[name] = round(g.value, 2)
    del buf
    torch.cuda.empty_cache()
    out["what"] = ("one 1024-thread block per SM, uniform random addresses unless hotN (N distinct "
                   "addresses per block; fma: 8 independent chains per thread); Gop/s")
    return out


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def row_slab(A, rank, ws):
    """Contiguous rows of C = A*A for this rank, balanced by the prefix sum
    of the per-row intermediate products (the library's row sharding)."""
    if ws == 1:
        return 0, A.rows
    from paper_2206_07244_gb300 import shard
    return shard.slab_bounds(shard.nprod_per_row(A.rpt, A.col, A.rpt), ws)[rank]


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"opsparse_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[4:]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        pmax = max(r[2] for r in rows)
        load = [r for r in rows if r[2] >= 0.5 * pmax] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in load for i, v in enumerate(r[3][1:5])
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "samples_under_load": len(load),
                "power_w_max": pmax}


def compulsory_bytes(A, r0, r1, nnzC):
    """Bytes a row window of C = A*A must move at least (the roofline model):
    A's rows, the distinct B (= A) rows they reference, and C."""
    rpt = A.rpt.astype(np.int64)
    a_bytes = 4 * (r1 - r0 + 1) + 12 * int(rpt[r1] - rpt[r0])
    ks = np.unique(A.col[rpt[r0]:rpt[r1]])
    lens = rpt[ks + 1] - rpt[ks]
    b_bytes = 8 * ks.size + 12 * int(lens.sum())
    c_bytes = 8 * (r1 - r0 + 1) + 12 * int(nnzC)
    return a_bytes + b_bytes + c_bytes, b_bytes


def cpu_baseline(A, target_products=1.5e9):
    """The oracle as it stands, on a strided row sample of the same workload."""
    import oracle
    nprod = oracle.nprod(A, A)
    total = int(nprod.sum())
    stride = max(1, int(np.ceil(total / target_products)))
    rows = np.arange(0, A.rows, stride)
    rpt = A.rpt.astype(np.int64)
    lens = rpt[rows + 1] - rpt[rows]
    srpt = np.zeros(rows.size + 1, dtype=np.int64)
    np.cumsum(lens, out=srpt[1:])
    idx = np.concatenate([np.arange(rpt[r], rpt[r + 1]) for r in rows]) if rows.size else np.zeros(0, np.int64)
    As = W.Csr(rows.size, A.cols, srpt, A.col[idx], A.val[idx])
    sprod = int(nprod[rows].sum())
    threads = oracle.max_threads()
    t = time.perf_counter()
    oracle.spgemm(As, A, threads=threads, with_abs=False)
    dt = time.perf_counter() - t
    return {"value": round(2.0 * sprod / dt / 1e9, 4), "unit": "GFLOPS", "cores": threads,
            "kind": "oracle", "seconds": round(dt, 3), "workload_fraction": round(sprod / total, 6) if total else 1.0,
            "sample": f"every {stride}th row of A ({rows.size} rows, {sprod} products, "
                      f"{sprod / total:.3f} of the workload); full two-phase oracle (count, "
                      f"dense-accumulator multiply, sort) on {threads} threads"}


def _time_multiply(h, dA, r0, r1, reps=3):
    import torch
    for _ in range(3):   # warm-up; in learned mode the load feedback settles here
        h.symbolic(dA, dA, r0, r1)
        C = h.numeric(dA, dA)
        del C
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        h.symbolic(dA, dA, r0, r1)
        C = h.numeric(dA, dA)
        e1.record()
        e1.synchronize()
        del C
        ts.append(e0.elapsed_time(e1))
    h.status()
    return float(np.median(ts))


def _serial_breakdown(h, dA, r0, r1):
    """Per-kernel milliseconds of one multiply with every kernel on one
    stream (untimed step; events around each launch)."""
    import ctypes

    from paper_2206_07244_gb300 import _abi
    lib = _abi.lib()
    ms_arr = (ctypes.c_double * NSLOTS)()
    ln_arr = (ctypes.c_int64 * NSLOTS)()
    _abi.check(lib.spgemm_set_timing(h._h, 2), "spgemm_set_timing")
    _abi.check(lib.spgemm_kernel_times(h._h, ms_arr, ln_arr, NSLOTS, 1), "spgemm_kernel_times")
    h.symbolic(dA, dA, r0, r1)
    C = h.numeric(dA, dA)
    del C
    _abi.check(lib.spgemm_kernel_times(h._h, ms_arr, ln_arr, NSLOTS, 1), "spgemm_kernel_times")
    lib.spgemm_set_timing(h._h, 0)
    return {SLOT_NAMES[i]: round(ms_arr[i], 3) for i in range(NSLOTS) if ms_arr[i] > 0}


def learned_eval(workload_name, A, r0, r1):
    """Plain vs learned sizing (trained weights) vs the n_prod upper bound
    (a predictor that over-predicts every row) on rows [r0, r1) of A*A."""
    import paper_2206_07244_gb300 as ops
    from paper_2206_07244_gb300 import learned
    man = json.load(open(learned.MANIFEST))
    theta = np.load(learned.WEIGHTS)
    dA = ops.CSR.from_workload(A)
    out = {"workload": workload_name, "rows": [int(r0), int(r1)], "margin": man["margin"],
           "val_mae_log1p": round(man["val_mae_log1p"], 4)}
    with ops.Handle() as h:
        t_plain = _time_multiply(h, dA, r0, r1)
        st = h.stats()
        nprod = st["total_nprod"]
        out["nnzC"] = st["total_nnz"]
        out["plain_kernel_ms_serial"] = _serial_breakdown(h, dA, r0, r1)
        h.set_predictor(theta, man["margin"])
        h.set_mode("learned")
        t_learned = _time_multiply(h, dA, r0, r1)
        out["learned_stats"] = h.learned_stats()
        out["learned_kernel_ms_serial"] = _serial_breakdown(h, dA, r0, r1)
        big = np.zeros_like(theta)
        big[-1] = 30.0
        h.set_predictor(big, 0.0)
        t_bound = _time_multiply(h, dA, r0, r1)
    g = lambda t: round(2.0 * nprod / (t / 1e3) / 1e9, 3)
    out.update({"plain_ms": round(t_plain, 3), "learned_ms": round(t_learned, 3),
                "nprod_bound_ms": round(t_bound, 3), "plain_gflops": g(t_plain),
                "learned_gflops": g(t_learned), "nprod_bound_gflops": g(t_bound),
                "learned_over_plain": round(t_plain / t_learned, 4),
                "learned_over_nprod_bound": round(t_bound / t_learned, 4)})
    return out


def _product_bytes(arpt, acol, brpt, b_rpt_bytes, rows, nnzC):
    """Compulsory bytes of one product: A's rows, the distinct B rows they
    reference, and C (int64 row pointer)."""
    a_bytes = arpt.itemsize * (rows + 1) + 12 * int(arpt[-1])
    ks = np.unique(acol)
    b_bytes = b_rpt_bytes * ks.size + 12 * int((brpt[ks + 1] - brpt[ks]).sum())
    return a_bytes + b_bytes + 8 * (rows + 1) + 12 * int(nnzC)


def batched_eval(count=512, seed=0, reps=3, tune=True):
    """Multigrid Galerkin products P^T (A P) for `count` seeded grid sides
    uniform in [8, 48] (A the 7-point Laplacian, P the 2x2x2 aggregation
    prolongator); every product has its own device copy of its inputs.
    Plain: 2 * count calls through the handle (A P, then P^T (A P)). Batched:
    the same products in one persistent launch under a CUDA graph (default
    and autotuned variant / rows per item). Times are wall-clock per whole
    batch, from the first launch to the sizes on the host; the batch's
    results are compared with the plain path's (exact: integer values)."""
    import torch

    import paper_2206_07244_gb300 as ops
    from paper_2206_07244_gb300 import autotune
    from paper_2206_07244_gb300.batch import Batch, galerkin_batch
    sides = W.galerkin_sides(count, seed=seed)
    peak, peak_kind = peaks()
    host = {int(s): W.galerkin_problem(int(s)) for s in np.unique(sides)}
    out = {"workload": f"{count} Galerkin products P^T(A P), A = 7-point Laplacian on s^3, "
                       f"s uniform in [8, 48] (seed {seed}), P = 2x2x2 aggregation; "
                       "inputs copied per product",
           "sides_sum_rows": int(sum(int(s) ** 3 for s in sides))}
    with ops.Handle() as h:
        As, Bs, dep, inputs = galerkin_batch(h, sides, share_inputs=False)

        def plain_once(keep=False):
            kept = []
            for A, P, PT in inputs:
                C1 = h.multiply(A, P)
                C2 = h.multiply(PT, C1)
                if keep:
                    kept.append((C1.rpt.cpu().numpy(), C1.nnz, C2))
                del C1
            return kept

        kept = plain_once(keep=True)
        h.status()
        nprod = 0
        bytes_ = 0
        for i, s in enumerate(sides):
            A, P, PT = host[int(s)]
            rpt1, nnz1, C2 = kept[i]
            nprod += int(np.diff(P.rpt)[A.col].sum()) + int(np.diff(rpt1)[PT.col].sum())
            bytes_ += _product_bytes(A.rpt, A.col, P.rpt.astype(np.int64), 4, A.rows, nnz1)
            bytes_ += _product_bytes(PT.rpt, PT.col, rpt1, 8, PT.rows, C2.nnz)
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plain_once()
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
        t_plain = float(np.median(ts))
        with Batch(h, As, Bs, dep) as b:
            t_batch = autotune.time_batch(b, reps)
            info = b.info()
            match = True
            for i in range(count):
                C = b.result(count + i)
                ref = kept[i][2]
                match &= (C.nnz == ref.nnz and torch.equal(C.rpt, ref.rpt) and torch.equal(C.col, ref.col)
                          and torch.equal(C.val, ref.val))
        best = hist = None
        if tune:
            best, hist = autotune.tune_batch(h, As, Bs, dep, reps=reps)
            with Batch(h, As, Bs, dep, variant=best["variant"], tile_rows=best["tile_rows"]) as b:
                t_tuned = autotune.time_batch(b, reps)
    g = lambda t: round(2.0 * nprod / (t / 1e3) / 1e9, 3)
    bw = lambda t: round(bytes_ / (t / 1e3) / 1e9, 1)
    out.update({"nprod": nprod, "compulsory_bytes": bytes_, "plain_calls": 2 * count,
                "plain_ms": round(t_plain, 3), "batched_ms": round(t_batch, 3),
                "plain_gflops": g(t_plain), "batched_gflops": g(t_batch),
                "batched_over_plain": round(t_plain / t_batch, 3),
                "batched_gbs": bw(t_batch), "batched_hbm_frac": round(bw(t_batch) / peak, 4),
                "peak_gbs": peak, "peak_kind": peak_kind, "batch_info": info,
                "batch_matches_plain": bool(match)})
    if best is not None:
        out.update({"tuned": best, "tuned_ms": round(t_tuned, 3), "tuned_gflops": g(t_tuned),
                    "tuned_gbs": bw(t_tuned), "tuned_hbm_frac": round(bw(t_tuned) / peak, 4),
                    "tuned_over_plain": round(t_plain / t_tuned, 3), "tune_trials": len(hist)})
    return out


def hash_ablation_eval(reps=3):
    """The paper's hashing comparison (Sec. 6): one atomicCAS per probe
    (Algorithms 4-5, hash_access = 0) against a read of the slot before the
    compare-and-swap (hash_access = 1), everything else the same, on the
    27-point stencil 128^3, whose rows all take hash kernels. Kernel times of
    the symbolic and numeric hash bins, serialised on one stream."""
    import ctypes
    import torch
    import paper_2206_07244_gb300 as ops
    from paper_2206_07244_gb300 import _abi
    lib = _abi.lib()
    S = W.stencil27(128, seed=3)
    dS = ops.CSR.from_workload(S)
    del S
    res = {}
    for mode in (0, 1):
        h = ops.Handle()
        C = h.multiply(dS, dS)        # the default bins for this B
        del C
        cfg = h.get_config()
        cfg["hash_access"] = mode
        h.set_config(cfg)
        for _ in range(2):
            C = h.multiply(dS, dS)
            del C
        ms = (ctypes.c_double * NSLOTS)()
        ln = (ctypes.c_int64 * NSLOTS)()
        _abi.check(lib.spgemm_set_timing(h._h, 2), "spgemm_set_timing")
        _abi.check(lib.spgemm_kernel_times(h._h, ms, ln, NSLOTS, 1), "spgemm_kernel_times")
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            C = h.multiply(dS, dS)
            del C
        e1.record(s)
        h.status()
        _abi.check(lib.spgemm_kernel_times(h._h, ms, ln, NSLOTS, 1), "spgemm_kernel_times")
        lib.spgemm_set_timing(h._h, 0)
        nbs, nbn = len(ops.kernel_table(0)) - 1, len(ops.kernel_table(1)) - 1
        sym = sum(ms[j] for j, k in enumerate(cfg["sym_kernel"]) if k != nbs) / reps
        num = sum(ms[16 + j] for j, k in enumerate(cfg["num_kernel"]) if k != nbn) / reps
        res[mode] = {"sym_hash_ms": round(sym, 3), "num_hash_ms": round(num, 3),
                     "multiply_ms_serial": round(e0.elapsed_time(e1) / reps, 3)}
        h.close()
    return {"workload": "C = A*A, A = 27-point stencil 128^3 (every row in a hash bin)",
            "single_access": res[0], "multi_access": res[1],
            "sym_speedup_single_over_multi": round(res[1]["sym_hash_ms"] / max(res[0]["sym_hash_ms"], 1e-9), 3),
            "num_speedup_single_over_multi": round(res[1]["num_hash_ms"] / max(res[0]["num_hash_ms"], 1e-9), 3)}


def _kernel_bytes(bins_sym, bins_num, k, b_bytes):
    """Algorithmic bytes of bin kernel k (slot index) in one multiply: its
    A rows, the referenced B rows (b_bytes, the whole product's) and its
    output (C rows for a numeric bin, 16 bytes per row for a symbolic one)."""
    phase, j = divmod(k, 16)
    bs = list(bins_num if phase else bins_sym)
    rows_j, size_j, nnza_j = bs[j], bs[16 + j], bs[32 + j]
    return 8 * rows_j + 12 * nnza_j + b_bytes + ((16 * rows_j + 12 * size_j) if phase else 16 * rows_j)


def nprod_rows(A):
    rpt = A.rpt.astype(np.int64)
    cs = np.concatenate([[0], np.cumsum(np.diff(rpt)[A.col])])
    return cs[rpt[1:]] - cs[rpt[:-1]]


def slabs_by_products(A, per_slab):
    """Contiguous row slabs of A*A with about per_slab products each."""
    csum = np.concatenate([[0], np.cumsum(nprod_rows(A))])
    cuts = [0]
    while cuts[-1] < A.rows:
        r = int(np.searchsorted(csum, csum[cuts[-1]] + per_slab, side="right")) - 1
        cuts.append(min(A.rows, max(r, cuts[-1] + 1)))
    return list(zip(cuts[:-1], cuts[1:]))


def config_line(name, A, slabs, cfg=None, learned_theta=None, margin=0.0, warm=1, note=None):
    """One whole multiply of A*A as a sequence of row slabs (one slab = the
    whole matrix when it fits): CUDA-event time of a pass over all slabs after
    `warm` untimed passes, GFLOPS, the dominant kernel (longest summed over
    the slabs with every kernel serialised on one stream, one more pass) and
    its fraction of the measured copy bandwidth, and the whole pass's
    compulsory-byte fraction."""
    import ctypes

    import torch

    import paper_2206_07244_gb300 as ops
    from paper_2206_07244_gb300 import _abi
    lib = _abi.lib()
    peak, peak_kind = peaks()
    dA = ops.CSR.from_workload(A)
    h = ops.Handle(cfg)
    if learned_theta is not None:
        h.set_predictor(learned_theta, margin)
        h.set_mode("learned")

    def one_pass():
        for r0, r1 in slabs:
            h.symbolic(dA, dA, r0, r1)
            C = h.numeric(dA, dA)
            del C

    for _ in range(warm):
        one_pass()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    one_pass()
    e1.record(s)
    h.status()
    ms = e0.elapsed_time(e1)
    # serialised per-kernel times and bin statistics, summed over the slabs
    ms_arr = (ctypes.c_double * NSLOTS)()
    ln_arr = (ctypes.c_int64 * NSLOTS)()
    _abi.check(lib.spgemm_set_timing(h._h, 2), "spgemm_set_timing")
    _abi.check(lib.spgemm_kernel_times(h._h, ms_arr, ln_arr, NSLOTS, 1), "spgemm_kernel_times")
    nprod = nnz = 0
    kbytes = {}
    total_bytes = 0
    slot_ms = np.zeros(NSLOTS)
    for r0, r1 in slabs:
        h.symbolic(dA, dA, r0, r1)
        C = h.numeric(dA, dA)
        del C
        _abi.check(lib.spgemm_kernel_times(h._h, ms_arr, ln_arr, NSLOTS, 1), "spgemm_kernel_times")
        slot_ms += np.array(list(ms_arr))
        st = h.stats()
        nprod += st["total_nprod"]
        nnz += st["total_nnz"]
        bins_sym = (ctypes.c_int64 * 48)()
        bins_num = (ctypes.c_int64 * 48)()
        lib.spgemm_bin_stats(h._h, 0, bins_sym, 48)
        lib.spgemm_bin_stats(h._h, 1, bins_num, 48)
        tb, b_bytes = compulsory_bytes(A, r0, r1, st["total_nnz"])
        total_bytes += tb
        for k in range(32):
            kbytes[k] = kbytes.get(k, 0) + _kernel_bytes(bins_sym, bins_num, k, b_bytes)
    lib.spgemm_set_timing(h._h, 0)
    lstats = h.learned_stats() if learned_theta is not None else None
    h.close()
    del dA
    torch.cuda.empty_cache()
    k = int(np.argmax(slot_ms[:32]))
    kb = kbytes[k]
    kgbs = kb / (slot_ms[k] / 1e3) / 1e9
    wgbs = total_bytes / (ms / 1e3) / 1e9
    out = {"config": name, "slabs": len(slabs), "ms": round(ms, 3), "nprod": int(nprod), "nnzC": int(nnz),
           "gflops": round(2.0 * nprod / (ms / 1e3) / 1e9, 3),
           "dominant_kernel": SLOT_NAMES[k], "dominant_kernel_ms_serial": round(float(slot_ms[k]), 3),
           "dominant_kernel_share_serial": round(float(slot_ms[k] / max(slot_ms[:38].sum(), 1e-9)), 4),
           "dominant_kernel_gbs": round(kgbs, 2), "dominant_kernel_frac": round(kgbs / peak, 4),
           "whole_step_gbs": round(wgbs, 2), "whole_step_frac": round(wgbs / peak, 4),
           "peak_gbs": peak, "peak_kind": f"{peak_kind} copy bandwidth",
           "kernel_ms_serial": {SLOT_NAMES[i]: round(float(slot_ms[i]), 3)
                                for i in range(NSLOTS) if slot_ms[i] > 0}}
    if lstats is not None:
        out["learned_stats"] = lstats
    if note:
        out["note"] = note
    return out


def configs_eval():
    """One line per workload configuration besides the main one (the
    batched leg covers the Galerkin batch): the 5-point Laplacian 64x64, the
    27-point stencil 128^3 with the default and the autotuned bins, and the
    held-out R-MAT n=2^21, degree 32, whole, in row slabs, plain and learned."""
    import torch

    import paper_2206_07244_gb300 as ops
    from paper_2206_07244_gb300 import autotune, learned
    lines = []
    L = W.laplacian_2d(64)
    lines.append(config_line("5-point Laplacian 64x64 (n=4096)", L, [(0, L.rows)], warm=3,
                             note="latency-bound: 100,104 products; the fraction is reported, not meaningful"))
    S = W.stencil27(128, seed=3)
    lines.append(config_line("27-point stencil 128^3, default bins", S, [(0, S.rows)], warm=3))
    dS = ops.CSR.from_workload(S)
    best, hist = autotune.tune(dS, dS, reps=2)
    del dS
    torch.cuda.empty_cache()
    tuned = config_line("27-point stencil 128^3, autotuned bins", S, [(0, S.rows)], cfg=best, warm=3)
    tuned["tuned_config"] = best
    tuned["trials"] = len(hist)
    tuned["tuned_over_default"] = round(lines[-1]["ms"] / tuned["ms"], 4)
    lines.append(tuned)
    del S
    R = W.rmat(21, 32, seed=2021)
    slabs = slabs_by_products(R, 1.5e9)
    man = json.load(open(learned.MANIFEST))
    theta = np.load(learned.WEIGHTS)
    plain = config_line("held-out R-MAT n=2^21, degree 32, seed 2021, whole matrix, plain", R, slabs, warm=1)
    lines.append(plain)
    lrn = config_line("held-out R-MAT n=2^21, degree 32, seed 2021, whole matrix, learned sizing", R, slabs,
                      learned_theta=theta, margin=man["margin"], warm=3)
    lrn["learned_over_plain"] = round(plain["ms"] / lrn["ms"], 4)
    # the learned path does not count products; the multiply is the same
    lrn["nprod"] = plain["nprod"]
    lrn["gflops"] = round(2.0 * plain["nprod"] / (lrn["ms"] / 1e3) / 1e9, 3)
    lines.append(lrn)
    return lines


def pick_slab(A, budget_entries):
    """A contiguous row slab of A*A, starting at row A.rows/2, whose C has at
    most budget_entries entries (sized with the library's symbolic phase)."""
    import paper_2206_07244_gb300 as ops
    dA = ops.CSR.from_workload(A)
    r0 = A.rows // 2
    r1 = A.rows
    with ops.Handle() as h:
        while r1 - r0 > 1024:
            nnz = h.symbolic(dA, dA, r0, r1)
            if nnz <= budget_entries:
                break
            r1 = r0 + (r1 - r0) // 2
    return r0, r1


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    desc, gen = WORKLOADS[args.workload]
    A = gen()
    import oracle
    vals = []
    info = None
    for i in range(args.warmup + args.steps):
        info = cpu_baseline(A, target_products=args.ref_products)
        if i >= args.warmup:
            vals.append(info["value"])
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GFLOPS",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(info["seconds"] * 1000, 2), "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc},
            # a step is the bounded sample; the whole workload at the same rate
            "ms_per_step_is": "the sample's time (a fraction of the workload's products)",
            "workload_fraction": info["workload_fraction"],
            "ms_whole_workload_at_this_rate": round(info["seconds"] * 1000 / max(info["workload_fraction"], 1e-6), 1),
            "cpu_baseline": {"value": round(v, 4), "unit": "GFLOPS", "cores": info["cores"],
                             "kind": "oracle", "sample": info["sample"]},
            "e2e": {"value": round(v, 4), "unit": "GFLOPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="rmat20", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-rerun", action="store_true",
                    help="skip the numeric-only re-run over the kept structure")
    ap.add_argument("--ref-products", type=float, default=1.5e9)
    ap.add_argument("--config", default=None, help="bin configuration JSON file")
    ap.add_argument("--autotune", action="store_true",
                    help="also tune the bin configuration and time plain vs tuned")
    ap.add_argument("--save-config", default=None)
    ap.add_argument("--rows", default=None,
                    help="R0:R1 — measure only rows [R0, R1) of C (single GPU; for profiling "
                         "a window of a workload too large to capture whole)")
    ap.add_argument("--window-lists", type=int, default=None,
                    help="set the numeric bitmap kernel's window_lists option on top of the "
                         "configuration in use (0 = whole-row pass 2)")
    ap.add_argument("--legs", default="all",
                    choices=["all", "none", "learned", "batched", "ablation", "peaks", "configs"],
                    help="extra comparisons after the main line: learned sizing vs plain "
                         "(trained weights), 512 Galerkin products plain vs batched, "
                         "single- vs multi-access hash probes, the operation-rate probes, and "
                         "one line per other workload configuration")
    args = ap.parse_args()
    args.learned = args.legs in ("all", "learned")
    args.batched = args.legs in ("all", "batched")
    args.ablation = args.legs in ("all", "ablation")
    args.peaks = args.legs in ("all", "peaks")
    args.configs = args.legs in ("all", "configs")
    if args.warmup < 3 and args.impl == "ours" and not os.environ.get("BENCH_ALLOW_SHORT"):
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2206_07244_gb300 as ops
    from paper_2206_07244_gb300 import _abi

    desc, gen = WORKLOADS[args.workload]
    A = gen()
    r0, r1 = row_slab(A, rank, ws)
    if args.rows:
        if ws > 1:
            raise SystemExit("--rows is for one GPU")
        r0, r1 = (int(x) for x in args.rows.split(":"))
    dA = ops.CSR.from_workload(A, device=f"cuda:{local}")
    cfg = json.load(open(args.config)) if args.config else None
    h = ops.Handle(cfg)
    if args.window_lists is not None:
        # the configuration the handle uses for this B (the default one adapts
        # its bins to B's columns at every symbolic call), with the option set
        h.symbolic(dA, dA, r0, min(r1, r0 + 1))
        C = h.numeric(dA, dA)
        del C
        cfg = h.get_config()
        cfg["window_lists"] = args.window_lists
        h.set_config(cfg)
    lib = _abi.lib()
    import ctypes

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def step():
        h.symbolic(dA, dA, r0, r1)
        C = h.numeric(dA, dA)
        return C

    for _ in range(args.warmup):
        C = step()
        del C
    h.status()
    stats = h.stats()
    nnzC_slab = stats["total_nnz"]
    nprod_slab = stats["total_nprod"]

    _abi.check(lib.spgemm_set_timing(h._h, 1), "spgemm_set_timing")
    ms_arr = (ctypes.c_double * NSLOTS)()
    ln_arr = (ctypes.c_int64 * NSLOTS)()
    _abi.check(lib.spgemm_kernel_times(h._h, ms_arr, ln_arr, NSLOTS, 1), "spgemm_kernel_times")

    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            C = step()
            del C
        ev1.record(stream)
        barrier()
    h.status()
    ms = ev0.elapsed_time(ev1)
    _abi.check(lib.spgemm_kernel_times(h._h, ms_arr, ln_arr, NSLOTS, 1), "spgemm_kernel_times")
    kms = list(ms_arr)
    kln = list(ln_arr)
    # Bins of one phase run concurrently on side streams, so a small bin's
    # events also cover time spent waiting for SMs. Two extra, untimed steps
    # with the bins serialised on one stream give each kernel's own duration;
    # the dominant kernel is the longest of those.
    _abi.check(lib.spgemm_set_timing(h._h, 2), "spgemm_set_timing")
    for _ in range(2):
        C = step()
        del C
    _abi.check(lib.spgemm_kernel_times(h._h, ms_arr, ln_arr, NSLOTS, 1), "spgemm_kernel_times")
    lib.spgemm_set_timing(h._h, 0)
    sms_ = list(ms_arr)
    sln = list(ln_arr)
    serial = {SLOT_NAMES[i]: round(sms_[i] / max(sln[i], 1), 3) for i in range(len(sms_)) if sms_[i] > 0}
    ms_max = ms
    nprod_all = nprod_slab
    nnz_all = nnzC_slab
    rank_offset = 0
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
        p = torch.tensor([nprod_slab], dtype=torch.int64, device="cuda")
        dist.all_reduce(p)
        nprod_all = int(p.item())
        # the one exchange of the sharded product: every rank's entry count,
        # so that its part of C.rpt gets its global offset
        from paper_2206_07244_gb300 import shard
        rank_offset, nnz_all = shard.rpt_offset(nnzC_slab)
    value = 2.0 * nprod_all * args.steps / (ms_max / 1e3) / 1e9

    # dominant kernel (longest in the serialised pass) and its roofline,
    # from its live launches in the timed region
    k = int(np.argmax(sms_))
    bins_sym = (ctypes.c_int64 * 48)()
    bins_num = (ctypes.c_int64 * 48)()
    lib.spgemm_bin_stats(h._h, 0, bins_sym, 48)
    lib.spgemm_bin_stats(h._h, 1, bins_num, 48)
    rpt64 = A.rpt.astype(np.int64)
    total_bytes, b_bytes = compulsory_bytes(A, r0, r1, nnzC_slab)
    if k < 32:
        phase, j = divmod(k, 16)
        bs = list(bins_num if phase else bins_sym)
        rows_j, size_j, nnza_j = bs[j], bs[16 + j], bs[32 + j]
        a_b = 8 * rows_j + 12 * nnza_j
        out_b = (16 * rows_j + 12 * size_j) if phase else 16 * rows_j
        algo = a_b + b_bytes + out_b
        algo_desc = (f"{'numeric' if phase else 'symbolic'} bin {j}: {rows_j} rows, "
                     f"{nnza_j} A entries, {'n_nz' if phase else 'n_prod'} {size_j}; bytes = A rows "
                     f"(12/entry + 8/row) + referenced B rows + "
                     f"{'C rows (12/entry + 16/row)' if phase else 'n_nz out (16/row)'}")
    else:
        algo = total_bytes
        algo_desc = "whole product (A + referenced B + C)"
    launches = max(kln[k], 1)
    avg_ms = kms[k] / launches
    peak, peak_kind = peaks()
    achieved = algo / (avg_ms / 1e3) / 1e9
    # intermediate products of the dominant kernel's launch (the rows of its
    # bin), from one more step's row sizes: the units the operation-rate
    # ceilings count
    is_num_bitmap = 16 <= k < 32 and k - 16 == len(h.get_config()["num_kernel"]) - 1
    kernel_products = None
    phases = None
    if is_num_bitmap:
        # the same untimed step with the kernel's phase clocks on: SM clock
        # cycles of each phase summed over the launch's blocks
        h.set_phase_clocks(True)
        C = step()
        clk_ph = h.bitmap_phase_clocks(reset=True)
        h.set_phase_clocks(False)
        nnz_row = np.diff(C.rpt.cpu().numpy())
        del C
        n_sm = torch.cuda.get_device_properties(0).multi_processor_count
        tot = max(sum(clk_ph.values()), 1)
        phases = {"sm_cycles": clk_ph, "frac": {k: round(v / tot, 4) for k, v in clk_ph.items()},
                  "mean_sm_cycles_per_launch": int(tot / n_sm),
                  "note": "one untimed step with a block barrier ending each phase; thread 0 of every "
                          "block adds its SM clock cycles per phase"}
        cut = h.get_config()["num_range"][-2] if len(h.get_config()["num_range"]) > 1 else -1
        cs = np.concatenate([[0], np.cumsum(np.diff(rpt64)[A.col])])
        row_np = cs[rpt64[1:]] - cs[rpt64[:-1]]
        kernel_products = int(row_np[r0:r1][nnz_row > cut].sum())
    # DRAM traffic of this launch, scaled from a windowed capture of the same
    # kernel sources, workload and configuration (default, whole matrix, 1 GPU)
    traffic = traffic_src = None
    tw = TRAFFIC_WINDOWED.get((args.workload, "num_bitmap_kernel"))
    if is_num_bitmap and tw and kernel_products and ws == 1 and args.rows is None \
            and not args.window_lists and args.config is None and tw["sources_sha"] == kernel_sources_sha():
        scale = kernel_products / tw["window_products"]
        traffic = int(tw["dram_bytes"] * scale)
        traffic_src = (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of the launch for rows "
                       f"{tw['rows']} ({tw['dram_bytes']} bytes, {tw['window_products']} products), "
                       f"scaled by products x{scale:.2f}")
    rates = op_rates(lib) if args.peaks and rank == 0 else None
    roofline = {"bound": "hbm", "kernel": SLOT_NAMES[k], "achieved": round(achieved, 2),
                "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": traffic, "traffic_source": traffic_src,
                "traffic_over_algorithmic": round(traffic / algo, 3) if traffic else None,
                "peak_kind": f"{peak_kind} copy bandwidth",
                "algorithmic_bytes_per_launch": int(algo), "avg_launch_ms": round(avg_ms, 4),
                "serial_launch_ms": round(sms_[k] / max(sln[k], 1), 4),
                "bytes_model": algo_desc}
    if kernel_products:
        # beside the memory roofline: every product costs one float64
        # multiply(-add) and one scattered float64 accumulation
        prate = kernel_products / (avg_ms / 1e3) / 1e9
        roofline["products_per_launch"] = kernel_products
        roofline["products_gops"] = round(prate, 2)
        if rates:
            roofline["atomic_frac"] = round(prate / rates["l2_red_scattered_gops"], 4)
            roofline["atomic_peak_gops"] = rates["l2_red_scattered_gops"]
            roofline["fp64_frac"] = round(prate / rates["fp64_fma_gops"], 4)
            roofline["fp64_peak_gops"] = rates["fp64_fma_gops"]
    if phases:
        roofline["phases"] = phases
    whole = {"bytes_per_step": int(total_bytes),
             "achieved_gbs": round(total_bytes / (ms / args.steps / 1e3) / 1e9, 2),
             "frac": round(total_bytes / (ms / args.steps / 1e3) / 1e9 / peak, 4)}
    breakdown = {SLOT_NAMES[i]: round(kms[i] / args.steps, 3) for i in range(len(kms)) if kms[i] > 0}
    gpu_launches = int(sum(kln) + kln[37])   # the scan slot covers two kernels

    bins = {"sym_rows": list(bins_sym)[:16], "sym_nprod": list(bins_sym)[16:32],
            "num_rows": list(bins_num)[:16], "num_nnz": list(bins_num)[16:32]}
    cfg_used = h.get_config()

    tuned = None
    if args.autotune and rank == 0:
        from paper_2206_07244_gb300 import autotune
        best, hist = autotune.tune(dA, dA, reps=2)
        t_best = autotune.time_config(dA, dA, best, reps=3)
        t_plain = autotune.time_config(dA, dA, None or cfg_used, reps=3)
        tuned = {"plain_ms": round(t_plain, 3), "tuned_ms": round(t_best, 3),
                 "plain_gflops": round(2.0 * nprod_slab / (t_plain / 1e3) / 1e9, 3),
                 "tuned_gflops": round(2.0 * nprod_slab / (t_best / 1e3) / 1e9, 3),
                 "config": best, "trials": len(hist)}
        if args.save_config:
            json.dump(best, open(args.save_config, "w"))

    # numeric phase again over the kept structure, with new values of A (the
    # repeated products of an iterative setup): only the numeric kernels run
    rerun = None
    if not args.no_rerun:
        C = step()
        g = torch.Generator(device=dA.val.device)
        g.manual_seed(5)
        dA2 = ops.CSR(dA.rows, dA.cols, dA.rpt, dA.col,
                      torch.rand(dA.nnz, dtype=torch.float64, device=dA.val.device, generator=g) * 2 - 1)
        h.numeric_values(dA2, dA2, C)   # warm-up
        reps = 3
        barrier()
        ev0.record(stream)
        for _ in range(reps):
            h.numeric_values(dA2, dA2, C)
        ev1.record(stream)
        barrier()
        h.status()
        rms = ev0.elapsed_time(ev1) / reps
        rerun = {"ms": round(rms, 3), "gflops": round(2.0 * nprod_slab / (rms / 1e3) / 1e9, 3),
                 "full_step_ms": round(ms / args.steps, 3),
                 "speedup_over_full_step": round(ms / args.steps / rms, 3),
                 "reps": reps, "what": "spgemm_numeric_values: new A values, same structure"}
        del C, dA2

    # the device-resident handle and the C blocks cached by torch are given
    # back before the other legs, which start from a clean allocator, as a
    # fresh process would
    h.close()
    del dA
    torch.cuda.empty_cache()

    e2e = None
    if not args.no_e2e and rank == 0:
        e2e = run_e2e(A, lib, args.e2e_steps, nprod_slab if ws == 1 else None)
        torch.cuda.empty_cache()

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and ws == 1:
        cpu = cpu_baseline(A)

    learned_legs = batched = ablation = configs = None
    if args.configs and rank == 0:
        configs = configs_eval()
        torch.cuda.empty_cache()
    if args.ablation and rank == 0:
        ablation = hash_ablation_eval()
        torch.cuda.empty_cache()
    if args.batched and rank == 0:
        batched = batched_eval()
        torch.cuda.empty_cache()
    if args.learned and rank == 0:
        # (the held-out R-MAT n=2^21 is measured whole, in row slabs, by the
        # configs leg)
        learned_legs = []
        S = W.stencil27(128, seed=3)
        learned_legs.append(learned_eval("27-point stencil 128^3", S, 0, S.rows))
        del S
        D = W.block_diagonal(1 << 20, 1024, 24.0, seed=7)
        learned_legs.append(learned_eval("random block-diagonal n=2^20, 1024 blocks, mean degree 24, "
                                         "seed 7 (the training families, unseen size and seed)",
                                         D, 0, D.rows))

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": "GFLOPS", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(ms_max / args.steps, 3), "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": desc, "rows": A.rows, "nnzA": A.nnz,
                           "nprod": nprod_all, "nnzC": nnz_all,
                           "cache": "inputs larger than L2 (A 193 MB for rmat20; each step "
                                    "writes C, far larger than L2)",
                           "parallelism": (f"row slabs x{ws}, balanced by n_prod; C.rpt offsets by one "
                                           "all-gather of per-rank nnz") if ws > 1 else "single GPU",
                           "bin_config": "autotuned" if args.config else "default"},
                "roofline": roofline, "roofline_whole_step": whole,
                "stage_ms_live": breakdown, "kernel_ms_serial": serial,
                "bins": bins, "autotune": tuned, "numeric_values": rerun,
                "learned": learned_legs, "batched": batched, "hash_access": ablation,
                "op_rates": rates, "configs": configs,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_e2e(A, lib, steps, nprod):
    """The same multiply through spgemm_multiply_host: A from pinned host
    memory, C streamed back chunk by chunk into pinned host buffers."""
    import ctypes

    import torch

    import paper_2206_07244_gb300 as ops
    from paper_2206_07244_gb300 import _abi
    rpt = torch.from_numpy(A.rpt).pin_memory()
    col = torch.from_numpy(A.col).pin_memory()
    val = torch.from_numpy(A.val).pin_memory()
    a = _abi.CsrIn()
    a.rows, a.cols, a.nnz = A.rows, A.cols, A.nnz
    a.rpt, a.rpt_is_i64 = rpt.data_ptr(), 0
    a.col, a.val = col.data_ptr(), val.data_ptr()
    SINK = _abi.SINK_FN
    got = {"nnz": 0, "chunks": 0}

    def sink(ctx, r0, rows, prpt, pcol, pval, n):
        got["nnz"] += n
        got["chunks"] += 1
        return 0

    cb = SINK(sink)
    h = ops.Handle()
    nnz = ctypes.c_int64()
    chunk = 1 << 30
    # one untimed call allocates the pinned staging buffers
    _abi.check(lib.spgemm_multiply_host(h._h, ctypes.byref(a), ctypes.byref(a), chunk, cb, None,
                                        ctypes.byref(nnz)), "spgemm_multiply_host")
    if nprod is None:
        nprod = h.stats()["total_nprod"]
    times = []
    for _ in range(steps):
        got["nnz"] = 0
        torch.cuda.synchronize()
        t = time.perf_counter()
        _abi.check(lib.spgemm_multiply_host(h._h, ctypes.byref(a), ctypes.byref(a), chunk, cb,
                                            None, ctypes.byref(nnz)), "spgemm_multiply_host")
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
    h.close()
    assert got["nnz"] == nnz.value
    t = float(np.mean(times))
    h2d = 4 * (A.rows + 1) + 12 * A.nnz
    d2h = 8 * (A.rows + 1) + 12 * int(nnz.value)
    return {"value": round(2.0 * nprod / t / 1e9, 3), "unit": "GFLOPS", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "seconds_per_step": round(t, 4), "steps": steps,
            "chunks": got["chunks"], "call": "spgemm_multiply_host (pinned host A in, C streamed "
                                              "back in 1 GiB chunks)"}


if __name__ == "__main__":
    sys.exit(main())
