"""Row sharding of C = A*B over several ranks, on CPU with gloo (world size
2): slabs are contiguous, cover every row once and are balanced by the prefix
sum of n_prod; each rank multiplies its slab (here with the CPU oracle, which
the GPU ranks replace with the library's row-window calls), the ranks
exchange one int64 each (their entry counts) to offset their parts of C.rpt,
and the stitched C equals the single-rank product bit for bit. The benchmark
path's step time is the maximum over ranks while products add up."""

import os
import socket

import numpy as np
import pytest

import bench
import oracle
import workloads as W
from paper_2206_07244_gb300 import shard


def test_nprod_per_row_matches_oracle():
    A = W.rmat(11, 8, seed=3)
    B = W.random_csr(A.cols, 300, 0.03, seed=4)
    assert np.array_equal(shard.nprod_per_row(A.rpt, A.col, B.rpt), oracle.nprod(A, B))
    E = W.Csr(3, 5, np.zeros(4, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0))
    assert shard.nprod_per_row(E.rpt, E.col, np.zeros(6, dtype=np.int32)).tolist() == [0, 0, 0]


def test_slabs_partition_rows_and_balance_products():
    A = W.rmat(12, 8, seed=3)
    npr = oracle.nprod(A, A)
    for ws in (1, 2, 3, 4, 8):
        slabs = shard.slab_bounds(npr, ws)
        assert len(slabs) == ws and slabs[0][0] == 0 and slabs[-1][1] == A.rows
        for (a0, a1), (b0, b1) in zip(slabs, slabs[1:]):
            assert a1 == b0 and a0 <= a1
        share = [int(npr[r0:r1].sum()) for r0, r1 in slabs]
        # a contiguous cut misses the ideal share by at most one row's products
        assert max(share) - int(npr.sum()) // ws <= int(npr.max())
        assert [bench.row_slab(A, r, ws) for r in range(ws)] == slabs


def test_slabs_with_one_giant_row():
    npr = np.array([0, 5, 1000, 3, 0, 2], dtype=np.int64)
    slabs = shard.slab_bounds(npr, 4)
    assert slabs[0][0] == 0 and slabs[-1][1] == 6
    assert sum(r1 - r0 for r0, r1 in slabs) == 6


def test_stitch_offsets():
    parts = [(np.array([0, 2, 3]), np.array([1, 4, 0]), np.array([1.0, 2.0, 3.0])),
             (np.array([0]), np.zeros(0, np.int32), np.zeros(0)),
             (np.array([0, 1]), np.array([7]), np.array([4.0]))]
    rpt, col, val = shard.stitch(parts)
    assert rpt.tolist() == [0, 2, 3, 4] and col.tolist() == [1, 4, 0, 7]
    assert shard.exclusive_offsets([3, 0, 1]) == [0, 3, 3]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _product_worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    A = W.rmat(11, 8, seed=5)
    B = W.rmat(11, 6, seed=6)
    r0, r1 = shard.slab_bounds(shard.nprod_per_row(A.rpt, A.col, B.rpt), ws)[rank]
    rpt, col, val, _ = oracle.spgemm(A, B, r0, r1, with_abs=False)
    off, total = shard.rpt_offset(int(rpt[-1]))
    parts = [None] * ws
    dist.all_gather_object(parts, (rpt, col, val))
    offs = [None] * ws
    dist.all_gather_object(offs, off)
    dist.barrier()
    if rank == 0:
        out["stitched"] = shard.stitch(parts)
        out["offsets"] = offs
        out["total"] = total
        out["slabs"] = [shard.slab_bounds(shard.nprod_per_row(A.rpt, A.col, B.rpt), ws)[r] for r in range(ws)]
    dist.destroy_process_group()


def test_gloo_two_ranks_stitched_product_equals_single_rank():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ws = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_product_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
    A = W.rmat(11, 8, seed=5)
    B = W.rmat(11, 6, seed=6)
    rpt, col, val, _ = oracle.spgemm(A, B, with_abs=False)
    g_rpt, g_col, g_val = out["stitched"]
    assert np.array_equal(g_rpt, rpt)
    assert np.array_equal(g_col, col)
    assert np.array_equal(g_val, val)
    assert out["total"] == int(rpt[-1])
    (a0, a1), (b0, b1) = out["slabs"]
    assert out["offsets"] == [0, int(rpt[a1])] and a1 == b0


def _timing_worker(rank, ws, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    A = W.rmat(10, 8, seed=4)
    r0, r1 = bench.row_slab(A, rank, ws)
    rows = torch.tensor([r1 - r0], dtype=torch.int64)
    dist.all_reduce(rows)
    ms = torch.tensor([10.0 + rank], dtype=torch.float64)
    dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    dist.barrier()
    out[rank] = (int(rows.item()), float(ms.item()))
    dist.destroy_process_group()


def test_gloo_two_ranks_cover_all_rows_and_take_max_time():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ws = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_timing_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
    A = W.rmat(10, 8, seed=4)
    assert out[0] == out[1] == (A.rows, 11.0)
