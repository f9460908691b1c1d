"""Host-side logic of the multi-rank benchmark path, on CPU with gloo
(world size 2): every output row belongs to exactly one rank's slab, the
slabs are contiguous and balanced by A's non-zeros, and the step time is the
maximum over ranks while products add up."""

import os
import socket

import numpy as np
import pytest

import bench
import workloads as W


def test_row_slabs_partition_rows():
    A = W.rmat(12, 8, seed=3)
    for ws in (1, 2, 3, 4, 8):
        slabs = [bench.row_slab(A, r, ws) for r in range(ws)]
        assert slabs[0][0] == 0 and slabs[-1][1] == A.rows
        for (a0, a1), (b0, b1) in zip(slabs, slabs[1:]):
            assert a1 == b0 and a0 <= a1
        if ws > 1:
            rpt = A.rpt.astype(np.int64)
            share = [int(rpt[r1] - rpt[r0]) for r0, r1 in slabs]
            assert max(share) - min(share) <= int(np.diff(rpt).max()) + A.nnz // 100


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
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
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ws = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
    A = W.rmat(10, 8, seed=4)
    assert out[0] == out[1] == (A.rows, 11.0)
