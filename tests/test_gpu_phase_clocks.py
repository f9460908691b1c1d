"""Phase clocks of the numeric bitmap kernel (a profiling aid): with them on,
every phase of the 1024-thread whole-row form reports SM clock cycles, the
product is still the oracle's, the counters reset on read, and with them off
again nothing more is counted."""

import numpy as np
import pytest

import oracle
import workloads as W
from helpers import assert_values_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2206_07244_gb300 as ops  # noqa: E402

ops.build()


def bitmap_bin_only():
    """Every row of C to the numeric bitmap kernel (whole-row form)."""
    cfg = ops.default_config()
    nb = len(ops.kernel_table(1)) - 1
    cfg["num_kernel"], cfg["num_range"] = [nb], [-1]
    cfg["bitmap_path"] = 0
    return cfg


def test_phase_clocks_cover_every_phase_and_keep_c():
    # 2^19 columns: 96 KB of bitmap and prefix counts, so one 1024-thread
    # block per SM (the form that keeps the clocks)
    A = W.rmat(19, 8, seed=7)
    r0, r1 = 0, 64
    dA = ops.CSR.from_arrays(A.rows, A.cols, A.rpt, A.col, A.val)
    with ops.Handle(bitmap_bin_only()) as h:
        assert all(v == 0 for v in h.bitmap_phase_clocks().values())
        h.set_phase_clocks(True)
        h.symbolic(dA, dA, r0, r1)
        C = h.numeric(dA, dA)
        h.status()
        got = C.numpy()
        clk = h.bitmap_phase_clocks(reset=True)
        assert list(clk) == list(ops.Handle.PHASES)
        assert all(v > 0 for v in clk.values()), clk
        assert all(v == 0 for v in h.bitmap_phase_clocks().values())
        h.set_phase_clocks(False)
        h.symbolic(dA, dA, r0, r1)
        C2 = h.numeric(dA, dA)
        h.status()
        assert all(v == 0 for v in h.bitmap_phase_clocks().values())
        got2 = C2.numpy()
    rpt, col, val, ab = oracle.spgemm(A, A, r0, r1)
    for g_rpt, g_col, g_val in (got, got2):
        assert np.array_equal(g_rpt, rpt)
        assert np.array_equal(g_col, col)
        assert_values_close(g_val, val, ab)
