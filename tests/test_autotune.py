"""The autotuner's search space: every configuration it can produce is valid
for the library (CPU), and multiplies give the oracle's result under each of
them (GPU)."""

import itertools

import numpy as np
import pytest

import workloads as W


def _space():
    from paper_2206_07244_gb300 import autotune
    nsym = len(autotune.kernel_table(0)) - 1
    nnum = len(autotune.kernel_table(1)) - 1
    for sr, nr, sc, nc, ln in itertools.product(autotune.SYM_RATIOS, autotune.NUM_RATIOS,
                                                (nsym - 1, nsym - 4, 0), (nnum - 1, nnum - 5, 0),
                                                (0, 8)):
        yield autotune.make_config(sr, nr, sc, nc, ln, 32 - 3 * ln)


def test_every_candidate_is_a_valid_configuration():
    import paper_2206_07244_gb300 as ops
    ops.build()
    from paper_2206_07244_gb300 import autotune
    tabs = {0: autotune.kernel_table(0), 1: autotune.kernel_table(1)}
    n = 0
    for cfg in _space():
        n += 1
        for key, phase in (("sym", 0), ("num", 1)):
            ks, rs = cfg[f"{key}_kernel"], cfg[f"{key}_range"]
            assert ks[-1] == len(tabs[phase]) - 1 and rs[-1] == -1
            assert all(a < b for a, b in zip(rs[:-2], rs[1:-1]))
            for k, r in zip(ks[:-1], rs[:-1]):
                assert 0 <= r <= tabs[phase][k][3]
    assert n > 50


@pytest.mark.gpu
def test_tuned_configurations_keep_results_exact():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import oracle
    import paper_2206_07244_gb300 as ops
    from helpers import assert_values_close
    A = W.rmat(11, 16, seed=13)
    want = oracle.spgemm(A, A)
    dA = ops.CSR.from_workload(A)
    for cfg in list(_space())[::7]:
        with ops.Handle(cfg) as h:
            C = h.multiply(dA, dA)
            h.status()
            rpt, col, val = C.numpy()
        assert np.array_equal(rpt, want[0]) and np.array_equal(col, want[1])
        assert_values_close(val, want[2], want[3])


@pytest.mark.gpu
def test_tune_runs_and_returns_a_configuration():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2206_07244_gb300 as ops
    from paper_2206_07244_gb300 import autotune
    A = ops.CSR.from_workload(W.rmat(12, 8, seed=2))
    best, hist = autotune.tune(A, A, reps=1)
    assert len(hist) >= 10
    with ops.Handle(best) as h:
        h.multiply(A, A)
        h.status()
