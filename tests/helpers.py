"""Comparison helpers shared by the tests (no arithmetic of the method)."""

from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# Value tolerance for float64 results. Two correct implementations sum the
# same products in different orders; the difference of two such sums is
# bounded by about 2*n*u*sum|a_ik*b_kj| (u = 2^-53, n = products per entry).
# For the row sizes of these workloads n*u < 1e-12, so entries must agree to
# 1e-12 relative to max(|c|, sum|a*b|). Integer-valued inputs sum exactly and
# must agree bit for bit.
VALUE_RTOL = 1e-12


def assert_values_close(got, want, scale, rtol=VALUE_RTOL, what="values"):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = np.maximum(np.abs(want), np.asarray(scale, dtype=np.float64))
    err = np.abs(got - want)
    bad = err > rtol * scale
    if bad.any():
        i = int(np.nonzero(bad)[0][0])
        raise AssertionError(
            f"{what}: {int(bad.sum())} of {got.size} entries outside "
            f"{rtol} relative; first at {i}: got {got[i]!r}, want {want[i]!r}, "
            f"scale {scale[i]!r}")


def load_binning_golden():
    ranges, cases = {}, []
    with open(os.path.join(GOLDEN, "binning_ranges.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "ranges":
                ranges[parts[1]] = [int(x) if int(x) >= 0 else 2**62 for x in parts[2:]]
            elif parts[0] == "case":
                cases.append((parts[1], int(parts[2]), int(parts[3])))
    return ranges, cases
