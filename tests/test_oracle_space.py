"""Space accounting of the oracle against the paper's figures (order of magnitude).

Sec. 1 / abstract: BuRR has under 1% space overhead; Fig. 3: each additional
thread (cut) costs about 10^1..10^3 bytes for an 8-bit filter.  The paper's
exact numbers depend on the authors' hash, threshold levels and overload
factor, which it does not state, so these are loose bands (exact per-cut
parity is unpinned).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_12365_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig3_overhead_per_cut.txt")


def _fig3():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            n, mode, t, b = line.split()
            rows.append((int(n), mode, int(t), float(b)))
    return rows


def test_golden_fig3_band():
    vals = [b for *_, b in _fig3()]
    assert len(vals) == 6 and 10 <= min(vals) and max(vals) <= 1000


@pytest.fixture(scope="module")
def kv():
    n = 1 << 20
    k = I.keys_np(n)
    return k, I.values_np(k, 8).astype(np.uint32)


def test_total_overhead_near_one_percent(kv):
    k, v = kv
    s = O.build(k, v, r=8)              # calibrated default load
    assert s.ok and 0.005 < s.overhead() < 0.015


def test_overhead_per_cut_in_fig3_band(kv):
    k, v = kv
    n = len(k)
    base = O.build(k, v, r=8, partition_slots=1 << 24, min_partition_slots=0)
    cut = O.build(k, v, r=8, partition_slots=1 << 14, min_partition_slots=1 << 14)
    ncuts = sum(max(0, cut.layer(l)["nparts"] - 1) for l in range(4))
    extra_bytes = (cut.overhead() - base.overhead()) * n      # r = 8: 1 byte per key
    per_cut = extra_bytes / ncuts
    lo = min(b for *_, b in _fig3()) / 10
    hi = max(b for *_, b in _fig3()) * 4
    assert ncuts >= 50 and lo <= per_cut <= hi
