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


def test_1plus_costs_less_per_cut_than_2bit(kv):
    # Fig. 3: 1+-bit thresholds lose fewer bytes per additional thread than
    # 2-bit thresholds (their bumping is more granular), both within the band
    k, v = kv
    n = len(k)
    per_cut = {}
    for mode in (O.THRESH_2BIT, O.THRESH_1PLUS):
        base = O.build(k, v, r=8, partition_slots=1 << 24, min_partition_slots=0, threshold_mode=mode)
        cut = O.build(k, v, r=8, partition_slots=1 << 14, min_partition_slots=1 << 14, threshold_mode=mode)
        ncuts = sum(max(0, cut.layer(l)["nparts"] - 1) for l in range(4))
        per_cut[mode] = (cut.overhead() - base.overhead()) * n / ncuts
    fig3 = {mode: [b for nn, md, _, b in _fig3() if md == mode] for mode in ("2bit", "1plus")}
    assert all(a < b for a, b in zip(fig3["1plus"], fig3["2bit"]))      # the paper's ordering
    assert per_cut[O.THRESH_1PLUS] < per_cut[O.THRESH_2BIT]
    assert min(fig3["1plus"]) / 10 <= per_cut[O.THRESH_1PLUS] <= max(fig3["1plus"]) * 4


def test_1plus_total_overhead_below_2bit(kv):
    k, v = kv
    a = O.build(k, v, r=8)
    b = O.build(k, v, r=8, threshold_mode=O.THRESH_1PLUS)
    assert b.ok and 0.0 < b.overhead() < a.overhead()
