"""The threaded oracle (partitions spread over host threads, Sec. 3: once the
cuts are placed every partition is inserted and back-substituted on its own)
must give the serial oracle's structure byte for byte: sizes, thresholds,
tables, bumped keys of every layer and the base case.  The serial oracle is
the pinned one; this ties the threaded variant, which the benchmark times and
the full-size GPU parity tests use, to it."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_12365_gb300 import inputs as I

CASES = [
    (0, 8, {}),
    (1, 8, {}),
    (70_000, 8, dict(partition_slots=1024, min_partition_slots=1024)),
    (65_573, 8, dict(partition_slots=4096, min_partition_slots=4096)),      # ragged remainder
    (200_003, 16, dict(partition_slots=8192, min_partition_slots=8192)),
    (90_000, 4, dict(partition_slots=128, min_partition_slots=0)),          # a cut at every bucket
    (70_000, 5, dict(partition_slots=384, min_partition_slots=0)),          # cuts inside 2-bit words
    (100_000, 8, dict(partition_slots=2048, min_partition_slots=2048, threshold_mode=O.THRESH_1PLUS)),
    (120_000, 8, dict(partition_slots=2048, min_partition_slots=2048, cut_search=O.CUT_DIFF)),
    (60_000, 8, dict(partition_slots=1024, min_partition_slots=0, alpha=1.6)),   # heavy bumping
    (50_000, 8, dict(partition_slots=2048, min_partition_slots=2048, B=64, levels=(0, 16, 32, 64))),
    (1 << 20, 8, {}),
]


@pytest.mark.parametrize("n,r,params", CASES)
@pytest.mark.parametrize("threads", [2, 7])
def test_threaded_oracle_equals_serial(n, r, params, threads):
    keys = I.keys_np(n, seed=n + 3)
    vals = I.values_np(keys, r).astype(np.uint32)
    a = O.build(keys, vals, r=r, **params)
    b = O.build(keys, vals, r=r, threads=threads, **params)
    assert a.ok and b.ok
    assert a.export() == b.export()
    assert a.stats.xor_steps == b.stats.xor_steps and a.stats.inserted == b.stats.inserted
    assert a.stats.max_drift == b.stats.max_drift
    for l in range(4):
        assert a.stats.bumped[l] == b.stats.bumped[l]


def test_threaded_layer_bumps_in_serial_order():
    n, r, m = 300_000, 8, O.layer_slots(300_000, 1.015)
    keys = I.keys_np(n, seed=5)
    vals = I.values_np(keys, r).astype(np.uint32)
    sigma = O.layer_seed(1, 0)
    cuts = list(range(4096, m - 64, 4096))
    a = O.build_layer(keys, vals, r, m, sigma, cuts=cuts)
    b = O.build_layer(keys, vals, r, m, sigma, cuts=cuts, threads=5)
    assert a.status == 0 and b.status == 0
    assert np.array_equal(a.thresh, b.thresh) and np.array_equal(a.z, b.z)
    assert np.array_equal(a.bumped_keys, b.bumped_keys) and np.array_equal(a.bumped_vals, b.bumped_vals)


def test_threaded_base_case_failure_is_reported():
    keys = I.keys_np(5000, seed=9)
    keys[7] = keys[3]
    vals = I.values_np(keys, 8).astype(np.uint32)
    s = O.build(keys, vals, r=8, threads=4, fb_max_retries=1, partition_slots=1024, min_partition_slots=1024)
    assert s.status == O.UNSOLVABLE
