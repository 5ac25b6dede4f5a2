"""The oracle's layer build against dense GF(2) brute force on tiny inputs.

Covers the bumping rules of Sec. 2 (2-bit and 1+-bit thresholds,
overloading), the partition cuts of Sec. 3 and the back-substitution (Fig. 7's
third phase).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_12365_gb300 import inputs as I
from tests.bruteforce import check_layer, check_layer_1plus, codes_of, unpack_z
from tests.gf2 import solve_free_zero


def _layer_inputs(n, r, seed=11):
    k = I.keys_np(n, seed=seed)
    v = I.values_np(k, r).astype(np.uint32)
    return k, v


@pytest.mark.parametrize("n,alpha,P,r", [
    (300, 1.015, 1 << 20, 8),      # one partition, near the calibrated load
    (600, 1.015, 256, 8),          # cuts every 2 buckets
    (600, 1.30, 256, 1),           # heavy overload: every level gets used
    (900, 1.10, 384, 5),
    (500, 0.70, 128, 16),          # underloaded, a cut at every bucket
    (400, 1.50, 512, 32),
])
def test_layer_matches_dense_gf2(n, alpha, P, r):
    k, v = _layer_inputs(n, r, seed=n + r)
    m = O.layer_slots(n, alpha)
    K = O.num_partitions(m, P, 0)
    cuts = [j * P for j in range(1, K)]
    sigma = O.layer_seed(99, 0)
    res, codes = check_layer(k, v, r, m, sigma, cuts)
    if alpha >= 1.3:
        assert max(codes) >= 1           # the overloaded cases do bump


def test_all_threshold_levels_exercised_across_seeds():
    # loads from calibrated to heavily overloaded: every 2-bit level occurs
    seen = set()
    for seed, alpha in enumerate((1.3, 1.6, 2.2)):
        k, v = _layer_inputs(1500, 4, seed=100 + seed)
        m = O.layer_slots(1500, alpha)
        _, codes = check_layer(k, v, 4, m, O.layer_seed(seed, 0), [256, 512])
        seen |= set(codes)
    assert seen == {0, 1, 2, 3}


def test_single_key_closed_form():
    # one equation: it is stored at its start slot and the table holds its
    # value there, zeros elsewhere
    r, m = 8, 128
    sigma = O.layer_seed(1, 0)
    key, val = 0xDEADBEEF, 0xA5
    res = O.build_layer([key], [val], r, m, sigma)
    s, _ = O.hash_key(key, sigma, m)
    z = unpack_z(res.z, r, m)
    assert z[s] == val and sum(1 for x in z if x) == 1
    assert codes_of(res.thresh, O.num_buckets(m)) == [0] * O.num_buckets(m)


def test_fallback_layer_is_plain_ribbon():
    # base case: no thresholds, every row must insert (Sec. 3, last paragraph)
    r = 8
    k, v = _layer_inputs(200, r, seed=5)
    m = O.fallback_slots(200, 0.1)
    sigma = O.layer_seed(5, 4)
    res = O.build_layer(k, v, r, m, sigma, fallback=True)
    assert res.status == 0 and len(res.bumped_keys) == 0
    rows = []
    for key in k:
        s, c = O.hash_key(int(key), sigma, m)
        rows.append(c << s)
    z = solve_free_zero(rows, [int(x) for x in v], m)
    assert unpack_z(res.z, r, m) == z
    # too few slots: the base case reports failure instead of bumping
    tiny = O.build_layer(k, v, r, 128, sigma, fallback=True)
    assert tiny.status == O.FAIL


@pytest.mark.parametrize("n,alpha,P,r", [
    (300, 1.015, 1 << 20, 8),
    (600, 1.015, 256, 8),
    (600, 1.30, 256, 1),
    (900, 1.10, 384, 5),
    (500, 0.70, 128, 16),
    (400, 1.50, 512, 32),
    (1500, 2.2, 256, 4),           # most buckets bump, some entirely
])
def test_layer_1plus_matches_dense_gf2(n, alpha, P, r):
    k, v = _layer_inputs(n, r, seed=n + r + 7)
    m = O.layer_slots(n, alpha)
    K = O.num_partitions(m, P, 0)
    cuts = [j * P for j in range(1, K)]
    res, t = check_layer_1plus(k, v, r, m, O.layer_seed(98, 0), cuts)
    if alpha >= 1.5:
        # exact thresholds: values between the 2-bit levels occur
        assert set(t) - {0, 32, 64, 128}


def test_1plus_equals_2bit_when_nothing_bumps_but_the_cuts():
    # underloaded: only the forced bumps after cuts remain, and both modes
    # force exactly offsets < 64 there, so the kept sets and tables agree
    r, n, P = 8, 400, 256
    k, v = _layer_inputs(n, r, seed=3)
    m = O.layer_slots(n, 0.5)
    cuts = [j * P for j in range(1, O.num_partitions(m, P, 0))]
    sigma = O.layer_seed(4, 0)
    a = O.build_layer(k, v, r, m, sigma, cuts=cuts)
    b = O.build_layer(k, v, r, m, sigma, cuts=cuts, mode=O.THRESH_1PLUS)
    codes = codes_of(a.thresh, O.num_buckets(m))
    assert set(codes) <= {0, 2} and list(b.texact) == [64 if c == 2 else 0 for c in codes]
    assert np.array_equal(a.z, b.z) and sorted(a.bumped_keys) == sorted(b.bumped_keys)
