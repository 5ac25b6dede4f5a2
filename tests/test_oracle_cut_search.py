"""Cut-point search (Sec. 3, "Selecting Cut Points") in the oracle.

* The chosen cuts equal a NumPy re-derivation from the definition: for a cut
  at bucket b, bumped = keys starting in its first w slots, prev = keys in the
  w-1 slots before it; minbump minimises bumped, maxprev maximises prev, diff
  minimises bumped - prev, over the first min(range, P/B) buckets from the
  nominal cut (first best wins).
* A layer built with searched cuts passes the dense GF(2) brute force (kept
  sets, minimal thresholds, forced bumps at the cuts, supports inside their
  partitions, the table).
* Searching saves space, as in Fig. 5; a range of 1 is the plain cut.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_12365_gb300 import inputs as I
from tests.bruteforce import check_layer, check_layer_1plus

B, W = 128, 64


def _kv(n, r, seed):
    k = I.keys_np(n, seed=seed)
    return k, I.values_np(k, r).astype(np.uint32)


def _numpy_cuts(keys, m, sigma, P, K, mode, rng):
    starts, _ = O.hash_many(keys, sigma, m)
    starts = starts.astype(np.int64)
    nb = O.num_buckets(m)
    off = starts % B
    lo = np.bincount(starts[off < W] // B, minlength=nb + 1)
    hi = np.bincount(starts[off >= B - (W - 1)] // B, minlength=nb + 1)
    cuts = []
    R = min(rng, P // B)
    for j in range(1, K):
        b0 = j * P // B
        cand = [b for b in range(b0, b0 + R) if b < nb]
        scores = []
        for b in cand:
            bumped, prev = int(lo[b]), int(hi[b - 1]) if b > 0 else 0
            scores.append({1: bumped, 2: -prev, 3: bumped - prev}[mode])
        cuts.append(cand[int(np.argmin(scores))] * B)
    return np.array(cuts, dtype=np.uint64)


@pytest.mark.parametrize("mode", [O.CUT_MINBUMP, O.CUT_MAXPREV, O.CUT_DIFF])
@pytest.mark.parametrize("n,P,rng", [(200_000, 8192, 50), (60_000, 1024, 50), (100_000, 4096, 7)])
def test_search_matches_numpy_definition(mode, n, P, rng):
    k, _ = _kv(n, 8, seed=n + mode)
    m = O.layer_slots(n, 1.015)
    K = O.num_partitions(m, P, 0)
    sigma = O.layer_seed(3, 0)
    got = O.search_cuts(k, m, sigma, P, K, mode, rng)
    assert np.array_equal(got, _numpy_cuts(k, m, sigma, P, K, mode, rng))
    assert np.any(got != np.arange(1, K, dtype=np.uint64) * P)     # the search moves cuts


@pytest.mark.parametrize("mode", [O.CUT_MINBUMP, O.CUT_MAXPREV, O.CUT_DIFF])
def test_layer_with_searched_cuts_matches_dense_gf2(mode):
    n, P = 900, 512
    k, v = _kv(n, 5, seed=40 + mode)
    m = O.layer_slots(n, 1.1)
    K = O.num_partitions(m, P, 0)
    sigma = O.layer_seed(8, 0)
    cuts = [int(c) for c in O.search_cuts(k, m, sigma, P, K, mode, 3)]
    check_layer(k, v, 5, m, sigma, cuts)
    check_layer_1plus(k, v, 5, m, sigma, cuts)


@pytest.mark.parametrize("mode", [O.CUT_MINBUMP, O.CUT_MAXPREV, O.CUT_DIFF])
def test_structure_with_search(mode):
    k, v = _kv(1 << 16, 8, seed=9)
    kw = dict(r=8, partition_slots=2048, min_partition_slots=2048, cut_search=mode)
    s = O.build(k, v, **kw)
    assert s.ok and np.array_equal(s.query(k), v)
    L = s.layer(0)
    sigma = O.layer_seed(s.params.seed, 0)
    assert np.array_equal(L["cuts"], O.search_cuts(k, L["m"], sigma, 2048, L["nparts"], mode, 50))
    one = O.build(k, v, **{**kw, "cut_search_range": 1}).export()
    assert one == O.build(k, v, **{**kw, "cut_search": O.CUT_NONE}).export()


def test_search_saves_space_per_cut():
    # Fig. 5: searching for better cut buckets lowers the overhead per thread
    n = 1 << 20
    k, v = _kv(n, 8, seed=0)
    for tmode in (O.THRESH_2BIT, O.THRESH_1PLUS):
        base = O.build(k, v, r=8, partition_slots=1 << 24, min_partition_slots=0, lower_partition_slots=0,
                       threshold_mode=tmode)
        per = {}
        for mode in (O.CUT_NONE, O.CUT_MINBUMP, O.CUT_MAXPREV, O.CUT_DIFF):
            s = O.build(k, v, r=8, partition_slots=1 << 14, min_partition_slots=1 << 14, lower_partition_slots=0,
                        threshold_mode=tmode, cut_search=mode)
            ncuts = sum(max(0, s.layer(l)["nparts"] - 1) for l in range(4))
            per[mode] = (s.overhead() - base.overhead()) * n / ncuts
        assert all(per[m] < per[O.CUT_NONE] for m in (O.CUT_MINBUMP, O.CUT_MAXPREV, O.CUT_DIFF)), per
