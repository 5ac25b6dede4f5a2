"""Invariants of the whole layered structure, checked on the oracle.

* query(x) = f(x) for every x in S (retrieval problem, Sec. 1);
* on keys outside S the answer is arbitrary; for a filter (values = r-bit
  fingerprints) it matches the fingerprint with probability 2^-r (Sec. 1);
* the result does not depend on the input order (S is a set);
* partitions are independent: building one partition alone gives the same
  thresholds and table bits as building it inside its layer (Sec. 3);
* the same holds with 1+-bit thresholds, whose export stores exactly one
  threshold byte per bucket that bumps (Sec. 2, threshold storage);
* a key set that is not a set (a duplicated key) cannot be solved: the base
  case exhausts its retries (Sec. 4: the last layer is scaled up until it
  solves, and never does here).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_12365_gb300 import inputs as I
from tests.bruteforce import codes_of, unpack_z
from tests.export_format import exact_thresholds, parse


def _kv(n, r, seed=I.KEY_SEED):
    k = I.keys_np(n, seed=seed)
    return k, I.values_np(k, r).astype(np.uint32)


@pytest.mark.parametrize("n,r,P", [(0, 8, 65536), (1, 8, 65536), (2, 1, 65536), (77, 3, 65536),
                                   (5000, 8, 1024), (1 << 16, 8, 4096), (1 << 16, 16, 65536),
                                   (20000, 32, 2048), (30000, 1, 4096)])
def test_query_returns_stored_value(n, r, P):
    k, v = _kv(n, r, seed=n * 31 + r)
    s = O.build(k, v, r=r, partition_slots=P, min_partition_slots=P)
    assert s.ok
    assert np.array_equal(s.query(k), v)


def test_false_positive_rate_is_two_to_minus_r():
    n, r = 1 << 16, 8
    k, v = _kv(n, r)
    s = O.build(k, v, r=r, partition_slots=4096, min_partition_slots=4096)
    neg = I.keys_np(n, offset=n)                   # counters [n, 2n): disjoint from S
    fp = I.values_np(neg, r).astype(np.uint32)
    hits = int(np.sum(s.query(neg) == fp))
    mean = n / 2 ** r
    sd = math.sqrt(n * 2 ** -r * (1 - 2 ** -r))
    assert abs(hits - mean) < 6 * sd


def test_permutation_invariance():
    n, r = 20000, 8
    k, v = _kv(n, r)
    a = O.build(k, v, r=r, partition_slots=2048, min_partition_slots=2048).export()
    perm = np.random.default_rng(3).permutation(n)
    b = O.build(k[perm], v[perm], r=r, partition_slots=2048, min_partition_slots=2048).export()
    assert a == b


def test_partition_alone_equals_partition_in_layer():
    n, r, P = 12000, 8, 2048
    k, v = _kv(n, r)
    m = O.layer_slots(n, 1.015)
    K = O.num_partitions(m, P, 0)
    cuts = [j * P for j in range(1, K)]
    sigma = O.layer_seed(17, 0)
    full = O.build_layer(k, v, r, m, sigma, cuts=cuts)
    nb = O.num_buckets(m)
    zf = unpack_z(full.z, r, m)
    cf = codes_of(full.thresh, nb)
    starts = np.array([O.hash_key(int(x), sigma, m)[0] for x in k])
    bounds = [0] + cuts + [m - 63]
    own = [0] + [c + 64 for c in cuts] + [m]
    for j in (0, 1, K // 2, K - 1):
        sel = (starts >= bounds[j]) & (starts < bounds[j + 1])
        alone = O.build_layer(k[sel], v[sel], r, m, sigma, cuts=cuts)
        za = unpack_z(alone.z, r, m)
        ca = codes_of(alone.thresh, nb)
        assert za[own[j]:own[j + 1]] == zf[own[j]:own[j + 1]]
        b0, b1 = bounds[j] // 128, (bounds[j + 1] + 127) // 128
        assert ca[b0:b1] == cf[b0:b1]
        assert sorted(alone.bumped_keys.tolist()) == sorted(
            x for x in full.bumped_keys.tolist() if bounds[j] <= O.hash_key(int(x), sigma, m)[0] < bounds[j + 1])


def test_single_partition_when_layer_is_small():
    # minimum partition size (minbpt analogue, Sec. 3): below it no cut is made
    n, r = 3000, 8
    k, v = _kv(n, r)
    a = O.build(k, v, r=r, partition_slots=1024, min_partition_slots=1 << 20)
    b = O.build(k, v, r=r, partition_slots=1 << 20, min_partition_slots=0)
    assert a.layer(0)["nparts"] == 1 and a.export()[200:] == b.export()[200:]


def test_duplicate_key_is_unsolvable():
    k, v = _kv(1000, 8)
    k[10] = k[20]
    v[10] = v[20]
    s = O.build(k, v, r=8, fb_max_retries=3)
    assert s.status == O.UNSOLVABLE


def test_empty_input():
    s = O.build(np.zeros(0, np.uint64), np.zeros(0, np.uint32), r=8)
    assert s.ok and s.layer(0)["m"] == 0 and s.layer("fallback")["m"] == 0
    assert s.query(I.keys_np(10)).tolist() == [0] * 10


def test_invalid_params_rejected():
    k, v = _kv(10, 8)
    for bad in (dict(r=0), dict(r=33), dict(w=32), dict(partition_slots=100),
                dict(levels=(0, 32, 64, 100)), dict(levels=(0, 32, 32, 128)),
                dict(levels=(5, 32, 64, 128)), dict(alpha=0.0)):
        assert O.build(k, v, **bad).status == O.EINVAL


@pytest.mark.parametrize("n,r,P", [(0, 8, 65536), (1, 8, 65536), (77, 3, 65536), (5000, 8, 1024),
                                   (1 << 16, 8, 4096), (20000, 32, 2048), (30000, 1, 256)])
def test_1plus_query_returns_stored_value(n, r, P):
    k, v = _kv(n, r, seed=n * 37 + r)
    s = O.build(k, v, r=r, partition_slots=P, min_partition_slots=P, threshold_mode=O.THRESH_1PLUS)
    assert s.ok
    assert np.array_equal(s.query(k), v)


def test_1plus_export_stores_the_exact_thresholds():
    n, r, P = 1 << 15, 8, 2048
    k, v = _kv(n, r)
    s = O.build(k, v, r=r, partition_slots=P, min_partition_slots=P, threshold_mode=O.THRESH_1PLUS)
    ex = parse(s.export())
    assert ex["version"] == 2
    for l, L in enumerate(ex["layers"]):
        t = exact_thresholds(L)
        assert np.array_equal(t, s.layer(l)["texact"].astype(np.int64))
        assert len(L["exact"]) == int(np.count_nonzero(t)) and (L["exact"] > 0).all()
        # every partition start (a cut) is flagged with at least w
        for j in range(1, L["parts"]):
            assert t[j * P // 128] >= 64


def test_1plus_permutation_invariance():
    n, r = 20000, 8
    k, v = _kv(n, r)
    kw = dict(r=r, partition_slots=2048, min_partition_slots=2048, threshold_mode=O.THRESH_1PLUS)
    a = O.build(k, v, **kw).export()
    perm = np.random.default_rng(5).permutation(n)
    assert O.build(k[perm], v[perm], **kw).export() == a


def _insert_tagged(band, s, c, tag):
    """Ribbon insertion of row c at slot s into band {slot: (row, tag)}; tags are XORed along.
    Returns the slot stored at, or None and the accumulated tag when the row reduces to zero."""
    pos, cur = s, c
    while pos in band:
        bc, bt = band[pos]
        cur ^= bc
        tag ^= bt
        if cur == 0:
            return None, tag
        tz = (cur & -cur).bit_length() - 1
        pos += tz
        cur >>= tz
    band[pos] = (cur, tag)
    return pos, None


@pytest.mark.parametrize("alpha,cut_every", [(1.015, 0), (1.0, 0), (1.015, 2048)])
def test_1plus_threshold_follows_from_dependencies_in_any_order(alpha, cut_every):
    # Sec. 2, 1+-bit thresholds: a bucket's threshold is the least t whose rows at offsets >= t
    # insert.  The set's dependencies do not depend on the insertion order, so t can be
    # recovered from one insertion of the whole bucket in any order: tag the rows of the
    # bucket (ascending offset), drop the rows that reduce to zero, reduce their tags to
    # distinct lowest bits; t = offset of the row of the largest such bit + 1.  Checked against
    # the oracle's descending-offset insertion on hashed equations, bucket by bucket.  With cuts
    # (Sec. 3), the first bucket of a partition starts from the forced threshold w: its set is
    # the rows at offsets >= w, and t >= w.
    n, r, B, w = 24_000, 8, 128, 64
    k, v = _kv(n, r, seed=4242)
    m = O.layer_slots(n, alpha)
    sigma = O.layer_seed(7, 0)
    cuts = list(range(cut_every, m - w, cut_every)) if cut_every else []
    res = O.build_layer(k, v, r, m, sigma, cuts=cuts, mode=O.THRESH_1PLUS)
    assert res.status == 0
    starts, coeffs = O.hash_many(k, sigma, m)
    buckets = {}
    for s, c in zip(starts.tolist(), coeffs.tolist()):
        buckets.setdefault(s // B, []).append((s, c))
    rng = np.random.default_rng(11)
    band, failing = {}, 0
    forced_buckets = {c // B for c in cuts}
    for b in range(len(res.texact)):
        forced = w if b in forced_buckets else 0
        rows = [sc for sc in sorted(buckets.get(b, []), key=lambda sc: sc[0] % B) if sc[0] % B >= forced]
        order = rng.permutation(len(rows))
        stored, tags = [], []
        for i in order:
            s, c = rows[i]
            p, tag = _insert_tagged(band, s, c, 1 << int(i))
            (stored.append(p) if p is not None else tags.append(tag))
        t = forced
        if not tags:
            for p in stored:                             # the bucket inserted: clear its tags
                band[p] = (band[p][0], 0)
        else:
            failing += 1
            for p in stored:
                del band[p]
            top = -1
            for bit in range(len(rows)):
                piv = next((j for j, x in enumerate(tags) if (x >> bit) & 1 and x & ((1 << bit) - 1) == 0), None)
                if piv is None:
                    continue
                for j in range(len(tags)):
                    if j != piv and (tags[j] >> bit) & 1:
                        tags[j] ^= tags[piv]
                top = bit
            assert all(x != 0 for x in tags)          # independent dependencies, one per dropped row
            t = rows[top][0] % B + 1
            for s, c in rows:                            # the rows above t insert, untagged
                if s % B >= t:
                    assert _insert_tagged(band, s, c, 0)[0] is not None
        assert t == int(res.texact[b]), b
    assert failing >= 20


def test_invalid_threshold_mode_rejected():
    k, v = _kv(10, 8)
    assert O.build(k, v, threshold_mode=2).status == O.EINVAL


@pytest.mark.parametrize("lower", [0, 4096, 1024, 128])
def test_lower_layers_cut_at_their_own_partition_size(lower):
    # deep layers are cut every lower_partition_slots (0: as layer 0), with
    # the same minimum-size rule; queries are unaffected (cuts are invisible)
    n, r, P, minP = 1 << 17, 8, 8192, 1024
    k, v = _kv(n, r, seed=lower + 5)
    s = O.build(k, v, r=r, partition_slots=P, min_partition_slots=minP, lower_partition_slots=lower)
    assert s.ok and np.array_equal(s.query(k), v)
    for l in range(4):
        L = s.layer(l)
        Pl = P if (l == 0 or lower == 0) else lower
        assert L["nparts"] == O.num_partitions(L["m"], Pl, minP)
    if lower and 2 * lower <= s.layer(1)["m"]:
        assert s.layer(1)["nparts"] > O.num_partitions(s.layer(1)["m"], P, minP)


@pytest.mark.parametrize("P,minP", [(65536, 4096), (4096, 4096), (1024, 1024), (65536, 0), (2048, 2048)])
def test_partitions_have_balanced_lengths(P, minP):
    # Sec. 3 gives each thread a near-equal share.  With cuts at j*P, no
    # partition may be much longer than P: at most P plus half a partition
    # (plus 1024 slots for tiny P), and a separate last partition is never
    # shorter than 1024 slots.  A layer below max(P, minP) is one partition.
    for m in range(64, 40 * P + 1, 64 * max(1, P // 4096)):
        K = O.num_partitions(m, P, minP)
        if m < max(P, minP):
            assert K == 1
            continue
        lens = [P] * (K - 1) + [m - (K - 1) * P]
        assert all(x > 0 for x in lens)
        assert max(lens) < P + max(P // 2, 1024)
        if m % P and K > m // P:
            assert lens[-1] >= 1024


def test_remainder_at_the_threshold_gets_its_own_partition():
    # the remainder rule at its edge (P = 4096, min 4096: threshold 2048 slots)
    assert O.num_partitions(5 * 4096 + 2048, 4096, 4096) == 6
    assert O.num_partitions(5 * 4096 + 1984, 4096, 4096) == 5
    assert O.num_partitions(1000 * 65536 + 4096, 65536, 4096) == 1001
    assert O.num_partitions(1000 * 65536 + 4032, 65536, 4096) == 1000
