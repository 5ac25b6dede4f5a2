"""GPU parity: the CUDA path through the C ABI against the serial CPU oracle.

Bit-exact everywhere (integer GF(2) work): hash records, bucket grouping,
whole-structure exports (sizes, thresholds, tables of every layer and the
base case) and query outputs.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_12365_gb300 import inputs as I
from tests.export_format import describe_difference, parse

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_12365_gb300 import burr  # noqa: E402

DEV = "cuda"


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _vals_np(t):
    a = t.cpu().numpy()
    return a.view({1: np.uint8, 2: np.uint16, 4: np.uint32}[a.dtype.itemsize]).astype(np.uint32)


def _kv(n, r, seed=I.KEY_SEED, offset=0):
    k = I.keys_torch(n, DEV, seed=seed, offset=offset)
    return k, I.values_torch(k, r)


@pytest.mark.parametrize("n,m,layer", [(1_000_003, 1_015_872, 0), (4097, 4160, 3), (1, 64, 7)])
def test_stage_hash_matches_oracle(n, m, layer):
    seed = 0xABCDEF
    keys = I.keys_torch(n, DEV)
    s, c = burr.stage_hash(keys, seed, layer, m)
    os_, oc = O.hash_many(_u64(keys), O.layer_seed(seed, layer), m)
    assert np.array_equal(s.cpu().numpy().view(np.uint32).astype(np.uint64), os_)
    assert np.array_equal(c.cpu().numpy().view(np.uint64), oc)


@pytest.mark.parametrize("n,r", [(300_007, 8), (70_001, 16), (5, 32), (10_000_019, 8), (3_000_017, 32)])
def test_stage_sort_groups_by_bucket(n, r):
    seed, layer = 77, 1
    keys, vals = _kv(n, r, seed=n)
    m = O.layer_slots(n, 1.015)
    sk, sv, bs = burr.stage_sort(keys, vals, r, seed, layer, m)
    sk, sv, bs = _u64(sk), _vals_np(sv), bs.cpu().numpy().astype(np.int64)
    nb = (m - 64 + 128) // 128
    assert bs[0] == 0 and bs[-1] == n and np.all(np.diff(bs) >= 0) and len(bs) == nb + 1
    starts, _ = O.hash_many(sk, O.layer_seed(seed, layer), m)
    bucket_of_pos = np.repeat(np.arange(nb), np.diff(bs))
    assert np.array_equal(starts // 128, bucket_of_pos)
    # same (key, value) pairs
    ok, ov = _u64(keys), _vals_np(vals)
    a = np.lexsort((ov, ok))
    b = np.lexsort((sv, sk))
    assert np.array_equal(ok[a], sk[b]) and np.array_equal(ov[a], sv[b])


def _check_build(n, r, seed=I.KEY_SEED, flags=0, **params):
    keys, vals = _kv(n, r, seed=seed)
    h = burr.build(keys, vals, r, flags=flags, **params)
    got = h.export()
    names = {"load_factor": "alpha", "fallback_max_retries": "fb_max_retries", "fallback_slack": "fb_slack",
             "bucket_slots": "B"}
    ref = O.build(_u64(keys), _vals_np(vals), r=r, **{names.get(k, k): v for k, v in params.items()})
    assert ref.ok
    want = ref.export()
    assert got == want, describe_difference(got, want)
    if n:
        assert torch.equal(h.query(keys), vals)
    return h, ref, keys, vals


BUILD_CASES = [
    (0, 8, {}), (1, 8, {}), (2, 1, {}), (100, 3, {}),
    (5000, 8, dict(partition_slots=1024, min_partition_slots=1024)),
    (65573, 8, dict(partition_slots=4096, min_partition_slots=4096)),       # ragged tail
    (1 << 20, 8, {}),                                                       # 2^20, P = 2^16
    (200_003, 16, dict(partition_slots=8192, min_partition_slots=8192)),
    (100_000, 32, dict(partition_slots=2048, min_partition_slots=2048)),
    (150_001, 1, dict(partition_slots=4096, min_partition_slots=0)),
    (70_000, 5, dict(partition_slots=384, min_partition_slots=0)),
    (90_000, 4, dict(partition_slots=128, min_partition_slots=0)),          # a cut at every bucket
    (300_000, 8, dict(lower_partition_slots=0, min_partition_slots=65536)),  # deep layers as layer 0
    (400_000, 8, dict(partition_slots=16384, lower_partition_slots=256, min_partition_slots=256)),
    (22_736, 8, dict(partition_slots=4096, min_partition_slots=4096)),      # remainder 2048: own partition
    (22_672, 8, dict(partition_slots=4096, min_partition_slots=4096)),      # remainder 1984: joins the last
]


@pytest.mark.parametrize("n,r,params", BUILD_CASES)
def test_build_matches_oracle(n, r, params):
    _check_build(n, r, **params)


@pytest.mark.parametrize("alpha,P", [(1.3, 256), (1.6, 4096), (2.2, 1024), (0.8, 65536)])
def test_overloaded_layers_match_oracle(alpha, P):
    h, ref, *_ = _check_build(60_000, 8, load_factor=alpha, partition_slots=P, min_partition_slots=0)
    if alpha >= 1.6:
        codes = set()
        for L in parse(h.export())["layers"]:
            for wd in L["thresh"]:
                codes |= {(int(wd) >> (2 * i)) & 3 for i in range(32)}
        assert codes == {0, 1, 2, 3}


@pytest.mark.parametrize("layers", [0, 1, 2, 8])
def test_layer_count_and_base_case(layers):
    _check_build(30_000, 8, layers=layers, partition_slots=2048, min_partition_slots=2048)


def test_negative_queries_match_oracle():
    h, ref, keys, vals = _check_build(1 << 18, 8, partition_slots=8192, min_partition_slots=8192)
    neg = I.keys_torch(1 << 18, DEV, offset=1 << 18)
    assert np.array_equal(_vals_np(h.query(neg)), ref.query(_u64(neg)))


def test_host_pointers():
    n, r = 50_000, 16
    keys, vals = _kv(n, r)
    hd = burr.build(keys, vals, r, partition_slots=4096)
    hh = burr.build(_u64(keys), vals.cpu().numpy().view(np.uint16), r, partition_slots=4096)
    assert hd.export() == hh.export()
    out = hh.query(_u64(keys))
    assert isinstance(out, np.ndarray) and np.array_equal(out.astype(np.uint32), _vals_np(vals))


def test_determinism():
    keys, vals = _kv(300_000, 8)
    a = burr.build(keys, vals, 8).export()
    b = burr.build(keys, vals, 8).export()
    assert a == b


def test_duplicate_keys_are_unsolvable():
    keys, vals = _kv(10_000, 8)
    keys[5] = keys[9]
    vals[5] = vals[9]
    with pytest.raises(burr.BurrError) as e:
        burr.build(keys, vals, 8, fallback_max_retries=2)
    assert e.value.code == burr.ERR_UNSOLVABLE


@pytest.mark.parametrize("bad", [dict(ribbon_width=32), dict(bucket_slots=96), dict(partition_slots=100),
                                 dict(levels=(0, 32, 64, 100)), dict(load_factor=0.0), dict(layers=9)])
def test_invalid_params(bad):
    keys, vals = _kv(100, 8)
    with pytest.raises(burr.BurrError) as e:
        burr.build(keys, vals, 8, **bad)
    assert e.value.code == burr.ERR_INVALID


def test_invalid_r():
    keys, vals = _kv(100, 8)
    for r in (0, 33):
        with pytest.raises(burr.BurrError):
            burr.build(keys, vals, r)


# 1+-bit thresholds (Sec. 2): exact per-bucket thresholds, exports bit-equal

ONEP_CASES = [
    (0, 8, {}), (1, 8, {}), (100, 3, {}),
    (65573, 8, dict(partition_slots=4096, min_partition_slots=4096)),       # ragged tail
    (1 << 20, 8, {}),
    (200_003, 16, dict(partition_slots=8192, min_partition_slots=8192)),
    (100_000, 32, dict(partition_slots=2048, min_partition_slots=2048)),
    (90_000, 4, dict(partition_slots=128, min_partition_slots=0)),          # a cut at every bucket
    (30_000, 8, dict(layers=1, partition_slots=2048, min_partition_slots=2048)),
]


@pytest.mark.parametrize("n,r,params", ONEP_CASES)
def test_1plus_build_matches_oracle(n, r, params):
    _check_build(n, r, threshold_mode=burr.THRESH_1PLUS, **params)


@pytest.mark.parametrize("alpha,P", [(1.3, 256), (1.6, 4096), (2.2, 1024), (0.8, 65536)])
def test_1plus_overloaded_layers_match_oracle(alpha, P):
    h, ref, *_ = _check_build(60_000, 8, threshold_mode=burr.THRESH_1PLUS, load_factor=alpha,
                              partition_slots=P, min_partition_slots=0)
    if alpha >= 1.6:
        from tests.export_format import exact_thresholds
        t = np.concatenate([exact_thresholds(L) for L in parse(h.export())["layers"] if L["nb"]])
        assert set(np.unique(t)) - {0, 32, 64, 128}        # thresholds between the 2-bit levels


def test_1plus_10m_whole_structure_and_space():
    n, r = 10_000_000, 8
    keys, vals = _kv(n, r, seed=99)
    h1 = burr.build(keys, vals, r, threshold_mode=burr.THRESH_1PLUS)
    ref = O.build(_u64(keys), _vals_np(vals), r=r, threshold_mode=O.THRESH_1PLUS)
    got, want = h1.export(), ref.export()
    assert got == want, describe_difference(got, want)
    assert torch.equal(h1.query(keys), vals)
    neg = I.keys_torch(1 << 20, DEV, seed=99, offset=n)
    assert np.array_equal(_vals_np(h1.query(neg)), ref.query(_u64(neg)))
    h2 = burr.build(keys, vals, r)
    assert h1.size_bytes() < h2.size_bytes()               # the point of 1+-bit thresholds


# Layers sorted in two scatter passes (more than 2^16 buckets) go into bins
# of fixed capacity (mean + 8 standard deviations) instead of counted ones;
# FLAG_TEST_SLACK halves the bins, so every such layer overflows and is sorted
# and banded again with exact counts.  The structure must not change, and
# plain builds of these sizes take the fixed-capacity path without a redo.
SLACK_CASES = [
    (9_000_000, 8, {}),
    (8_700_001, 3, dict(partition_slots=24576, min_partition_slots=0)),
    (9_500_000, 8, dict(threshold_mode=burr.THRESH_1PLUS)),
]


@pytest.mark.parametrize("n,r,params", SLACK_CASES)
def test_sort_bin_overflow_is_sorted_again_exactly(n, r, params):
    h, ref, keys, vals = _check_build(n, r, seed=n, flags=burr.FLAG_TEST_SLACK, **params)
    plain = burr.build(keys, vals, r, **params)
    assert h.export() == plain.export()
    # the redo's kernels: the overflowing attempt and the exact one
    assert h.stats()["kernel_launches"] > plain.stats()["kernel_launches"] + 6


def test_host_inputs_streamed_into_the_sort():
    """Host keys and values of a layer sorted with fixed-capacity bins are
    copied in chunks of 2^24 keys, each taken by the sort's first pass as it
    arrives: same structure as from device memory (3 chunks and a ragged one;
    pinned and pageable host memory; keys on the host with values on the
    device)."""
    n, r = 3 * (1 << 24) + 12345, 8
    keys, vals = _kv(n, r, seed=321)
    want = burr.build(keys, vals, r).export()
    hk, hv = keys.cpu(), vals.cpu()
    assert burr.build(hk, hv, r).export() == want
    assert burr.build(hk.pin_memory(), hv.pin_memory(), r).export() == want
    assert burr.build(hk.pin_memory(), vals, r).export() == want


@pytest.mark.parametrize("mode", [burr.THRESH_2BIT, burr.THRESH_1PLUS])
def test_split_band_matches_oracle(mode):
    """A layer of 4096 or more partitions bands in two launches started
    together (90% of the partitions, then the rest on a second stream), the
    first launch's back-substitution beside the second; small launches read
    three slots ahead, large ones two.  4.5*10^6 keys with 1024-slot
    partitions give ~4,400 layer-0 partitions."""
    _check_build(4_500_000, 8, seed=45, partition_slots=1024, min_partition_slots=1024, threshold_mode=mode)


# Cut-point search (Sec. 3): cuts moved by the library's search kernel give
# the same structure as the oracle's search

CUT_CASES = [
    (300_000, dict(partition_slots=8192)),
    (200_003, dict(partition_slots=2048, min_partition_slots=2048, cut_search_range=7)),
    (90_000, dict(partition_slots=1024, lower_partition_slots=512, min_partition_slots=512,
                  threshold_mode=burr.THRESH_1PLUS)),
    (120_000, dict(partition_slots=384, lower_partition_slots=256, min_partition_slots=0, load_factor=1.3)),
]


@pytest.mark.parametrize("mode", [burr.CUT_MINBUMP, burr.CUT_MAXPREV, burr.CUT_DIFF])
@pytest.mark.parametrize("n,params", CUT_CASES)
def test_cut_search_matches_oracle(mode, n, params):
    _check_build(n, 8, cut_search=mode, **params)


def test_cut_search_10m_whole_structure():
    n, r = 10_000_000, 8
    keys, vals = _kv(n, r, seed=5)
    h = burr.build(keys, vals, r, cut_search=burr.CUT_DIFF)
    ref = O.build(_u64(keys), _vals_np(vals), r=r, cut_search=O.CUT_DIFF)
    got, want = h.export(), ref.export()
    assert got == want, describe_difference(got, want)
    plain = burr.build(keys, vals, r)
    assert h.size_bytes() <= plain.size_bytes()


@pytest.mark.parametrize("pinned", [False, True])
def test_large_host_query_is_pipelined_and_exact(pinned):
    # more than two 2^22-key chunks through host memory: chunks alternate
    # between two streams; results equal the device-pointer query
    keys, vals = _kv(1 << 20, 8, seed=21)
    h = burr.build(keys, vals, 8)
    q = torch.cat([keys, I.keys_torch(9_000_000, DEV, seed=21, offset=1 << 20)])
    want = h.query(q).cpu().numpy()
    qh = q.cpu()
    out = torch.empty(q.numel(), dtype=torch.uint8)
    if pinned:
        qh, out = qh.pin_memory(), out.pin_memory()
    got = h.query(qh.numpy().view(np.uint64), out=out.numpy())
    assert np.array_equal(got, want)
    assert np.array_equal(got[: 1 << 20], vals.cpu().numpy())



QUERY_STRIDE = 9728 * 256   # threads of the largest query grid: keys a thread's walk steps over


@pytest.mark.parametrize("r", [1, 8, 16])
def test_query_lengths_around_the_grid_stride(r):
    """A query thread takes keys i, i + stride, ... and reads its next key
    while the current one's table reads are in flight: lengths just below, at
    and above one and two strides answer as the oracle does, key by key
    (members and negatives interleaved)."""
    keys, vals = _kv(1 << 20, r, seed=77)
    h = burr.build(keys, vals, r)
    ref = O.build(_u64(keys), _vals_np(vals), r=r)
    assert ref.ok
    neg = I.keys_torch(1 << 20, DEV, seed=77, offset=1 << 20)
    pool = torch.stack([keys, neg], dim=1).reshape(-1)          # member, negative, member, ...
    want_pool = np.stack([_vals_np(vals), ref.query(_u64(neg)).astype(np.uint32)], axis=1).reshape(-1)
    for L in (QUERY_STRIDE - 1, QUERY_STRIDE, QUERY_STRIDE + 1, 2 * QUERY_STRIDE + 3):
        idx = torch.arange(L, device=DEV) % pool.numel()
        got = _vals_np(h.query(pool[idx]))
        assert np.array_equal(got, want_pool[idx.cpu().numpy()]), L



# Buckets of 64 start slots (the forced level after a cut is the whole bucket)

@pytest.mark.parametrize("n,r,params", [
    (100_000, 8, dict(partition_slots=4096, min_partition_slots=4096)),
    (70_001, 3, dict(partition_slots=1024, min_partition_slots=0, levels=(0, 8, 40, 64))),
    (50_000, 16, dict(threshold_mode=burr.THRESH_1PLUS, partition_slots=2048, min_partition_slots=2048)),
    (80_000, 8, dict(cut_search=burr.CUT_DIFF, partition_slots=2048, min_partition_slots=2048)),
])
def test_64_slot_buckets_match_oracle(n, r, params):
    params = dict(params)
    params.setdefault("levels", (0, 16, 32, 64))
    _check_build(n, r, bucket_slots=64, **params)


@pytest.mark.parametrize("mode", [burr.THRESH_2BIT, burr.THRESH_1PLUS])
def test_band_window_overflow_is_an_error(mode):
    """A pivot past the band's on-chip window is reported (BURR_ERR_INTERNAL),
    never turned into a wrong table.  BURR_FLAG_TEST_WINDOW shrinks the window
    to 136 slots past the bucket's first slot, which ordinary layers exceed, so
    the path runs without a real overflow; the library stays usable after it."""
    keys, vals = _kv(1 << 18, 8, seed=31)
    with pytest.raises(burr.BurrError) as e:
        burr.build(keys, vals, 8, threshold_mode=mode, flags=burr.FLAG_TEST_WINDOW)
    assert e.value.code == burr.ERR_INTERNAL and "window" in str(e.value)
    _check_build(1 << 18, 8, seed=31, threshold_mode=mode)
