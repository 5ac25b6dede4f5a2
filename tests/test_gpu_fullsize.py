"""GPU parity at the benchmark's sizes: 10^9 keys (r = 1, 8, 16) and 10^8 keys.

At 10^9 keys the GPU structure is compared with the oracle part by part:
  * layer 0, every partition: the oracle builds the layer's partitions in
    groups (all keys of a group of consecutive partitions, with the layer's
    cuts; partitions are independent once the cuts are placed, Sec. 3) and
    each group's thresholds and table words must equal the GPU's;
  * the bumped keys of those groups are layer 1's input, and every deeper
    layer and the base case are built whole by the oracle and compared;
  * query(x) = f(x) for every key, and negatives hit at rate 2^-r.
The oracle runs with each layer's partitions spread over the host's cores
(tests/test_oracle_threaded.py ties that to the serial oracle).  At 10^8
keys the whole export is compared at once.  The pivots' distance from their
rows' starts (the oracle's max_drift) is checked against the band kernel's
on-chip window in both threshold modes.
"""
import concurrent.futures as cf
import os

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

SEED = 0x5EED5EED5EED5EED      # the library's and the oracle's default hash seed
ALPHA = 1.015
P0, PL = 65536, 4096           # partition slots of layer 0 and of deeper layers
THREADS = os.cpu_count() or 1
N9 = 1_000_000_000
WINDOW = 509                   # band kernel: 512-slot ring less its deepest read-ahead (3 slots)
B = 128


def _mem_available_gb():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / (1 << 20)
    except OSError:
        pass
    return 0.0


def _vals32(v):
    a = v.cpu().numpy()
    return a.view({1: np.uint8, 2: np.uint16, 4: np.uint32}[a.dtype.itemsize])


def _hash_starts(keys, sigma, m):
    """Start slot of every key (uint32), by the oracle's hash, on all cores
    (ctypes releases the GIL during each chunk)."""
    starts = np.empty(len(keys), dtype=np.uint32)
    step = 1 << 24

    def one(lo):
        s, _ = O.hash_many(keys[lo:lo + step], sigma, m)
        starts[lo:lo + step] = s

    with cf.ThreadPoolExecutor(THREADS) as ex:
        list(ex.map(one, range(0, len(keys), step)))
    return starts


@pytest.fixture(scope="module")
def keys9():
    if _mem_available_gb() < 80:
        pytest.skip("the 10^9-key comparison needs about 80 GB of host memory")
    k = I.keys_torch(N9, "cuda")
    host = k.cpu().numpy().view(np.uint64)
    del k
    torch.cuda.empty_cache()
    m0 = O.layer_slots(N9, ALPHA)
    starts = _hash_starts(host, O.layer_seed(SEED, 0), m0)
    return host, starts, m0


def _compare_deeper_layers(ex, k1, v1, r, mode=O.THRESH_2BIT):
    """Layers 1.. and the base case, built whole by the oracle from layer 1's
    input keys, against the GPU export."""
    layers = ex["layers"]
    cur_k, cur_v = k1, v1
    for l in range(1, len(layers)):
        L = layers[l]
        n = len(cur_k)
        assert L["n"] == n, f"layer {l}: {L['n']} keys on the GPU, {n} by the oracle"
        if n == 0:
            break
        m = O.layer_slots(n, ALPHA)
        K = O.num_partitions(m, PL, 4096)
        assert (L["m"], L["parts"]) == (m, K)
        res = O.build_layer(cur_k, cur_v, r, m, O.layer_seed(SEED, l), cuts=[j * PL for j in range(1, K)],
                            mode=mode, threads=THREADS)
        assert res.status == 0
        assert np.array_equal(res.thresh, L["thresh"]), f"layer {l} thresholds differ"
        assert np.array_equal(res.z, L["z"]), f"layer {l} table differs"
        assert L["bumped"] == len(res.bumped_keys)
        cur_k, cur_v = res.bumped_keys, res.bumped_vals
    F = ex["fallback"]
    assert F["n"] == len(cur_k)
    if len(cur_k):
        for a in range(17):
            m = O.fallback_slots(len(cur_k), 0.1, 64, a)
            res = O.build_layer(cur_k, cur_v, r, m, O.layer_seed(SEED, len(layers) + a), fallback=True)
            if res.status == 0:
                break
        assert res.status == 0 and (F["attempt"], F["m"], F["seed_index"]) == (a, m, len(layers) + a)
        assert np.array_equal(res.z, F["z"]), "base-case table differs"


@pytest.mark.parametrize("r", [8, 1, 16])
def test_1e9_every_partition_and_every_layer_match_oracle(keys9, r):
    """n = 10^9, w = 64, 2-bit thresholds, P = 2^16 (the benchmark's launch)."""
    k_np, starts, m0 = keys9
    kd = torch.from_numpy(k_np.view(np.int64)).cuda()
    vd = I.values_torch(kd, r)
    h = burr.build(kd, vd, r)
    assert torch.equal(h.query(kd), vd), "query(x) != f(x)"
    neg = I.keys_torch(1 << 22, "cuda", offset=N9)
    hits = int((h.query(neg) == I.values_torch(neg, r)).sum())
    mean = (1 << 22) / 2.0 ** r
    assert abs(hits - mean) < 6 * (mean * (1 - 2.0 ** -r)) ** 0.5
    ex = parse(h.export())
    v_np = _vals32(vd)
    del kd, vd, neg, h
    torch.cuda.empty_cache()

    L0 = ex["layers"][0]
    K = O.num_partitions(m0, P0, 4096)
    assert (L0["n"], L0["m"], L0["parts"]) == (N9, m0, K)
    cuts = [j * P0 for j in range(1, K)]
    sigma0 = O.layer_seed(SEED, 0)
    part = np.minimum(starts >> 16, K - 1).astype(np.uint32)          # P0 = 2^16
    groups = 8
    per = -(-K // groups)
    bumped_k, bumped_v, drift = [], [], 0
    for g in range(groups):
        j0, j1 = g * per, min((g + 1) * per, K)
        idx = np.flatnonzero((part >= j0) & (part < j1))
        res = O.build_layer(k_np[idx], v_np[idx].astype(np.uint32), r, m0, sigma0, cuts=cuts, threads=THREADS)
        assert res.status == 0
        # thresholds of the group's buckets (a partition is 512 buckets = 16 whole words)
        w0, w1 = j0 * P0 // B // 32, (L0["nb"] + 31) // 32 if j1 == K else j1 * P0 // B // 32
        assert np.array_equal(res.thresh[w0:w1], L0["thresh"][w0:w1]), f"layer-0 thresholds, partitions {j0}..{j1}"
        # table words of the slots the group's partitions own
        s0 = 0 if j0 == 0 else j0 * P0 + 64
        s1 = m0 if j1 == K else j1 * P0 + 64
        z0, z1 = (s0 // 64) * r, (s1 // 64) * r
        assert np.array_equal(res.z[z0:z1], L0["z"][z0:z1]), f"layer-0 table, partitions {j0}..{j1}"
        bumped_k.append(res.bumped_keys)
        bumped_v.append(res.bumped_vals)
        drift = max(drift, res.stats.max_drift)
        del idx, res
    k1, v1 = np.concatenate(bumped_k), np.concatenate(bumped_v)
    assert L0["bumped"] == len(k1)
    # every pivot stayed well inside the band kernel's window: a row starts at
    # most B-1 slots past its bucket's first slot
    assert drift + (B - 1) < WINDOW, f"max drift {drift}"
    _compare_deeper_layers(ex, k1, v1, r)


def test_1e9_pivot_drift_inside_the_band_window_1plus(keys9):
    """1+-bit thresholds keep more rows per bucket, so the band is denser:
    the oracle's largest pivot distance on 10^9-key layer-0 partitions
    (two groups of 256 partitions) must still leave the window room."""
    k_np, starts, m0 = keys9
    K = O.num_partitions(m0, P0, 4096)
    part = np.minimum(starts >> 16, K - 1)
    for j0 in (0, K // 2):
        idx = np.flatnonzero((part >= j0) & (part < j0 + 256))
        # values do not move pivots (a row fails when its coefficients vanish), so zeros stand in
        res = O.build_layer(k_np[idx], np.zeros(len(idx), np.uint32), 8, m0, O.layer_seed(SEED, 0),
                            cuts=[j * P0 for j in range(1, K)], mode=O.THRESH_1PLUS, threads=THREADS)
        assert res.status == 0
        assert res.stats.max_drift + (B - 1) < WINDOW, f"max drift {res.stats.max_drift}"


@pytest.mark.parametrize("n,r,seed", [(100_000_000, 8, I.KEY_SEED), (10_000_000, 8, 77), (10_000_000, 16, 78)])
def test_whole_structure_2bit_matches_oracle(n, r, seed):
    """Every byte of the export: sizes, thresholds and tables of every layer
    and the base case (10^8 keys is the second benchmark configuration)."""
    kd = I.keys_torch(n, "cuda", seed=seed)
    vd = I.values_torch(kd, r)
    h = burr.build(kd, vd, r)
    got = h.export()
    assert torch.equal(h.query(kd), vd)
    k_np = kd.cpu().numpy().view(np.uint64)
    ref = O.build(k_np, _vals32(vd).astype(np.uint32), r=r, threads=THREADS)
    assert ref.ok
    want = ref.export()
    assert got == want, describe_difference(got, want)
    st = h.stats()
    for l in range(4):
        assert st["layer_m"][l] == O.layer_slots(st["layer_n"][l], ALPHA)
    neg = I.keys_torch(1 << 20, "cuda", seed=seed, offset=n)
    assert np.array_equal(_vals32(h.query(neg)).astype(np.uint32), ref.query(neg.cpu().numpy().view(np.uint64)))
