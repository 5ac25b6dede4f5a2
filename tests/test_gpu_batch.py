"""Batched build (many independent structures in one pass of launches).

Each structure of a batch follows the single-structure rules, so its export
must equal burr_build of the same keys with the same parameters (and that one
equals the serial CPU oracle); queries of each structure return its values.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_12365_gb300 import inputs as I
from tests.export_format import describe_difference

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_12365_gb300 import burr  # noqa: E402


def _batch_inputs(sizes, rs, seed=7):
    keys = I.keys_torch(int(sum(sizes)), "cuda", seed=seed)
    vals = I.values_torch(keys, max(rs))
    # each structure's values masked to its own width
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return keys, vals, offs


def _check_batch(sizes, rs, **params):
    keys, vals, offs = _batch_inputs(sizes, rs)
    hs = burr.build_batch(keys, vals, offs, rs, **params)
    P = hs[0].export()[56:64] if False else None  # noqa: F841
    for s, h in enumerate(hs):
        a, b = int(offs[s]), int(offs[s + 1])
        k, v = keys[a:b], vals[a:b]
        p = burr.default_params(**params)
        ex = h.export()
        if params.get("partition_slots", 1) == 0:
            # the chosen P is recorded in the export header (u64 after seed, alpha bits, n)
            chosen = int(np.frombuffer(ex[64:72], dtype=np.uint64)[0])
            p = burr.default_params(**{**params, "partition_slots": chosen, "min_partition_slots": chosen})
        vt = burr.value_torch_dtype(rs[s])
        vs = (v.to(torch.int64) & ((1 << rs[s]) - 1)).to(vt) if vt != vals.dtype or rs[s] < 8 else v
        solo = burr.build(k, vs, rs[s], params=p).export()
        assert ex == solo, f"structure {s}: {describe_difference(ex, solo)}"
        if b > a:
            got = h.query(k).cpu().numpy().astype(np.int64) & ((1 << rs[s]) - 1)
            want = vs.cpu().numpy().astype(np.int64) & ((1 << rs[s]) - 1)
            assert np.array_equal(got, want)
    return hs, keys, vals, offs


def test_batch_small_mixed():
    rng = np.random.default_rng(1)
    sizes = [int(x) for x in np.exp(rng.uniform(np.log(100), np.log(30000), size=40))]
    sizes[3] = 0                       # an empty structure
    sizes[7] = 1
    rs = [int(x) for x in rng.choice([1, 2, 3, 4, 8], size=len(sizes))]
    _check_batch(sizes, rs, partition_slots=4096, min_partition_slots=4096)


def test_batch_matches_oracle():
    sizes = [5000, 123, 70000, 2]
    rs = [8, 3, 1, 4]
    hs, keys, vals, offs = _check_batch(sizes, rs, partition_slots=2048, min_partition_slots=2048)
    k_np = keys.cpu().numpy().view(np.uint64)
    v_np = vals.cpu().numpy().astype(np.uint32)
    for s in range(len(sizes)):
        a, b = int(offs[s]), int(offs[s + 1])
        ref = O.build(k_np[a:b], v_np[a:b] & ((1 << rs[s]) - 1), r=rs[s], partition_slots=2048,
                      min_partition_slots=2048)
        assert ref.ok and hs[s].export() == ref.export(), s


def test_batch_autotuned_partition_size_and_large_structures():
    rng = np.random.default_rng(2)
    sizes = [int(x) for x in np.exp(rng.uniform(np.log(1000), np.log(600000), size=12))]
    rs = [8] * len(sizes)
    hs, *_ = _check_batch(sizes, rs, partition_slots=0)
    chosen = {int(np.frombuffer(h.export()[64:72], dtype=np.uint64)[0]) for h in hs}
    assert len(chosen) == 1 and chosen.pop() in (16384, 32768, 65536)


def test_batch_base_case_heavy():
    # few bumping layers: every structure ends in the base case, some retry
    sizes = [3000, 40, 500, 12000]
    rs = [8, 8, 2, 8]
    _check_batch(sizes, rs, layers=1, partition_slots=1024, min_partition_slots=1024)


@pytest.mark.parametrize("mode", [burr.THRESH_2BIT, burr.THRESH_1PLUS])
def test_batch_with_split_band(mode):
    """A batch layer of 4096 or more partitions bands in two launches (the
    first 90% of the longest-first order, then the rest on a second stream),
    the first launch's back-substitution beside the second, and each layer's
    back-substitution runs beside the next layer over rotating band arrays:
    every structure still equals its solo build."""
    rng = np.random.default_rng(8)
    sizes = [int(x) for x in np.exp(rng.uniform(np.log(2000), np.log(60000), size=300))]
    rs = [int(x) for x in rng.choice([1, 4, 8], size=len(sizes))]
    assert sum(sizes) * 1.015 / 1024 > 4096 + 300          # partitions of layer 0
    _check_batch(sizes, rs, partition_slots=1024, min_partition_slots=1024, threshold_mode=mode)


def test_batch_rejects_too_large_structure():
    keys = I.keys_torch(9_000_000, "cuda")
    vals = I.values_torch(keys, 8)
    with pytest.raises(burr.BurrError) as e:
        burr.build_batch(keys, vals, [0, 9_000_000], [8])
    assert e.value.code == burr.ERR_INVALID


def test_batch_1plus_thresholds():
    # each structure of a 1+-bit batch equals its solo build and the oracle
    rng = np.random.default_rng(5)
    sizes = [int(x) for x in np.exp(rng.uniform(np.log(100), np.log(60000), size=30))]
    sizes[4] = 0
    rs = [int(x) for x in rng.choice([1, 3, 8], size=len(sizes))]
    hs, keys, vals, offs = _check_batch(sizes, rs, partition_slots=2048, min_partition_slots=2048,
                                        threshold_mode=burr.THRESH_1PLUS)
    k_np = keys.cpu().numpy().view(np.uint64)
    v_np = vals.cpu().numpy().astype(np.uint32)
    for s in (0, 7, len(sizes) - 1):
        a, b = int(offs[s]), int(offs[s + 1])
        ref = O.build(k_np[a:b], v_np[a:b] & ((1 << rs[s]) - 1), r=rs[s], partition_slots=2048,
                      min_partition_slots=2048, threshold_mode=O.THRESH_1PLUS)
        assert hs[s].export() == ref.export(), describe_difference(hs[s].export(), ref.export())


def test_batch_cut_search():
    rng = np.random.default_rng(6)
    sizes = [int(x) for x in np.exp(rng.uniform(np.log(100), np.log(200_000), size=25))]
    rs = [int(x) for x in rng.choice([2, 8], size=len(sizes))]
    hs, keys, vals, offs = _check_batch(sizes, rs, partition_slots=2048, min_partition_slots=2048,
                                        cut_search=burr.CUT_MAXPREV)
    k_np = keys.cpu().numpy().view(np.uint64)
    v_np = vals.cpu().numpy().astype(np.uint32)
    big = int(np.argmax(sizes))
    a, b = int(offs[big]), int(offs[big + 1])
    ref = O.build(k_np[a:b], v_np[a:b] & ((1 << rs[big]) - 1), r=rs[big], partition_slots=2048,
                  min_partition_slots=2048, cut_search=O.CUT_MAXPREV)
    assert hs[big].export() == ref.export(), describe_difference(hs[big].export(), ref.export())


def test_free_all_releases_a_batch_in_one_call():
    # burr_free_many: every handle of a batched build released with one call;
    # the wrappers are marked freed, so neither free() nor a second free_all()
    # touches them again, and a fresh batch builds the same structures
    sizes = [5000, 0, 1, 40_000, 12_345]
    rs = [8, 4, 8, 1, 3]
    keys, vals, offs = _batch_inputs(sizes, rs)
    hs = burr.build_batch(keys, vals, offs, rs, partition_slots=4096, min_partition_slots=4096)
    exports = [h.export() for h in hs]
    burr.free_all(hs)
    assert all(h._h is None for h in hs)
    burr.free_all(hs)
    for h in hs:
        h.free()
    hs2 = burr.build_batch(keys, vals, offs, rs, partition_slots=4096, min_partition_slots=4096)
    assert [h.export() for h in hs2] == exports
    burr.free_all(hs2[:2])
    assert hs2[0]._h is None and hs2[2]._h is not None
    for h in hs2:
        h.free()
