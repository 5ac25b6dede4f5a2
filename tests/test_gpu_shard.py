"""Sharded construction on the GPU (Sec. 3: partitions are independent once
the cuts are placed).  K ranks run as threads of this process, each a shard
of the one GPU: the library routes every rank's keys to the owners of their
start buckets, the exchange is a device copy, every rank bands and
back-substitutes its own partition range, and rank 0 builds the base case and
writes the export.  The merged export must equal the single-GPU build of all
keys byte for byte, for K in {2, 3, 4} and uneven splits; imported, it answers
every key."""
import numpy as np
import pytest

from paper_2411_12365_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_12365_gb300 import burr  # noqa: E402
from paper_2411_12365_gb300 import shard  # noqa: E402
from tests.export_format import describe_difference  # noqa: E402


def _split(keys, vals, ranks, uneven):
    n = keys.numel()
    if not uneven:
        return [keys[g::ranks].contiguous() for g in range(ranks)], [vals[g::ranks].contiguous() for g in range(ranks)]
    cut = np.sort(np.random.default_rng(ranks + n).choice(n + 1, ranks - 1)).tolist()
    b = [0] + cut + [n]
    return [keys[b[g]:b[g + 1]] for g in range(ranks)], [vals[b[g]:b[g + 1]] for g in range(ranks)]


CASES = [
    (1_000_000, 8, {}, 2, False),
    (1_000_000, 8, {}, 4, True),
    (10_000_000, 8, {}, 4, False),                    # 152 layer-0 partitions
    (3_000_017, 16, dict(partition_slots=8192, min_partition_slots=8192), 3, True),
    (500_000, 1, dict(partition_slots=1024, lower_partition_slots=256, min_partition_slots=256), 4, False),
    (200_000, 8, dict(partition_slots=384, min_partition_slots=0, load_factor=1.6), 3, False),
    (20_000, 8, {}, 4, False),                        # ranks without partitions
]


@pytest.mark.parametrize("n,r,pk,ranks,uneven", CASES)
def test_sharded_build_equals_single_gpu_build(n, r, pk, ranks, uneven):
    keys = I.keys_torch(n, "cuda", seed=n + 5)
    vals = I.values_torch(keys, r)
    want = burr.build(keys, vals, r, **pk).export()
    ks, vs = _split(keys, vals, ranks, uneven)
    got = shard.build_sharded_virtual(ks, vs, r, **pk)
    assert got == want, describe_difference(got, want)
    h = burr.import_export(got)
    assert torch.equal(h.query(keys), vals)


def test_sharded_rejects_what_it_does_not_support():
    keys = I.keys_torch(1000, "cuda")
    vals = I.values_torch(keys, 8)
    for bad in (dict(threshold_mode=burr.THRESH_1PLUS), dict(cut_search=burr.CUT_DIFF)):
        with pytest.raises(burr.BurrError) as e:
            shard.build_sharded_virtual([keys], [vals], 8, **bad)
        assert e.value.code == burr.ERR_INVALID
