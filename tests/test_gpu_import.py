"""Checkpoint/resume: burr_export -> burr_import gives the same structure.

A handle imported from an export answers every query like the original, and
its own export is byte-identical.  Tables built by the serial CPU oracle,
loaded with burr_import, are queried by the GPU kernel and give the oracle's
answers (members and non-members).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_12365_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_12365_gb300 import burr  # noqa: E402


@pytest.mark.parametrize("n,r,params", [
    (0, 8, {}), (1, 8, {}), (200_000, 8, {}),
    (150_000, 1, dict(partition_slots=4096)),
    (100_000, 16, dict(threshold_mode=burr.THRESH_1PLUS)),
    (80_000, 32, dict(bucket_slots=64, levels=(0, 16, 32, 64), partition_slots=2048, min_partition_slots=2048)),
    (60_000, 8, dict(layers=0)),
    (120_000, 8, dict(cut_search=burr.CUT_DIFF, partition_slots=4096)),
])
def test_roundtrip(n, r, params):
    keys = I.keys_torch(n, "cuda", seed=n + r)
    vals = I.values_torch(keys, r)
    h = burr.build(keys, vals, r, **params)
    ex = h.export()
    g = burr.import_export(ex)
    assert g.export() == ex
    q = torch.cat([keys, I.keys_torch(50_000, "cuda", seed=n + r, offset=n)])
    assert torch.equal(g.query(q), h.query(q))


@pytest.mark.parametrize("mode,cut", [(O.THRESH_2BIT, O.CUT_NONE), (O.THRESH_1PLUS, O.CUT_NONE),
                                      (O.THRESH_2BIT, O.CUT_MAXPREV)])
def test_oracle_tables_queried_on_the_gpu(mode, cut):
    n, r = 300_000, 8
    k = I.keys_np(n, seed=17)
    v = I.values_np(k, r).astype(np.uint32)
    ref = O.build(k, v, r=r, partition_slots=8192, min_partition_slots=8192, threshold_mode=mode, cut_search=cut)
    h = burr.import_export(ref.export())
    neg = I.keys_np(200_000, seed=17, offset=n)
    for q in (k, neg):
        got = h.query(torch.from_numpy(q.view(np.int64)).cuda()).cpu().numpy().astype(np.uint32)
        assert np.array_equal(got, ref.query(q))
