"""The allocation-free bucket sort (burr_stage_sort_noalloc) against the
allocating one (burr_stage_sort), through the C ABI.

Some callers cannot let a library allocate device memory: their device memory
belongs to their own pool allocator, or they run in a latency-critical loop
that cannot take cudaMalloc's implicit synchronisation.  The allocation-free
entry point keeps its scratch in one fixed device array instead.  Its result
must be the allocating sort's result: identical bucket offsets and, since the
order inside a bucket is free, the same (key, value) pairs in every bucket.
Two calls in a row check that the previous call's leftovers in the shared
array do not leak into the next one.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_2411_12365_gb300 import burr  # noqa: E402
from paper_2411_12365_gb300 import inputs as I  # noqa: E402

MAX_KEYS = 1 << 20


def _noalloc(keys, vals, r, seed, layer, m):
    L = burr.load()
    n = keys.numel()
    nb = (m - 64 + 128) // 128
    sk = torch.empty_like(keys)
    sv = torch.empty_like(vals)
    bs = torch.empty(nb + 1, dtype=torch.int32, device=keys.device)
    st = torch.cuda.current_stream().cuda_stream
    rc = L.burr_stage_sort_noalloc(C.c_void_p(keys.data_ptr()), C.c_void_p(vals.data_ptr()), n, r, seed, layer,
                                   m, C.c_void_p(sk.data_ptr()), C.c_void_p(sv.data_ptr()),
                                   C.c_void_p(bs.data_ptr()), st)
    return rc, sk, sv, bs


def _per_bucket_pairs(sk, sv, bs):
    k = sk.cpu().numpy().view(np.uint64)
    a = sv.cpu().numpy()
    v = a.view({1: np.uint8, 2: np.uint16, 4: np.uint32}[a.dtype.itemsize]).astype(np.uint64)
    b = np.repeat(np.arange(len(bs) - 1), np.diff(bs.cpu().numpy().astype(np.int64)))
    order = np.lexsort((v, k, b))
    return b[order], k[order], v[order]


MAX_SLOTS = 1 << 24


# (n, r, seed, layer, m): m None = the layer size of n keys.  m = 2^24 (the
# largest layer allowed) has 2048 sort groups, which takes the two-pass plan
# and fills the static array's group counters to their limit.
@pytest.mark.parametrize("calls", [[(MAX_KEYS, 8, 11, 0, None), (300_007, 8, 12, 1, None)],
                                   [(70_001, 16, 13, 2, None), (MAX_KEYS, 32, 14, 0, None)],
                                   [(MAX_KEYS, 8, 15, 0, MAX_SLOTS), (5000, 16, 16, 3, MAX_SLOTS)]])
def test_noalloc_sort_equals_allocating_sort(calls):
    for n, r, seed, layer, m in calls:               # two calls in a row
        keys = I.keys_torch(n, "cuda", seed=seed)
        vals = I.values_torch(keys, r)
        m = m or O.layer_slots(n, 1.015)
        rc, sk, sv, bs = _noalloc(keys, vals, r, seed, layer, m)
        assert rc == 0, burr.load().burr_last_error().decode()
        rk, rv, rb = burr.stage_sort(keys, vals, r, seed, layer, m)
        torch.cuda.synchronize()
        assert torch.equal(bs, rb)
        for x, y in zip(_per_bucket_pairs(sk, sv, bs), _per_bucket_pairs(rk, rv, rb)):
            assert np.array_equal(x, y)


def test_noalloc_rejects_too_many_keys():
    keys = torch.zeros(1, dtype=torch.int64, device="cuda")
    vals = torch.zeros(1, dtype=torch.uint8, device="cuda")
    L = burr.load()
    bs = torch.empty(16, dtype=torch.int32, device="cuda")
    rc = L.burr_stage_sort_noalloc(C.c_void_p(keys.data_ptr()), C.c_void_p(vals.data_ptr()), MAX_KEYS + 1, 8,
                                   1, 0, 1024, C.c_void_p(keys.data_ptr()), C.c_void_p(vals.data_ptr()),
                                   C.c_void_p(bs.data_ptr()), None)
    assert rc == burr.ERR_INVALID
    assert "allocation-free limit" in L.burr_last_error().decode()


def test_noalloc_rejects_too_many_slots():
    keys = torch.zeros(1, dtype=torch.int64, device="cuda")
    vals = torch.zeros(1, dtype=torch.uint8, device="cuda")
    L = burr.load()
    bs = torch.empty(16, dtype=torch.int32, device="cuda")
    rc = L.burr_stage_sort_noalloc(C.c_void_p(keys.data_ptr()), C.c_void_p(vals.data_ptr()), 1, 8, 1, 0,
                                   MAX_SLOTS + 64, C.c_void_p(keys.data_ptr()), C.c_void_p(vals.data_ptr()),
                                   C.c_void_p(bs.data_ptr()), None)
    assert rc == burr.ERR_INVALID
    assert "allocation-free limit" in L.burr_last_error().decode()


def test_noalloc_sort_allocates_nothing():
    """Every device allocation of the library goes through the allocator hook,
    so a counting allocator sees none during the allocation-free sort (and
    some during the allocating one, which shows the count works)."""
    import gc
    gc.collect()
    torch.cuda.synchronize()
    calls = []
    dev = torch.cuda.current_device()

    def alloc(nbytes, stream):
        calls.append(nbytes)
        return torch.cuda.caching_allocator_alloc(nbytes, dev, stream)

    burr.set_allocator(alloc, lambda ptr, stream: torch.cuda.caching_allocator_delete(ptr))
    try:
        n, r = 200_003, 8
        keys = I.keys_torch(n, "cuda", seed=17)
        vals = I.values_torch(keys, r)
        m = O.layer_slots(n, 1.015)
        for _ in range(2):
            rc, *_ = _noalloc(keys, vals, r, 17, 0, m)
            assert rc == 0, burr.load().burr_last_error().decode()
        torch.cuda.synchronize()
        assert calls == []
        burr.stage_sort(keys, vals, r, 17, 0, m)
        torch.cuda.synchronize()
        assert calls
    finally:
        burr.set_allocator(None, None)
