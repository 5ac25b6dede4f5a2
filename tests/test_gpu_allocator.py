"""Device memory through the caller's allocator (burr_set_allocator).

PyTorch's caching allocator backs every build, query and batched build; the
results equal those of the built-in pool, the tables of a live handle sit in
PyTorch's pool, the allocator cannot be changed while blocks are held, and
every block comes back.
"""
import numpy as np
import pytest

from paper_2411_12365_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_12365_gb300 import burr  # noqa: E402


def test_torch_caching_allocator_backs_the_library():
    keys = I.keys_torch(300_000, "cuda", seed=77)
    vals = I.values_torch(keys, 8)
    offs = [0, 1000, 50_000, 300_000]
    bp = dict(partition_slots=4096, min_partition_slots=4096, threshold_mode=burr.THRESH_1PLUS)
    ref = burr.build(keys, vals, 8, partition_slots=8192)
    ref_ex = ref.export()
    ref.free()
    refs_b = burr.build_batch(keys, vals, offs, [8, 8, 8], **bp)
    ref_bex = [h.export() for h in refs_b]
    del refs_b
    torch.cuda.synchronize()

    count = {"alloc": 0, "free": 0, "live": 0}
    dev = torch.cuda.current_device()

    def alloc(n, stream):
        count["alloc"] += 1
        count["live"] += 1
        return torch.cuda.caching_allocator_alloc(n, dev, stream)

    def free(ptr, stream):
        count["free"] += 1
        count["live"] -= 1
        torch.cuda.caching_allocator_delete(ptr)

    base = torch.cuda.memory_allocated()
    burr.set_allocator(alloc, free)
    handles = []
    try:
        h = burr.build(keys, vals, 8, partition_slots=8192)
        handles.append(h)
        assert h.export() == ref_ex
        assert torch.cuda.memory_allocated() - base >= h.size_bytes() - 64   # tables in torch's pool
        assert torch.equal(h.query(keys), vals)
        out = h.query(keys.cpu().numpy().view(np.uint64))                     # host pointers: staged
        assert np.array_equal(out, vals.cpu().numpy())
        hs = burr.build_batch(keys, vals, offs, [8, 8, 8], **bp)
        handles += hs
        assert [x.export() for x in hs] == ref_bex
        with pytest.raises(burr.BurrError):
            burr.set_allocator(None, None)                                    # blocks still held
        assert count["live"] > 0
    finally:
        for x in handles:
            x.free()
        handles.clear()
        hs = None
        torch.cuda.synchronize()
    assert count["alloc"] > 0 and count["live"] == 0 and count["alloc"] == count["free"]
    burr.set_allocator(None, None)
    # the built-in pool again
    h2 = burr.build(keys, vals, 8, partition_slots=8192)
    assert h2.export() == ref_ex
    h2.free()


@pytest.mark.parametrize("which", ["first", "middle", "last"])
@pytest.mark.parametrize("kind", ["plain", "batch", "1plus"])
def test_allocation_failure_is_clean(which, kind):
    # host-side fault injection: the caller's allocator refuses one request;
    # the call fails with BURR_ERR_OOM and every block it got is given back
    keys = I.keys_torch(200_000, "cuda", seed=5)
    vals = I.values_torch(keys, 8)
    dev = torch.cuda.current_device()

    def run():
        if kind == "plain":
            return [burr.build(keys, vals, 8, partition_slots=8192)]
        if kind == "1plus":
            return [burr.build(keys, vals, 8, threshold_mode=burr.THRESH_1PLUS)]
        return burr.build_batch(keys, vals, [0, 70_000, 200_000], [8, 8], partition_slots=4096,
                                min_partition_slots=4096)

    count = {"alloc": 0, "free": 0, "fail_at": 0}

    def alloc(n, stream):
        count["alloc"] += 1
        if count["alloc"] == count["fail_at"]:
            return 0
        return torch.cuda.caching_allocator_alloc(n, dev, stream)

    def free(ptr, stream):
        count["free"] += 1
        torch.cuda.caching_allocator_delete(ptr)

    burr.set_allocator(alloc, free)
    try:
        hs = run()                                  # count the allocations of one call
        total = count["alloc"]
        for h in hs:
            h.free()
        del hs
        torch.cuda.synchronize()
        assert count["free"] == total
        count.update(alloc=0, free=0, fail_at={"first": 1, "middle": total // 2, "last": total}[which])
        code = None
        try:
            run()
        except burr.BurrError as err:
            code = err.code
        assert code == burr.ERR_OOM
        torch.cuda.synchronize()
        assert count["free"] == count["alloc"] - 1  # all but the refused request came back
    finally:
        burr.set_allocator(None, None)
    hs = run()                                      # the library works normally afterwards
    if kind != "batch":
        assert torch.equal(hs[0].query(keys[:1000]), vals[:1000])
    for h in hs:
        h.free()


@pytest.mark.parametrize("r", [8, 16])
def test_tables_off_32_byte_boundaries_take_the_narrow_query(r):
    # A caller's allocator may return blocks that are 16-byte aligned but not
    # 32-byte aligned.  The query then reads table windows in 8-byte loads
    # instead of 32-byte ones; the answers and the export are unchanged.
    keys = I.keys_torch(400_000, "cuda", seed=91)
    vals = I.values_torch(keys, r)
    ref = burr.build(keys, vals, r, partition_slots=8192)
    ref_ex = ref.export()
    want = ref.query(keys)
    ref.free()
    dev = torch.cuda.current_device()
    shifted = {}

    def alloc(n, stream):
        p = torch.cuda.caching_allocator_alloc(n + 64, dev, stream)
        q = (p + 31) // 32 * 32 + 16          # 16 bytes past a 32-byte boundary
        shifted[q] = p
        return q

    def free(ptr, stream):
        torch.cuda.caching_allocator_delete(shifted.pop(ptr))

    burr.set_allocator(alloc, free)
    h = None
    try:
        h = burr.build(keys, vals, r, partition_slots=8192)
        assert h.export() == ref_ex
        assert torch.equal(h.query(keys), want)
        assert torch.equal(h.query(keys[::7]), want[::7])
    finally:
        if h is not None:
            h.free()
        torch.cuda.synchronize()
        burr.set_allocator(None, None)
    assert not shifted
