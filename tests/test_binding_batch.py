"""Host logic of the binding's batch container (no GPU): a batched build's
handles are made on access, free_all releases every live structure in one
call, single frees and slices mark the batch, and nothing is freed twice."""
import ctypes as C
import gc

import numpy as np
import pytest

from paper_2411_12365_gb300 import burr


class FakeLib:
    """Records the handle pointers the binding asks the library to free."""

    def __init__(self):
        self.freed = []
        self.many_calls = 0

    def burr_free(self, p):
        self.freed.append(int(p))

    def burr_free_many(self, arr, n):
        # a numpy pointer array's address, or a ctypes array of pointers
        self.many_calls += 1
        if isinstance(arr, int):
            ptrs = C.cast(C.c_void_p(arr), C.POINTER(C.c_uint64))
            self.freed.extend(int(ptrs[i]) for i in range(n))
        else:
            self.freed.extend(int(arr[i]) for i in range(n))


@pytest.fixture
def lib(monkeypatch):
    gc.collect()
    fake = FakeLib()
    monkeypatch.setattr(burr, "_lib", fake)
    yield fake
    gc.collect()


def batch(n):
    return burr.HandleBatch(np.arange(1, n + 1, dtype=np.uint64), [8] * n)


def test_free_all_of_a_batch_is_one_call(lib):
    hs = batch(10_000)
    h0 = hs[0]
    burr.free_all(hs)
    assert lib.many_calls == 1 and sorted(lib.freed) == list(range(1, 10_001))
    assert h0._h is None and hs[9_999]._h is None
    burr.free_all(hs)
    h0.free()
    assert len(lib.freed) == 10_000


def test_slices_and_single_frees_mark_the_batch(lib):
    hs = batch(5)
    burr.free_all(hs[:2])
    assert sorted(lib.freed) == [1, 2]
    assert hs[0]._h is None and hs[2]._h == 3
    for h in hs:
        h.free()
    del hs
    gc.collect()
    assert sorted(lib.freed) == [1, 2, 3, 4, 5]


def test_a_kept_handle_keeps_its_batch(lib):
    hs = batch(4)
    keep = hs[2]
    del hs
    gc.collect()
    assert lib.freed == [] and keep._h == 3
    del keep
    gc.collect()
    assert sorted(lib.freed) == [1, 2, 3, 4]


def test_sequence_behaviour(lib):
    hs = batch(3)
    assert len(hs) == 3 and hs[-1]._h == 3 and hs[np.int64(1)]._h == 2
    assert hs[1] is hs[1]
    with pytest.raises(IndexError):
        hs[3]
    out = []
    out += hs
    assert [h._h for h in out] == [1, 2, 3] and [h.r for h in hs] == [8, 8, 8]
    del out, hs
    gc.collect()
    assert sorted(lib.freed) == [1, 2, 3]
