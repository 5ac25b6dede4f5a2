"""burr_import rejects malformed export buffers before touching the device.

The buffers are the oracle's exports (2-bit and 1+-bit) with one field
broken at a time; every check runs on the host, so this runs without a GPU.
"""
import ctypes as C
import os
import struct

import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_12365_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def burr():
    from paper_2411_12365_gb300 import build as B
    from paper_2411_12365_gb300 import burr as mod
    B.build()
    mod.load(os.path.join(ROOT, "paper_2411_12365_gb300", "_lib", "libburr.so"))
    return mod


def _export(mode):
    k = I.keys_np(20_000)
    v = I.values_np(k, 8).astype(np.uint32)
    s = O.build(k, v, r=8, partition_slots=2048, min_partition_slots=2048, threshold_mode=mode)
    return s.export()


def _code(burr, buf):
    out = C.c_void_p()
    b = (C.c_uint8 * max(len(buf), 1)).from_buffer_copy(bytes(buf) or b"\0")
    return burr.load().burr_import(b, len(buf), None, C.byref(out))


def _patch(buf, off, fmt, value):
    b = bytearray(buf)
    struct.pack_into(fmt, b, off, value)
    return bytes(b)


@pytest.mark.parametrize("mode", [O.THRESH_2BIT, O.THRESH_1PLUS])
def test_malformed_exports_are_rejected(burr, mode):
    good = _export(mode)
    hdr = 10 * 4 + 4 * 8
    bad = {
        "empty": b"",
        "truncated header": good[:20],
        "magic": _patch(good, 0, "<I", 0x12345678),
        "version": _patch(good, 4, "<I", 3),
        "r": _patch(good, 8, "<I", 0),
        "ribbon width": _patch(good, 12, "<I", 32),
        "layers": _patch(good, 20, "<I", 9),
        "truncated body": good[:-8],
        "trailing bytes": good + b"\0" * 8,
        "layer-0 keys": _patch(good, hdr, "<Q", 19_999),
        "layer-0 slots": _patch(good, hdr + 8, "<Q", 12345),
        "base-case seed index": _patch(good, hdr + 4 * 40 + 16, "<Q", 99),
        "layer-0 no partitions": _patch(good, hdr + 16, "<Q", 0),
        "layer-0 more partitions than buckets": _patch(
            good, hdr + 16, "<Q", struct.unpack_from("<Q", good, hdr + 24)[0] + 1),
    }
    if mode == O.THRESH_1PLUS:
        # first threshold section follows the base-case record
        nb0 = struct.unpack_from("<Q", good, hdr + 24)[0]
        cnt_off = hdr + 4 * 40 + 32 + 8 * ((nb0 + 63) // 64)
        cnt = struct.unpack_from("<Q", good, cnt_off)[0]
        bad["flag count"] = _patch(good, cnt_off, "<Q", cnt + 1)
        bad["threshold 0"] = _patch(good, cnt_off + 8, "<B", 0)
        bad["threshold > B"] = _patch(good, cnt_off + 8, "<B", 200)
    for what, buf in bad.items():
        assert _code(burr, buf) == burr.ERR_INVALID, what
