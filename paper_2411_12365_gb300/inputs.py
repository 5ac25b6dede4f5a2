"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the retrieval method.  Keys and values come
from MurmurHash3's 64-bit finalizer ``fmix64`` (Appleby), used here purely as a
counter-based generator: ``key_i = fmix64(seed + i)``.  ``fmix64`` is a
bijection, so keys drawn from disjoint counter ranges are distinct; negative
query keys use the counters ``[n, 2n)``.  The stored value of a key (an r-bit
fingerprint, the filter use of the paper's experiments) is the low r bits of
``fmix64(key ^ value_seed)``.

Two implementations with identical output: numpy (host) and torch int64 ops
(any device, so 10^9 keys can be produced directly in device memory).
"""
from __future__ import annotations

import numpy as np

_M1 = 0xFF51AFD7ED558CCD
_M2 = 0xC4CEB9FE1A85EC53
_MASK = (1 << 64) - 1

KEY_SEED = 0x0123456789ABCDEF
VALUE_SEED = 0x7F4A7C159E3779B9


def value_dtype(r: int):
    """Smallest unsigned type holding r bits (u8, u16, u32)."""
    if not 1 <= r <= 32:
        raise ValueError("r must be in [1, 32]")
    return np.uint8 if r <= 8 else (np.uint16 if r <= 16 else np.uint32)


def fmix64_np(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        x ^= x >> np.uint64(33)
        x *= np.uint64(_M1)
        x ^= x >> np.uint64(33)
        x *= np.uint64(_M2)
        x ^= x >> np.uint64(33)
    return x


def keys_np(n: int, seed: int = KEY_SEED, offset: int = 0) -> np.ndarray:
    with np.errstate(over="ignore"):
        ctr = np.arange(offset, offset + n, dtype=np.uint64) + np.uint64(seed & _MASK)
    return fmix64_np(ctr)


def values_np(keys: np.ndarray, r: int, seed: int = VALUE_SEED) -> np.ndarray:
    h = fmix64_np(np.asarray(keys, dtype=np.uint64) ^ np.uint64(seed & _MASK))
    mask = np.uint64((1 << r) - 1)
    return (h & mask).astype(value_dtype(r))


# --- torch variant (int64 storage, same bits) -------------------------------

def _s64(c: int) -> int:
    c &= _MASK
    return c - (1 << 64) if c >= (1 << 63) else c


def _shr(x, k: int):
    import torch  # noqa: F401
    return (x >> k) & ((1 << (64 - k)) - 1)


def fmix64_torch(x):
    x = x ^ _shr(x, 33)
    x = x * _s64(_M1)
    x = x ^ _shr(x, 33)
    x = x * _s64(_M2)
    x = x ^ _shr(x, 33)
    return x


def keys_torch(n: int, device, seed: int = KEY_SEED, offset: int = 0, chunk: int = 1 << 26):
    """int64 tensor holding the same 64-bit patterns as ``keys_np``."""
    import torch
    out = torch.empty(n, dtype=torch.int64, device=device)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        ctr = torch.arange(offset + a, offset + b, dtype=torch.int64, device=device) + _s64(seed)
        out[a:b] = fmix64_torch(ctr)
    return out


def values_torch(keys, r: int, seed: int = VALUE_SEED, chunk: int = 1 << 26):
    """Values with the bit patterns of ``values_np`` in uint8 / int16 / int32 storage."""
    import torch
    vt = value_dtype(r)
    dt, bits = {np.uint8: (torch.uint8, 8), np.uint16: (torch.int16, 16),
                np.uint32: (torch.int32, 32)}[vt]
    out = torch.empty(keys.numel(), dtype=dt, device=keys.device)
    mask = (1 << r) - 1
    for a in range(0, keys.numel(), chunk):
        b = min(keys.numel(), a + chunk)
        h = fmix64_torch(keys[a:b] ^ _s64(seed)) & mask
        if bits < 64 and dt != torch.uint8:
            h = h - ((h >> (bits - 1)) & 1) * (1 << bits)   # two's-complement view
        out[a:b] = h.to(dt)
    return out
