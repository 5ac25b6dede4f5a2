"""Pins of the oracle's hashing step (Sec. 2: each key gives an equation whose
coefficients lie in a w-wide window starting at its start slot).

The paper leaves the hash to the SEA'22 BuRR paper; the reading used here is
SplitMix64's output function (Steele, Lea, Flood 2014) plus Lemire's
multiply-shift range reduction.  These tests pin it against the published
SplitMix64 stream, against an independently derived inverse, and against the
arithmetic definition of the range reduction.
"""
import random

import pytest

from oracle import oracle as O

M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def test_splitmix64_known_answers():
    # SplitMix64 seeded with 0 returns mix(k * GOLDEN) for k = 1, 2, ...; its
    # first outputs are widely published test vectors.
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    got = [O.mix64((k * GOLDEN) & M64) for k in range(1, 5)]
    assert got == expect


def _unxorshift(y, k):
    x = y
    for _ in range(64 // k + 1):
        x = y ^ (x >> k)
    return x & M64


def _inverse_mix(z):
    z = _unxorshift(z, 31)
    z = (z * pow(0x94D049BB133111EB, -1, 1 << 64)) & M64
    z = _unxorshift(z, 27)
    z = (z * pow(0xBF58476D1CE4E5B9, -1, 1 << 64)) & M64
    return _unxorshift(z, 30)


def test_mixer_is_a_bijection():
    rng = random.Random(1)
    for _ in range(2000):
        x = rng.getrandbits(64)
        assert _inverse_mix(O.mix64(x)) == x
    for x in (0, 1, M64, 1 << 63):
        assert _inverse_mix(O.mix64(x)) == x


@pytest.mark.parametrize("m", [64, 128, 192, 1 << 12, 1_015_872, (1 << 32) - 64])
def test_start_is_multiply_shift_range_reduction(m):
    rng = random.Random(m)
    sigma = O.layer_seed(7, 0)
    for _ in range(500):
        key = rng.getrandbits(64)
        s, c = O.hash_key(key, sigma, m)
        h = O.mix64(key ^ sigma)
        assert s == (h * (m - 63)) >> 64          # floor(h * range / 2^64)
        assert 0 <= s <= m - 64                   # window [s, s+63] inside [0, m)
        assert c & 1 == 1                         # first coefficient is always 1


def test_start_slots_are_uniform():
    # chi-square over 64 equal cells of the start range
    m = 64 * 65
    sigma = O.layer_seed(3, 1)
    rng = random.Random(5)
    cells = [0] * 64
    N = 64 * 400
    for _ in range(N):
        s, _ = O.hash_key(rng.getrandbits(64), sigma, m)
        cells[min(63, s * 64 // (m - 63))] += 1
    e = N / 64
    chi2 = sum((x - e) ** 2 / e for x in cells)
    assert chi2 < 120  # 63 d.o.f.; p < 1e-5 for larger values


def test_layer_seeds_differ():
    seeds = {O.layer_seed(0x1234, l) for l in range(32)}
    assert len(seeds) == 32
