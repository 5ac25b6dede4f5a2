"""Brute-force re-derivation of one BuRR layer from its definition (test helper).

Given the oracle's per-bucket thresholds, this recomputes with dense GF(2)
algebra (``gf2.py``), independently of the oracle's elimination code:

* the kept set of each bucket is {keys whose offset >= its threshold} and the
  kept set of the layer is linearly independent (Sec. 2: bumped keys leave the
  system so that it becomes solvable);
* every threshold is minimal among the four 2-bit levels: the next lower level
  would make the system dependent (the insertion bumps only on failure);
* the first bucket after each cut bumps at least w-1 slots (Sec. 3, Bumping);
* no kept equation overlaps a cut: each support lies inside one partition's
  slot range (Sec. 3, Fig. 2);
* the bumped keys are exactly the rows below their bucket's threshold;
* the table equals the unique solution of the kept system with every free
  slot set to 0, computed by Gauss-Jordan elimination.

``check_layer_1plus`` does the same for 1+-bit thresholds (Sec. 2, threshold
storage: a bit per bucket, the exact threshold of every bucket that bumps):
each threshold t is the least value for which the bucket's rows at offsets
>= t are independent of the rows kept before, so one less (a row sits there)
is dependent; after a cut t >= w.
"""
from __future__ import annotations

from collections import defaultdict

from oracle import oracle as O
from tests.gf2 import EchelonBasis, solve_free_zero


def unpack_z(z, r, m):
    """Slot values from the interleaved layout: bit k of slot s is bit s%64 of
    word (s//64)*r + k."""
    out = [0] * m
    for s in range(m):
        base = (s // 64) * r
        v = 0
        for k in range(r):
            v |= ((int(z[base + k]) >> (s % 64)) & 1) << k
        out[s] = v
    return out


def codes_of(thresh, nb):
    return [(int(thresh[b // 32]) >> (2 * (b % 32))) & 3 for b in range(nb)]


def check_layer(keys, vals, r, m, sigma, cuts, levels=(0, 32, 64, 128), B=128, w=64):
    keys = [int(k) for k in keys]
    vals = [int(v) & ((1 << r) - 1) for v in vals]
    res = O.build_layer(keys, vals, r, m, sigma, cuts=cuts, levels=levels, B=B, w=w)
    assert res.status == 0, res.status
    nb = O.num_buckets(m, w, B)
    codes = codes_of(res.thresh, nb)
    eqs = [O.hash_key(k, sigma, m, w) for k in keys]
    forced = next(i for i, l in enumerate(levels) if l >= w)
    cut_buckets = {c // B for c in cuts}
    bounds = [0] + [c + w for c in cuts] + [m]          # ownership boundaries
    by_bucket = defaultdict(list)
    for i, (s, _) in enumerate(eqs):
        by_bucket[s // B].append(i)

    def row(i):
        s, c = eqs[i]
        return c << s

    basis = EchelonBasis()
    kept_all, bumped_expect = [], []
    for b in range(nb):
        floor_code = forced if b in cut_buckets else 0
        assert codes[b] >= floor_code, (b, codes[b])
        t = levels[codes[b]]
        rows_b = by_bucket.get(b, [])
        kept = [i for i in rows_b if eqs[i][0] % B >= t]
        trial = basis.copy()
        for i in kept:
            assert trial.add(row(i)), f"bucket {b}: kept rows dependent"
        if codes[b] > floor_code:
            lower = levels[codes[b] - 1]
            probe = basis.copy()
            ok = True
            for i in rows_b:
                if eqs[i][0] % B >= lower and not probe.add(row(i)):
                    ok = False
                    break
            assert not ok, f"bucket {b}: threshold {t} is not minimal"
        basis = trial
        kept_all += kept
        bumped_expect += [keys[i] for i in rows_b if eqs[i][0] % B < t]
    assert sorted(int(k) for k in res.bumped_keys) == sorted(bumped_expect)

    # supports stay inside one partition's owned slot range
    for i in kept_all:
        s, c = eqs[i]
        hi = s + c.bit_length() - 1
        j = max(q for q in range(len(bounds) - 1) if bounds[q] <= s)
        assert bounds[j] <= s and hi < bounds[j + 1], (s, hi, bounds[j], bounds[j + 1])

    z_dense = solve_free_zero([row(i) for i in kept_all], [vals[i] for i in kept_all], m)
    assert z_dense is not None
    assert unpack_z(res.z, r, m) == z_dense
    return res, codes


def check_layer_1plus(keys, vals, r, m, sigma, cuts, B=128, w=64):
    keys = [int(k) for k in keys]
    vals = [int(v) & ((1 << r) - 1) for v in vals]
    res = O.build_layer(keys, vals, r, m, sigma, cuts=cuts, B=B, w=w, mode=O.THRESH_1PLUS)
    assert res.status == 0, res.status
    nb = O.num_buckets(m, w, B)
    t_of = [int(x) for x in res.texact]
    assert len(t_of) == nb
    eqs = [O.hash_key(k, sigma, m, w) for k in keys]
    cut_buckets = {c // B for c in cuts}
    bounds = [0] + [c + w for c in cuts] + [m]
    by_bucket = defaultdict(list)
    for i, (s, _) in enumerate(eqs):
        by_bucket[s // B].append(i)

    def row(i):
        s, c = eqs[i]
        return c << s

    basis = EchelonBasis()
    kept_all, bumped_expect = [], []
    for b in range(nb):
        floor = w if b in cut_buckets else 0
        t = t_of[b]
        assert floor <= t <= B, (b, t)
        rows_b = by_bucket.get(b, [])
        kept = [i for i in rows_b if eqs[i][0] % B >= t]
        trial = basis.copy()
        for i in kept:
            assert trial.add(row(i)), f"bucket {b}: kept rows dependent"
        if t > floor:
            below = [i for i in rows_b if eqs[i][0] % B == t - 1]
            assert below, f"bucket {b}: threshold {t} has no row at offset {t - 1}"
            probe = trial.copy()
            assert not all(probe.add(row(i)) for i in below), f"bucket {b}: threshold {t} is not minimal"
        basis = trial
        kept_all += kept
        bumped_expect += [keys[i] for i in rows_b if eqs[i][0] % B < t]
    assert sorted(int(k) for k in res.bumped_keys) == sorted(bumped_expect)
    for i in kept_all:
        s, c = eqs[i]
        hi = s + c.bit_length() - 1
        j = max(q for q in range(len(bounds) - 1) if bounds[q] <= s)
        assert bounds[j] <= s and hi < bounds[j + 1], (s, hi, bounds[j], bounds[j + 1])
    z_dense = solve_free_zero([row(i) for i in kept_all], [vals[i] for i in kept_all], m)
    assert z_dense is not None
    assert unpack_z(res.z, r, m) == z_dense
    return res, t_of
