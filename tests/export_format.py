"""Parser of the canonical export format (declared in include/burr.h), used by
the tests to report where two exports differ."""
import struct

import numpy as np


def parse(buf: bytes):
    hdr = struct.unpack_from("<10I4Q", buf, 0)
    magic, version, r, w, B, layers = hdr[:6]
    assert magic == 0x52525542 and version in (1, 2)   # 1: 2-bit thresholds, 2: 1+-bit
    off = 10 * 4 + 4 * 8
    L = []
    for _ in range(layers):
        n, m, parts, nb, bumped = struct.unpack_from("<5Q", buf, off)
        off += 40
        L.append(dict(n=n, m=m, parts=parts, nb=nb, bumped=bumped))
    fn, fm, fseed, fatt = struct.unpack_from("<4Q", buf, off)
    off += 32
    for d in L:
        if version == 1:
            tw = (d["nb"] + 31) // 32
            d["thresh"] = np.frombuffer(buf, dtype=np.uint64, count=tw, offset=off)
            off += 8 * tw
        else:
            fw = (d["nb"] + 63) // 64
            d["flags"] = np.frombuffer(buf, dtype=np.uint64, count=fw, offset=off)
            off += 8 * fw
            (cnt,) = struct.unpack_from("<Q", buf, off)
            off += 8
            d["exact"] = np.frombuffer(buf, dtype=np.uint8, count=cnt, offset=off)
            off += 8 * ((cnt + 7) // 8)
            # the whole section as words, for comparisons
            d["thresh"] = np.concatenate([d["flags"], np.array([cnt], np.uint64),
                                          np.frombuffer(buf, dtype=np.uint64, count=(cnt + 7) // 8,
                                                        offset=off - 8 * ((cnt + 7) // 8))])
        zw = (d["m"] // 64) * r
        d["z"] = np.frombuffer(buf, dtype=np.uint64, count=zw, offset=off)
        off += 8 * zw
    zw = (fm // 64) * r
    fz = np.frombuffer(buf, dtype=np.uint64, count=zw, offset=off)
    off += 8 * zw
    assert off == len(buf)
    return dict(r=r, w=w, B=B, version=version, layers=L,
                fallback=dict(n=fn, m=fm, seed_index=fseed, attempt=fatt, z=fz), header=hdr)


def exact_thresholds(layer) -> np.ndarray:
    """Per-bucket thresholds of a 1+-bit layer from its flags and stored bytes."""
    nb = layer["nb"]
    flags = np.unpackbits(layer["flags"].view(np.uint8), bitorder="little")[:nb].astype(bool)
    t = np.zeros(nb, dtype=np.int64)
    t[flags] = layer["exact"]
    return t


def describe_difference(a: bytes, b: bytes) -> str:
    if a == b:
        return "identical"
    pa, pb = parse(a), parse(b)
    if pa["header"] != pb["header"]:
        return f"headers differ: {pa['header']} vs {pb['header']}"
    out = []
    for i, (x, y) in enumerate(zip(pa["layers"], pb["layers"])):
        meta = {k: x[k] for k in ("n", "m", "parts", "nb", "bumped")}
        metb = {k: y[k] for k in ("n", "m", "parts", "nb", "bumped")}
        if meta != metb:
            out.append(f"layer {i} sizes {meta} vs {metb}")
            continue
        dt = np.nonzero(x["thresh"] != y["thresh"])[0]
        dz = np.nonzero(x["z"] != y["z"])[0]
        if len(dt):
            out.append(f"layer {i}: {len(dt)} threshold words differ, first word {dt[0]}")
        if len(dz):
            out.append(f"layer {i}: {len(dz)} table words differ, first word {dz[0]} (slot block {dz[0] // pa['r']})")
    fa, fb = pa["fallback"], pb["fallback"]
    if (fa["n"], fa["m"], fa["seed_index"], fa["attempt"]) != (fb["n"], fb["m"], fb["seed_index"], fb["attempt"]):
        out.append(f"base case {fa['n'], fa['m'], fa['seed_index'], fa['attempt']} vs "
                   f"{fb['n'], fb['m'], fb['seed_index'], fb['attempt']}")
    elif not np.array_equal(fa["z"], fb["z"]):
        out.append("base-case table differs")
    return "; ".join(out) or "differ (unknown section)"
