"""ctypes wrapper of the serial C oracle (``burr_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  The CUDA library never imports, links or
calls anything in this directory.

The oracle computes what the paper's method computes, step by step and
serially (Sec. 2 ribbon equations and bumping, Sec. 3 bumping at partition
boundaries, Sec. 4 layers and base case); see the C file for the readings of
the points the paper leaves to the SEA'22 BuRR paper.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "burr_oracle.c")
_HDR = os.path.join(_HERE, "burr_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libburr_oracle.so")

MAX_LAYERS = 8
EINVAL, ENOMEM, UNSOLVABLE, FAIL = -1, -2, -3, -4
THRESH_2BIT, THRESH_1PLUS = 0, 1
CUT_NONE, CUT_MINBUMP, CUT_MAXPREV, CUT_DIFF = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


def build_lib(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (portable C11, no intrinsics)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [
        ("r", C.c_uint32), ("w", C.c_uint32), ("B", C.c_uint32),
        ("levels", C.c_uint32 * 4), ("alpha", C.c_double),
        ("layers", C.c_uint32), ("fb_max_retries", C.c_uint32),
        ("partition_slots", C.c_uint64), ("min_partition_slots", C.c_uint64),
        ("seed", C.c_uint64), ("fb_slack", C.c_double),
        ("cut_P", C.c_uint64 * MAX_LAYERS), ("threshold_mode", C.c_uint32), ("pad", C.c_uint32),
        ("lower_partition_slots", C.c_uint64), ("cut_search", C.c_uint32), ("cut_search_range", C.c_uint32),
    ]


class Layer(C.Structure):
    _fields_ = [(f, C.c_uint64) for f in
                ("n", "m", "seed_index", "nbuckets", "nparts", "part_slots", "nbumped")] + [
        ("cuts", C.POINTER(C.c_uint64)), ("thresh", C.POINTER(C.c_uint64)), ("z", C.POINTER(C.c_uint64)),
        ("texact", C.POINTER(C.c_uint8))]


class Struct(C.Structure):
    _fields_ = [("params", Params), ("n", C.c_uint64), ("fb_attempt", C.c_uint64),
                ("layer", Layer * (MAX_LAYERS + 1))]


class Stats(C.Structure):
    _fields_ = [("xor_steps", C.c_uint64), ("inserted", C.c_uint64), ("max_drift", C.c_uint64),
                ("bumped", C.c_uint64 * MAX_LAYERS)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB lets the mutation tests load a deliberately broken copy
            L = C.CDLL(os.environ.get("ORACLE_LIB") or build_lib())
            u64, u32, p = C.c_uint64, C.c_uint32, C.c_void_p
            L.or_mix64.restype = u64; L.or_mix64.argtypes = [u64]
            L.or_layer_seed.restype = u64; L.or_layer_seed.argtypes = [u64, u64]
            L.or_hash.restype = None
            L.or_hash.argtypes = [u64, u64, u64, u32, C.POINTER(u64), C.POINTER(u64)]
            L.or_hash_batch.restype = None
            L.or_hash_batch.argtypes = [p, u64, u64, u64, u32, p, p]
            L.or_layer_slots.restype = u64; L.or_layer_slots.argtypes = [u64, C.c_double, u32]
            L.or_fallback_slots.restype = u64
            L.or_fallback_slots.argtypes = [u64, C.c_double, u32, u32]
            L.or_num_buckets.restype = u64; L.or_num_buckets.argtypes = [u64, u32, u32]
            L.or_num_partitions.restype = u64; L.or_num_partitions.argtypes = [u64, u64, u64]
            L.or_build_layer.restype = C.c_int
            L.or_build_layer.argtypes = [p, p, u64, u32, u64, u64, p, u32, u32, p, u64, C.c_int,
                                         p, p, p, p, C.POINTER(u64), C.POINTER(Stats)]
            L.or_build_layer_mode.restype = C.c_int
            L.or_build_layer_mode.argtypes = [p, p, u64, u32, u64, u64, p, u32, u32, p, u64, C.c_int,
                                              u32, p, p, p, p, p, C.POINTER(u64), C.POINTER(Stats)]
            L.or_build_layer_mt.restype = C.c_int
            L.or_build_layer_mt.argtypes = [p, p, u64, u32, u64, u64, p, u32, u32, p, u64, C.c_int,
                                            u32, p, p, p, p, p, C.POINTER(u64), C.POINTER(Stats), C.c_uint]
            L.or_search_cuts.restype = C.c_int
            L.or_search_cuts.argtypes = [p, u64, u64, u64, u32, u32, u64, u64, u32, u32, p]
            L.or_struct_size.restype = u64; L.or_struct_size.argtypes = []
            L.or_params_size.restype = u64; L.or_params_size.argtypes = []
            L.or_layer_size.restype = u64; L.or_layer_size.argtypes = []
            L.or_default_params.restype = None; L.or_default_params.argtypes = [C.POINTER(Params)]
            L.or_build.restype = C.c_int
            L.or_build.argtypes = [p, p, u64, C.POINTER(Params), C.POINTER(Struct), C.POINTER(Stats)]
            L.or_build_mt.restype = C.c_int
            L.or_build_mt.argtypes = [p, p, u64, C.POINTER(Params), C.POINTER(Struct), C.POINTER(Stats),
                                      C.c_uint]
            L.or_free.restype = None; L.or_free.argtypes = [C.POINTER(Struct)]
            L.or_query.restype = None; L.or_query.argtypes = [C.POINTER(Struct), p, p, u64]
            L.or_export.restype = u64; L.or_export.argtypes = [C.POINTER(Struct), p, u64]
            L.or_overhead.restype = C.c_double; L.or_overhead.argtypes = [C.POINTER(Struct)]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def default_params(**kw) -> Params:
    p = Params()
    lib().or_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "levels":
            p.levels = (C.c_uint32 * 4)(*v)
        elif k == "cut_P":
            arr = list(v) + [0] * (MAX_LAYERS - len(v))
            p.cut_P = (C.c_uint64 * MAX_LAYERS)(*arr)
        else:
            setattr(p, k, v)
    return p


def mix64(x: int) -> int:
    return int(lib().or_mix64(x & (2**64 - 1)))


def layer_seed(seed: int, index: int) -> int:
    return int(lib().or_layer_seed(seed, index))


def hash_key(key: int, sigma: int, m: int, w: int = 64):
    s, c = C.c_uint64(), C.c_uint64()
    lib().or_hash(key, sigma, m, w, C.byref(s), C.byref(c))
    return int(s.value), int(c.value)


def hash_many(keys, sigma: int, m: int, w: int = 64):
    """(starts, coeffs) of every key, as uint64 arrays."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    s = np.empty(len(keys), dtype=np.uint64)
    c = np.empty(len(keys), dtype=np.uint64)
    lib().or_hash_batch(_ptr(keys), len(keys), sigma, m, w, _ptr(s), _ptr(c))
    return s, c


def layer_slots(n, alpha, w=64):
    return int(lib().or_layer_slots(n, alpha, w))


def fallback_slots(n, slack, w=64, attempt=0):
    return int(lib().or_fallback_slots(n, slack, w, attempt))


def num_buckets(m, w=64, B=128):
    return int(lib().or_num_buckets(m, w, B))


def num_partitions(m, P, min_slots):
    return int(lib().or_num_partitions(m, P, min_slots))


class LayerResult:
    def __init__(self, status, thresh, z, bumped_keys, bumped_vals, stats, texact=None):
        self.status = status
        self.thresh = thresh
        self.texact = texact
        self.z = z
        self.bumped_keys = bumped_keys
        self.bumped_vals = bumped_vals
        self.stats = stats


def build_layer(keys, vals, r, m, sigma, cuts=(), fallback=False,
                levels=(0, 32, 64, 128), B=128, w=64, mode=THRESH_2BIT, threads=1) -> LayerResult:
    """One layer with an explicit cut list (start slots of partitions 1..K-1).
    mode THRESH_1PLUS gives exact per-bucket thresholds in .texact.  threads > 1
    spreads the partitions over host threads (same result)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    vals = np.ascontiguousarray(vals, dtype=np.uint32)
    n = len(keys)
    nb = num_buckets(m, w, B)
    thresh = np.zeros((nb + 31) // 32 + 1, dtype=np.uint64)
    z = np.zeros((m // 64) * r + 1, dtype=np.uint64)
    bk = np.zeros(max(n, 1), dtype=np.uint64)
    bv = np.zeros(max(n, 1), dtype=np.uint32)
    lv = np.array(levels, dtype=np.uint32)
    cu = np.array(cuts if len(cuts) else [0], dtype=np.uint64)
    nbumped = C.c_uint64()
    st = Stats()
    texact = np.zeros(nb + 1, dtype=np.uint8)
    if threads > 1:
        rc = lib().or_build_layer_mt(_ptr(keys), _ptr(vals), n, r, m, sigma, _ptr(lv), B, w,
                                     _ptr(cu), len(cuts), int(fallback), mode, _ptr(thresh),
                                     _ptr(texact), _ptr(z), _ptr(bk), _ptr(bv), C.byref(nbumped),
                                     C.byref(st), threads)
    elif mode == THRESH_2BIT:
        rc = lib().or_build_layer(_ptr(keys), _ptr(vals), n, r, m, sigma, _ptr(lv), B, w,
                                  _ptr(cu), len(cuts), int(fallback), _ptr(thresh), _ptr(z),
                                  _ptr(bk), _ptr(bv), C.byref(nbumped), C.byref(st))
    else:
        rc = lib().or_build_layer_mode(_ptr(keys), _ptr(vals), n, r, m, sigma, _ptr(lv), B, w,
                                       _ptr(cu), len(cuts), int(fallback), mode, _ptr(thresh),
                                       _ptr(texact), _ptr(z), _ptr(bk), _ptr(bv), C.byref(nbumped),
                                       C.byref(st))
    k = nbumped.value
    return LayerResult(rc, thresh[:(nb + 31) // 32], z[:(m // 64) * r], bk[:k].copy(),
                       bv[:k].copy(), st, texact[:nb].copy() if mode != THRESH_2BIT else None)


class OracleStruct:
    """A built structure: per-layer sizes, thresholds and tables, export and query."""

    def __init__(self, keys, vals, params: Params, threads: int = 1):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        vals = np.ascontiguousarray(vals, dtype=np.uint32)
        self._s = Struct()
        self.stats = Stats()
        self.params = params
        if threads > 1:
            self.status = lib().or_build_mt(_ptr(keys), _ptr(vals), len(keys), C.byref(params),
                                            C.byref(self._s), C.byref(self.stats), threads)
        else:
            self.status = lib().or_build(_ptr(keys), _ptr(vals), len(keys), C.byref(params),
                                         C.byref(self._s), C.byref(self.stats))

    def __del__(self):
        try:
            if getattr(self, "status", -1) == 0:
                lib().or_free(C.byref(self._s))
        except Exception:
            pass

    @property
    def ok(self):
        return self.status == 0

    def layer(self, l):
        """l in [0, layers) or 'fallback'."""
        L = self._s.layer[MAX_LAYERS if l == "fallback" else l]
        r = self.params.r
        nw = (L.nbuckets + 31) // 32
        nz = (L.m // 64) * r
        thresh = (np.ctypeslib.as_array(L.thresh, shape=(nw,)).copy()
                  if (nw and bool(L.thresh) and l != "fallback") else np.zeros(0, np.uint64))
        nc = max(int(L.nparts) - 1, 0)
        cuts = (np.ctypeslib.as_array(L.cuts, shape=(nc,)).copy()
                if (nc and bool(L.cuts) and l != "fallback") else np.zeros(0, np.uint64))
        texact = (np.ctypeslib.as_array(L.texact, shape=(L.nbuckets,)).copy()
                  if (L.nbuckets and bool(L.texact) and l != "fallback") else np.zeros(0, np.uint8))
        z = np.ctypeslib.as_array(L.z, shape=(nz,)).copy() if nz else np.zeros(0, np.uint64)
        return dict(n=L.n, m=L.m, seed_index=L.seed_index, nbuckets=L.nbuckets,
                    nparts=L.nparts, nbumped=L.nbumped, thresh=thresh, z=z, texact=texact, cuts=cuts)

    @property
    def fb_attempt(self):
        return int(self._s.fb_attempt)

    def export(self) -> bytes:
        need = lib().or_export(C.byref(self._s), None, 0)
        buf = (C.c_uint8 * need)()
        got = lib().or_export(C.byref(self._s), buf, need)
        assert got == need
        return bytes(buf)

    def overhead(self) -> float:
        return float(lib().or_overhead(C.byref(self._s)))

    def query(self, keys) -> np.ndarray:
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        out = np.zeros(max(len(keys), 1), dtype=np.uint32)
        lib().or_query(C.byref(self._s), _ptr(keys), _ptr(out), len(keys))
        return out[:len(keys)]


def build(keys, vals, threads: int = 1, **params) -> OracleStruct:
    """The whole structure; threads > 1 spreads each bumping layer's partitions
    over host threads (the paper's parallel construction; same result)."""
    return OracleStruct(keys, vals, default_params(**params), threads=threads)


def search_cuts(keys, m, sigma, P, K, mode, search_range, B=128, w=64) -> np.ndarray:
    """Cut start slots (K-1) chosen by the cut-point search of one layer."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    out = np.zeros(max(K - 1, 1), dtype=np.uint64)
    rc = lib().or_search_cuts(_ptr(keys), len(keys), m, sigma, B, w, P, K, mode, search_range, _ptr(out))
    assert rc == 0
    return out[:max(K - 1, 0)]
