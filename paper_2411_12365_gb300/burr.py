"""Thin Python binding of libburr.so (include/burr.h): argument marshalling only.

Every step of construction and query runs in the library's CUDA kernels.
Inputs may be torch tensors (CUDA or CPU) or numpy arrays; CUDA tensors are
passed as device pointers together with torch's current CUDA stream.  If the
library has not been built, every call raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import operator
import os
import threading
import weakref
from collections.abc import Sequence

import numpy as np

from . import build as _build

BURR_OK = 0
ERR_INVALID, ERR_OOM, ERR_UNSOLVABLE, ERR_TIMEOUT, ERR_CUDA, ERR_INTERNAL = -1, -2, -3, -4, -5, -6
MAX_LAYERS = 8
FLAG_TIMING = 1
FLAG_TEST_WINDOW = 2
FLAG_TEST_SLACK = 4
THRESH_2BIT, THRESH_1PLUS = 0, 1
CUT_NONE, CUT_MINBUMP, CUT_MAXPREV, CUT_DIFF = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


class BurrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"burr error {code}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [
        ("ribbon_width", C.c_uint32), ("bucket_slots", C.c_uint32), ("threshold_mode", C.c_uint32),
        ("layers", C.c_uint32), ("levels", C.c_uint32 * 4), ("load_factor", C.c_double),
        ("partition_slots", C.c_uint64), ("min_partition_slots", C.c_uint64), ("seed", C.c_uint64),
        ("fallback_slack", C.c_double), ("fallback_max_retries", C.c_uint32), ("flags", C.c_uint32),
        ("lower_partition_slots", C.c_uint64), ("cut_search", C.c_uint32), ("cut_search_range", C.c_uint32),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("n", C.c_uint64), ("r", C.c_uint32), ("layers", C.c_uint32),
        ("layer_n", C.c_uint64 * (MAX_LAYERS + 1)), ("layer_m", C.c_uint64 * (MAX_LAYERS + 1)),
        ("layer_parts", C.c_uint64 * (MAX_LAYERS + 1)), ("layer_bumped", C.c_uint64 * (MAX_LAYERS + 1)),
        ("fallback_attempt", C.c_uint32), ("pad", C.c_uint32),
        ("stage_ms", (C.c_float * 3) * (MAX_LAYERS + 1)), ("total_ms", C.c_float), ("pad2", C.c_float),
        ("table_bytes", C.c_uint64), ("kernel_launches", C.c_uint64),
    ]


class LayerGeometry(C.Structure):
    _fields_ = [(f, C.c_uint64) for f in ("n", "m", "buckets", "partitions", "partition_slots", "seed_index")]


class ServerConfig(C.Structure):
    _fields_ = [("memory_budget", C.c_uint64), ("host_staging_bytes", C.c_uint64),
                ("max_batch_structures", C.c_uint32), ("build_workers", C.c_uint32)]


class ServerStats(C.Structure):
    _fields_ = [(f, C.c_uint64) for f in ("bytes_resident", "bytes_inflight", "resident_structures",
                                          "queued_builds", "queued_queries", "batches", "batched_structures",
                                          "staged_requests", "pageable_requests", "built_keys")] + [
        ("build_busy_ms", C.c_double), ("query_busy_ms", C.c_double), ("max_concurrent_batches", C.c_uint64)]


EXPORTED = ["burr_default_params", "burr_build", "burr_build_batch", "burr_query", "burr_size_bytes", "burr_export",
            "burr_stats", "burr_free", "burr_free_many", "burr_strerror", "burr_last_error", "burr_stage_hash",
            "burr_stage_sort", "burr_stage_sort_noalloc", "burr_server_create", "burr_server_submit_build",
            "burr_server_submit_query", "burr_server_wait", "burr_server_handle", "burr_server_release",
            "burr_server_stats", "burr_server_destroy", "burr_set_allocator", "burr_import",
            "burr_layer_geometry", "burr_shard_route", "burr_shard_build_layer", "burr_shard_build_base"]

_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)
_allocator_refs = []   # keeps the installed callbacks alive


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libburr.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or os.environ.get("BURR_LIB") or _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libburr.so not built ({path}); run __graft_entry__.build()")
        L = C.CDLL(path)
        p, u64, u32, i = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int
        L.burr_default_params.argtypes = [C.POINTER(Params)]
        L.burr_default_params.restype = i
        L.burr_build.argtypes = [p, p, u64, u32, C.POINTER(Params), p, C.POINTER(p)]
        L.burr_build.restype = i
        L.burr_build_batch.argtypes = [p, p, C.POINTER(u64), C.POINTER(u32), u32, C.POINTER(Params), p,
                                       C.POINTER(p)]
        L.burr_build_batch.restype = i
        L.burr_query.argtypes = [p, p, p, u64, p]
        L.burr_query.restype = i
        L.burr_size_bytes.argtypes = [p, C.POINTER(u64)]
        L.burr_size_bytes.restype = i
        L.burr_export.argtypes = [p, p, C.POINTER(u64)]
        L.burr_export.restype = i
        L.burr_stats.argtypes = [p, C.POINTER(Stats)]
        L.burr_stats.restype = i
        L.burr_free.argtypes = [p]
        L.burr_free.restype = None
        L.burr_free_many.argtypes = [p, u64]
        L.burr_free_many.restype = None
        L.burr_strerror.argtypes = [i]
        L.burr_strerror.restype = C.c_char_p
        L.burr_last_error.argtypes = []
        L.burr_last_error.restype = C.c_char_p
        L.burr_stage_hash.argtypes = [p, u64, u64, u32, u64, p, p, p]
        L.burr_stage_hash.restype = i
        L.burr_stage_sort.argtypes = [p, p, u64, u32, u64, u32, u64, p, p, p, p]
        L.burr_stage_sort.restype = i
        L.burr_stage_sort_noalloc.argtypes = [p, p, u64, u32, u64, u32, u64, p, p, p, p]
        L.burr_stage_sort_noalloc.restype = i
        L.burr_server_create.argtypes = [C.POINTER(ServerConfig), C.POINTER(Params), C.POINTER(p)]
        L.burr_server_create.restype = i
        L.burr_server_submit_build.argtypes = [p, p, p, u64, u32, C.POINTER(u64)]
        L.burr_server_submit_build.restype = i
        L.burr_server_submit_query.argtypes = [p, u64, p, u64, p, C.POINTER(u64)]
        L.burr_server_submit_query.restype = i
        L.burr_server_wait.argtypes = [p, u64, C.POINTER(C.c_double)]
        L.burr_server_wait.restype = i
        L.burr_server_handle.argtypes = [p, u64, C.POINTER(p)]
        L.burr_server_handle.restype = i
        L.burr_server_release.argtypes = [p, u64]
        L.burr_server_release.restype = i
        L.burr_server_stats.argtypes = [p, C.POINTER(ServerStats)]
        L.burr_server_stats.restype = i
        L.burr_server_destroy.argtypes = [p]
        L.burr_server_destroy.restype = None
        L.burr_set_allocator.argtypes = [_ALLOC_FN, _FREE_FN, p]
        L.burr_set_allocator.restype = i
        L.burr_import.argtypes = [p, u64, p, C.POINTER(p)]
        L.burr_import.restype = i
        L.burr_layer_geometry.argtypes = [u64, u32, C.POINTER(Params), C.POINTER(LayerGeometry)]
        L.burr_layer_geometry.restype = i
        L.burr_shard_route.argtypes = [p, p, u64, u32, C.POINTER(Params), u32, u64, u32, C.POINTER(u32), p, p,
                                       C.POINTER(u64), p]
        L.burr_shard_route.restype = i
        L.burr_shard_build_layer.argtypes = [p, p, u64, u32, C.POINTER(Params), u32, u64, u32, u32, p, p, p, p,
                                             C.POINTER(u64), p]
        L.burr_shard_build_layer.restype = i
        L.burr_shard_build_base.argtypes = [p, p, u64, u32, C.POINTER(Params), p, u64, C.POINTER(u64),
                                            C.POINTER(u64), C.POINTER(u32), p]
        L.burr_shard_build_base.restype = i
        _lib = L
        return L


def _check(rc):
    if rc != BURR_OK:
        L = load()
        raise BurrError(rc, f"{L.burr_strerror(rc).decode()}: {L.burr_last_error().decode()}")


def value_np_dtype(r: int):
    return np.uint8 if r <= 8 else (np.uint16 if r <= 16 else np.uint32)


def value_torch_dtype(r: int):
    import torch
    return torch.uint8 if r <= 8 else (torch.int16 if r <= 16 else torch.int32)


def default_params(**kw) -> Params:
    p = Params()
    _check(load().burr_default_params(C.byref(p)))
    for k, v in kw.items():
        if k == "levels":
            p.levels = (C.c_uint32 * 4)(*v)
        else:
            setattr(p, k, v)
    return p


def _ptr_and_stream(x, stream):
    """(pointer, stream handle, keepalive) for a torch tensor or numpy array."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if not x.is_contiguous():
                x = x.contiguous()
            if x.is_cuda:
                s = stream if stream is not None else torch.cuda.current_stream(x.device).cuda_stream
                return x.data_ptr(), s, x
            return x.data_ptr(), stream, x
    except ImportError:
        pass
    a = np.ascontiguousarray(x)
    return a.ctypes.data, stream, a


def _stream_value(s):
    if s is None:
        return None
    return getattr(s, "cuda_stream", s)


class Handle:
    """A built structure owned by the library (freed by .free() or GC).
    A borrowed handle (owned=False, e.g. a server's resident structure) is
    never freed from Python."""

    def __init__(self, ptr, r, owned=True):
        self._h = ptr or None   # the library's handle pointer (an int), None once freed
        self.r = r
        self.owned = owned
        self._batch = None      # the HandleBatch this handle belongs to (which then frees it)
        self._idx = 0

    def __del__(self):
        if getattr(self, "_batch", None) is None:
            self.free()

    def free(self):
        if not getattr(self, "owned", False):
            return
        if getattr(self, "_h", None):
            load().burr_free(self._h)
            self._h = None
            if self._batch is not None:
                self._batch._ptrs[self._idx] = 0

    def query(self, keys, out=None, stream=None):
        """Values of `keys` (torch CUDA/CPU tensor or numpy array), same kind back."""
        kp, st, keep = _ptr_and_stream(keys, _stream_value(stream))
        n = int(keep.numel() if hasattr(keep, "numel") else keep.size)
        if out is None:
            if hasattr(keep, "numel"):
                import torch
                out = torch.empty(n, dtype=value_torch_dtype(self.r), device=keep.device)
            else:
                out = np.empty(n, dtype=value_np_dtype(self.r))
        op, _, okeep = _ptr_and_stream(out, st)
        _check(load().burr_query(self._h, kp, op, n, st))
        return okeep

    def export_size(self) -> int:
        """Bytes burr_export writes for this structure."""
        need = C.c_uint64(0)
        load().burr_export(self._h, None, C.byref(need))
        return need.value

    def export(self, out=None):
        """burr_export.  Without `out`: the export as bytes.  With `out` (a host
        uint8 numpy array or CPU tensor, e.g. page-locked, of at least
        export_size() bytes): written there; returns the bytes written."""
        L = load()
        if out is not None:
            op, _, keep = _ptr_and_stream(out, None)
            ln = C.c_uint64(int(keep.numel() if hasattr(keep, "numel") else keep.nbytes))
            _check(L.burr_export(self._h, C.c_void_p(op), C.byref(ln)))
            return ln.value
        need = self.export_size()
        buf = (C.c_uint8 * need)()
        ln = C.c_uint64(need)
        _check(L.burr_export(self._h, buf, C.byref(ln)))
        return bytes(buf[:ln.value])

    def size_bytes(self) -> int:
        b = C.c_uint64(0)
        _check(load().burr_size_bytes(self._h, C.byref(b)))
        return b.value

    def stats(self) -> dict:
        s = Stats()
        _check(load().burr_stats(self._h, C.byref(s)))
        nl = s.layers + 1
        return dict(n=s.n, r=s.r, layers=s.layers, layer_n=list(s.layer_n[:nl]), layer_m=list(s.layer_m[:nl]),
                    layer_parts=list(s.layer_parts[:nl]), layer_bumped=list(s.layer_bumped[:nl]),
                    fallback_attempt=s.fallback_attempt,
                    stage_ms=[list(s.stage_ms[l]) for l in range(nl)], total_ms=s.total_ms,
                    table_bytes=s.table_bytes, kernel_launches=s.kernel_launches)


def build(keys, values, r: int, params: Params | None = None, stream=None, **kw) -> Handle:
    """burr_build: keys uint64 (int64 tensors hold the same bits), values of the r-bit type."""
    if params is None:
        params = default_params(**kw)
    kp, st, kk = _ptr_and_stream(keys, _stream_value(stream))
    vp, _, vk = _ptr_and_stream(values, st)
    n = int(kk.numel() if hasattr(kk, "numel") else kk.size)
    out = C.c_void_p()
    _check(load().burr_build(kp, vp, n, r, C.byref(params), st, C.byref(out)))
    return Handle(out.value, r)


def import_export(buf: bytes, stream=None) -> Handle:
    """burr_import: a device-resident structure from export bytes."""
    import struct
    raw = bytes(buf)
    out = C.c_void_p()
    b = (C.c_uint8 * len(raw)).from_buffer_copy(raw) if raw else (C.c_uint8 * 1)()
    _check(load().burr_import(b, len(raw), _stream_value(stream), C.byref(out)))
    r = struct.unpack_from("<I", raw, 8)[0]
    return Handle(out.value, r)


class HandleBatch(Sequence):
    """The structures of one batched build, in order.  Its handles are made on
    first access (a batch of 10,000 structures does not build 10,000 Python
    objects when only a few are used) and stay valid while they or the batch
    are referenced; free_all(batch) releases every structure not yet freed in
    one library call, and dropping the batch and its handles frees the rest."""

    def __init__(self, ptrs, rs):
        self._ptrs = ptrs                   # numpy uint64 handle pointers, 0 once freed
        self._rs = rs
        self._made = weakref.WeakValueDictionary()

    def __len__(self):
        return int(self._ptrs.size)

    def _one(self, i):
        h = self._made.get(i)
        if h is None:
            h = Handle(int(self._ptrs[i]), self._rs[i])
            h._batch, h._idx = self, i
            self._made[i] = h
        return h

    def __getitem__(self, i):
        if isinstance(i, slice):
            return [self._one(j) for j in range(*i.indices(len(self)))]
        n = len(self)
        i = operator.index(i)
        if i < 0:
            i += n
        if not 0 <= i < n:
            raise IndexError(i)
        return self._one(i)

    def __iter__(self):
        for i in range(len(self)):
            yield self._one(i)

    def free(self):
        live = np.ascontiguousarray(self._ptrs[self._ptrs != 0])
        if live.size:
            load().burr_free_many(live.ctypes.data, int(live.size))
        self._ptrs[:] = 0
        for h in list(self._made.values()):
            h._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:   # interpreter shutdown: the library may be gone
            pass


def free_all(handles) -> None:
    """burr_free_many: release many handles (e.g. a batched build's) in one call."""
    if isinstance(handles, HandleBatch):
        handles.free()
        return
    hs = [h for h in handles if getattr(h, "owned", False) and h._h]
    if hs:
        ptrs = [h._h for h in hs]
        load().burr_free_many((C.c_void_p * len(ptrs))(*ptrs), len(ptrs))
    for h in hs:
        h._h = None
        if h._batch is not None:
            h._batch._ptrs[h._idx] = 0


def build_batch(keys, values, offsets, rs, params: Params | None = None, stream=None, **kw) -> HandleBatch:
    """burr_build_batch: structure s owns keys[offsets[s]:offsets[s+1]] with r = rs[s].
    Returns the structures as a HandleBatch (a sequence of Handles, made on access)."""
    if params is None:
        params = default_params(**kw)
    offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64).astype(np.uint64))
    rs_np = np.ascontiguousarray(np.asarray(rs, dtype=np.int64).astype(np.uint32))
    S = int(rs_np.size)
    assert offsets.size == S + 1
    kp, st, _kk = _ptr_and_stream(keys, _stream_value(stream))
    vp, _, _vk = _ptr_and_stream(values, st)
    offs = (C.c_uint64 * (S + 1)).from_buffer_copy(offsets)
    rr = (C.c_uint32 * S).from_buffer_copy(rs_np)
    outs = (C.c_void_p * S)()
    _check(load().burr_build_batch(kp, vp, offs, rr, S, C.byref(params), st, outs))
    # the pointers in one conversion (element-wise reads of a ctypes array cost ~1 us each)
    return HandleBatch(np.frombuffer(outs, dtype=np.uint64).copy(), rs_np.tolist())


def stage_hash(keys, seed: int, layer_index: int, m: int, stream=None):
    """Stage entry point: (start uint32 as int32, coeff uint64 as int64) CUDA tensors."""
    import torch
    n = keys.numel()
    start = torch.empty(n, dtype=torch.int32, device=keys.device)
    coeff = torch.empty(n, dtype=torch.int64, device=keys.device)
    kp, st, _ = _ptr_and_stream(keys, _stream_value(stream))
    _check(load().burr_stage_hash(kp, n, seed, layer_index, m, start.data_ptr(), coeff.data_ptr(), st))
    return start, coeff


def stage_sort(keys, values, r: int, seed: int, layer_index: int, m: int, stream=None):
    """Stage entry point: keys/values grouped by bucket plus bucket offsets."""
    import torch
    n = keys.numel()
    nb = (m - 64 + 128) // 128
    sk = torch.empty_like(keys)
    sv = torch.empty_like(values)
    bs = torch.empty(nb + 1, dtype=torch.int32, device=keys.device)
    kp, st, _ = _ptr_and_stream(keys, _stream_value(stream))
    _check(load().burr_stage_sort(kp, values.data_ptr(), n, r, seed, layer_index, m, sk.data_ptr(),
                                  sv.data_ptr(), bs.data_ptr(), st))
    return sk, sv, bs


def _host_array(x, dtype):
    try:
        import torch
        if isinstance(x, torch.Tensor):
            x = x.cpu().numpy()
    except ImportError:
        pass
    return np.ascontiguousarray(x).view(dtype) if np.asarray(x).dtype.itemsize == np.dtype(dtype).itemsize \
        else np.ascontiguousarray(x, dtype=dtype)


class Server:
    """burr_server_*: continuous batching of builds with resident structures and
    overlapping queries on one device (host keys, values and outputs)."""

    def __init__(self, memory_budget: int, params: Params | None = None, max_batch_structures: int = 0,
                 host_staging_bytes: int = 1 << 30, build_workers: int = 0, **kw):
        if params is None:
            params = default_params(**kw)
        cfg = ServerConfig(memory_budget=int(memory_budget), host_staging_bytes=int(host_staging_bytes),
                           max_batch_structures=int(max_batch_structures), build_workers=int(build_workers))
        out = C.c_void_p()
        _check(load().burr_server_create(C.byref(cfg), C.byref(params), C.byref(out)))
        self._s = out
        self._r = {}      # build ticket -> r
        self._outs = {}   # query ticket -> output array (kept alive until waited)

    def submit_build(self, keys, values, r: int) -> int:
        k = _host_array(keys, np.uint64)
        v = _host_array(values, value_np_dtype(r))
        assert k.size == v.size
        t = C.c_uint64(0)
        _check(load().burr_server_submit_build(self._s, k.ctypes.data, v.ctypes.data, k.size, r, C.byref(t)))
        self._r[t.value] = r
        return t.value

    def submit_query(self, build_ticket: int, keys) -> int:
        k = _host_array(keys, np.uint64)
        out = np.empty(k.size, dtype=value_np_dtype(self._r[build_ticket]))
        t = C.c_uint64(0)
        _check(load().burr_server_submit_query(self._s, build_ticket, k.ctypes.data, k.size, out.ctypes.data,
                                               C.byref(t)))
        self._outs[t.value] = out
        return t.value

    def wait(self, ticket: int):
        """Block until the request is done: latency in ms for a build, (values,
        latency ms) for a query.  Raises BurrError if the request failed."""
        ms = C.c_double(0.0)
        rc = load().burr_server_wait(self._s, ticket, C.byref(ms))
        out = self._outs.pop(ticket, None)
        _check(rc)
        return ms.value if out is None else (out, ms.value)

    def handle(self, build_ticket: int) -> Handle:
        h = C.c_void_p()
        _check(load().burr_server_handle(self._s, build_ticket, C.byref(h)))
        return Handle(h.value, self._r[build_ticket], owned=False)

    def release(self, build_ticket: int):
        _check(load().burr_server_release(self._s, build_ticket))
        self._r.pop(build_ticket, None)

    def stats(self) -> dict:
        st = ServerStats()
        _check(load().burr_server_stats(self._s, C.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_s", None) is not None and self._s.value:
            load().burr_server_destroy(self._s)
            self._s = C.c_void_p(None)
            self._outs.clear()

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def set_allocator(alloc=None, free=None):
    """burr_set_allocator: route the library's device memory through
    alloc(bytes, stream) -> int pointer (0 on failure) and free(ptr, stream);
    both None restores the built-in pool.  Raises while blocks are held."""
    if (alloc is None) != (free is None):
        raise ValueError("alloc and free must both be given or both None")
    if alloc is None:
        _check(load().burr_set_allocator(_ALLOC_FN(), _FREE_FN(), None))
        _allocator_refs.clear()
        return

    def a(n, stream, ctx):
        try:
            return int(alloc(int(n), int(stream or 0))) or None
        except Exception:
            return None

    def f(ptr, stream, ctx):
        free(int(ptr), int(stream or 0))

    fa, ff = _ALLOC_FN(a), _FREE_FN(f)
    _check(load().burr_set_allocator(fa, ff, None))
    _allocator_refs[:] = [fa, ff]


def use_torch_allocator(device=None):
    """Back the library's device memory with PyTorch's caching allocator."""
    import torch
    dev = torch.cuda.current_device() if device is None else device
    set_allocator(lambda n, stream: torch.cuda.caching_allocator_alloc(n, dev, stream),
                  lambda ptr, stream: torch.cuda.caching_allocator_delete(ptr))


# --- sharded construction (burr_layer_geometry, burr_shard_*) ----------------

def layer_geometry(n_layer: int, layer: int, params: Params | None = None, **kw) -> dict:
    """burr_layer_geometry: slots, buckets and partitions of a bumping layer."""
    if params is None:
        params = default_params(**kw)
    g = LayerGeometry()
    _check(load().burr_layer_geometry(int(n_layer), int(layer), C.byref(params), C.byref(g)))
    return {f: getattr(g, f) for f, _ in LayerGeometry._fields_}


def shard_route(keys, values, r: int, layer: int, n_layer: int, part_first, params: Params, stream=None):
    """burr_shard_route: (keys, values) grouped by owner rank, and the count of
    each rank (CUDA tensors in, CUDA tensors and a list out)."""
    import torch
    ranks = len(part_first) - 1
    n = keys.numel()
    ko, vo = torch.empty_like(keys), torch.empty_like(values)
    pf = (C.c_uint32 * (ranks + 1))(*[int(x) for x in part_first])
    cnt = (C.c_uint64 * ranks)()
    kp, st, _ = _ptr_and_stream(keys, _stream_value(stream))
    _check(load().burr_shard_route(kp, values.data_ptr(), n, r, C.byref(params), layer, int(n_layer), ranks, pf,
                                   ko.data_ptr(), vo.data_ptr(), cnt, st))
    return ko, vo, [int(c) for c in cnt]


def shard_build_layer(keys, values, r: int, layer: int, n_layer: int, part_lo: int, part_hi: int, params: Params,
                      stream=None):
    """burr_shard_build_layer: (threshold words, table words, bumped keys,
    bumped values) of partitions [part_lo, part_hi), CUDA tensors."""
    import torch
    g = layer_geometry(n_layer, layer, params)
    dev = keys.device
    thresh = torch.empty(max((g["buckets"] + 31) // 32, 1), dtype=torch.int64, device=dev)
    z = torch.empty(max((g["m"] // 64) * r, 1), dtype=torch.int64, device=dev)
    n = keys.numel()
    bk, bv = torch.empty(max(n, 1), dtype=keys.dtype, device=dev), torch.empty(max(n, 1), dtype=values.dtype,
                                                                                 device=dev)
    nb = C.c_uint64(0)
    kp, st, _ = _ptr_and_stream(keys, _stream_value(stream))
    _check(load().burr_shard_build_layer(kp, values.data_ptr(), n, r, C.byref(params), layer, int(n_layer),
                                         int(part_lo), int(part_hi), thresh.data_ptr(), z.data_ptr(), bk.data_ptr(),
                                         bv.data_ptr(), C.byref(nb), st))
    k = nb.value
    return (thresh[:(g["buckets"] + 31) // 32], z[:(g["m"] // 64) * r], bk[:k], bv[:k])


def shard_build_base(keys, values, r: int, params: Params, stream=None):
    """burr_shard_build_base: (table words, slots, seed index, attempt)."""
    import torch
    L = load()
    n = keys.numel()
    mo, so, ao = C.c_uint64(0), C.c_uint64(0), C.c_uint32(0)
    kp, st, _ = _ptr_and_stream(keys, _stream_value(stream))
    cap = 0
    if n:   # ask for the largest table the retries may need
        L.burr_shard_build_base(kp, values.data_ptr(), n, r, C.byref(params), None, 0, C.byref(mo), C.byref(so),
                                C.byref(ao), st)
        cap = (mo.value // 64) * r
    z = torch.zeros(max(cap, 1), dtype=torch.int64, device=keys.device)
    _check(L.burr_shard_build_base(kp, values.data_ptr(), n, r, C.byref(params), z.data_ptr(), cap,
                                   C.byref(mo), C.byref(so), C.byref(ao), st))
    return z[:(mo.value // 64) * r], mo.value, so.value, ao.value
