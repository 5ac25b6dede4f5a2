"""Sharded construction of one BuRR structure over several ranks.

Sec. 3 of the paper cuts every layer into partitions and makes the first
bucket after each cut bump at least w-1 slots, so that no kept equation
crosses a cut and the partitions are inserted and back-substituted
independently.  Here the ranks of a job own contiguous ranges of each layer's
partitions:

  1. the layer's size is the sum of the ranks' key counts (all-reduce);
  2. every rank groups its keys by the rank that owns their start bucket
     (``burr_shard_route``) and the groups are exchanged (all-to-all of
     (key, value) records, one per layer);
  3. every rank sorts, bands and back-substitutes its own partitions
     (``burr_shard_build_layer``); the keys it bumps are its input of the next
     layer;
  4. after the last bumping layer rank 0 gathers the remaining keys and builds
     the base case (``burr_shard_build_base``);
  5. rank 0 gathers the thresholds of the buckets and the table words of the
     slots each rank owns and writes the canonical export, which equals
     ``burr_build`` on the union of the keys byte for byte (``burr_import``
     loads it for queries).

The module is host orchestration only.  The method's steps run in the
engine's calls: ``GpuEngine`` calls the library's kernels; tests pass an
engine of their own.  The exchange goes through a communicator:
``ThreadComm`` runs several ranks as threads of one process (shards on one
GPU: the exchange is a device copy), ``TorchComm`` one rank per process with
``torch.distributed`` (NCCL between GPUs, gloo on CPUs).
"""
from __future__ import annotations

import pickle
import struct
import threading

import numpy as np

MAGIC = 0x52525542


# --- communicators ----------------------------------------------------------------

class ThreadComm:
    """`size` ranks as threads of one process.  Every rank thread calls the
    collectives in the same order; payloads are passed by reference."""

    def __init__(self, size: int):
        self.size = size
        self._bar = threading.Barrier(size)
        self._slots = [None] * size

    def rank_view(self, rank: int) -> "_ThreadRank":
        return _ThreadRank(self, rank)

    def run(self, fn, *per_rank_args):
        """fn(comm_view, *args_of_rank) on every rank; returns the results in rank order."""
        out, errs = [None] * self.size, []

        def body(g):
            try:
                out[g] = fn(self.rank_view(g), *[a[g] for a in per_rank_args])
            except BaseException as e:          # noqa: BLE001 -- reported below
                errs.append(e)
                self._bar.abort()

        ts = [threading.Thread(target=body, args=(g,)) for g in range(self.size)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        if errs:
            raise errs[0]
        return out


class _ThreadRank:
    def __init__(self, c: ThreadComm, rank: int):
        self.c, self.rank, self.size = c, rank, c.size

    def _exchange(self, payload):
        c = self.c
        c._bar.wait()
        c._slots[self.rank] = payload
        c._bar.wait()
        got = list(c._slots)
        c._bar.wait()
        return got

    def allreduce_sum(self, x: int) -> int:
        return int(sum(self._exchange(int(x))))

    def alltoallv(self, keys, vals, counts):
        """keys/vals grouped by destination with counts[d] entries for rank d;
        returns what every source sent here, concatenated in source order."""
        offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        mine = [(keys[offs[d]:offs[d + 1]], vals[offs[d]:offs[d + 1]]) for d in range(self.size)]
        allp = self._exchange(mine)
        ks = [allp[s][self.rank][0] for s in range(self.size)]
        vs = [allp[s][self.rank][1] for s in range(self.size)]
        return _cat(ks), _cat(vs)

    def gather(self, obj):
        got = self._exchange(obj)
        return got if self.rank == 0 else None


class TorchComm:
    """One rank per process through torch.distributed (an initialised default
    process group).  Tensors must live where the backend expects them (CUDA
    for NCCL, CPU for gloo)."""

    def __init__(self):
        import torch.distributed as dist
        self.d = dist
        self.rank, self.size = dist.get_rank(), dist.get_world_size()

    def _dev(self):
        import torch
        return torch.device("cuda", torch.cuda.current_device()) if self.d.get_backend() == "nccl" \
            else torch.device("cpu")

    def allreduce_sum(self, x: int) -> int:
        import torch
        t = torch.tensor([int(x)], dtype=torch.int64, device=self._dev())
        self.d.all_reduce(t)
        return int(t.item())

    def _a2a(self, x, send_counts, recv_counts):
        import torch
        out = torch.empty(int(sum(recv_counts)), dtype=x.dtype, device=x.device)
        self.d.all_to_all_single(out, x.contiguous(), [int(c) for c in recv_counts], [int(c) for c in send_counts])
        return out

    def alltoallv(self, keys, vals, counts):
        import torch
        sc = torch.tensor([int(c) for c in counts], dtype=torch.int64, device=self._dev())
        rc = torch.empty_like(sc)
        self.d.all_to_all_single(rc, sc)
        rcl = rc.tolist()
        rk = self._a2a(keys, counts, rcl)
        # values as bytes: NCCL has no 16-bit integer type
        isz = vals.element_size()
        rv = self._a2a(vals.view(torch.uint8), [c * isz for c in counts], [c * isz for c in rcl])
        return rk, rv.view(vals.dtype)

    def gather(self, obj):
        out = [None] * self.size if self.rank == 0 else None
        self.d.gather_object(obj, out, dst=0)
        return out


def _cat(xs):
    try:
        import torch
        if isinstance(xs[0], torch.Tensor):
            return torch.cat(xs)
    except ImportError:
        pass
    return np.concatenate(xs)


def _host(x) -> np.ndarray:
    try:
        import torch
        if isinstance(x, torch.Tensor):
            x = x.cpu().numpy()
    except ImportError:
        pass
    return np.asarray(x)


# --- the library as the engine ------------------------------------------------------

class GpuEngine:
    """Rank-local steps through libburr.so (CUDA tensors)."""

    def __init__(self, params=None, stream=None, **kw):
        from . import burr
        self.b = burr
        self.params = params if params is not None else burr.default_params(**kw)
        self.stream = stream

    def geometry(self, n_layer, layer):
        return self.b.layer_geometry(n_layer, layer, self.params)

    def route(self, keys, vals, r, layer, n_layer, part_first):
        return self.b.shard_route(keys, vals, r, layer, n_layer, part_first, self.params, self.stream)

    def build_layer(self, keys, vals, r, layer, n_layer, part_lo, part_hi):
        return self.b.shard_build_layer(keys, vals, r, layer, n_layer, part_lo, part_hi, self.params, self.stream)

    def build_base(self, keys, vals, r):
        return self.b.shard_build_base(keys, vals, r, self.params, self.stream)


# --- the sharded build ------------------------------------------------------------

def _codes_of(words: np.ndarray, b_lo: int, b_hi: int) -> np.ndarray:
    """2-bit codes of buckets [b_lo, b_hi) from packed threshold words."""
    b = np.arange(b_lo, b_hi, dtype=np.uint64)
    w = words.astype(np.uint64)[(b // np.uint64(32)).astype(np.int64)]
    return ((w >> (np.uint64(2) * (b % np.uint64(32)))) & np.uint64(3)).astype(np.uint8)


def _pack_codes(codes: np.ndarray) -> np.ndarray:
    nw = (len(codes) + 31) // 32
    c = np.zeros(nw * 32, dtype=np.uint64)
    c[:len(codes)] = codes
    return np.bitwise_or.reduce(c.reshape(nw, 32) << (np.uint64(2) * np.arange(32, dtype=np.uint64)), axis=1) \
        if nw else np.zeros(0, np.uint64)


def owned_range(geo: dict, B: int, lo: int, hi: int):
    """Buckets and slots that partitions [lo, hi) of a layer own: buckets from
    partition lo's first bucket to partition hi's; slots from c_lo + 64 (0 for
    partition 0) to c_hi + 64 (m after the last partition), c_j = j*P."""
    K, P, m, nb = geo["partitions"], geo["partition_slots"], geo["m"], geo["buckets"]
    if lo >= hi:
        return 0, 0, 0, 0
    b_lo, b_hi = lo * P // B, (nb if hi == K else hi * P // B)
    s_lo, s_hi = (0 if lo == 0 else lo * P + 64), (m if hi == K else hi * P + 64)
    return b_lo, b_hi, s_lo, s_hi


def build_sharded_rank(comm, engine, keys, vals, r: int, params):
    """One rank's part of the sharded build (SPMD: every rank calls it with its
    own keys).  Returns the export bytes on rank 0, None elsewhere."""
    R, rank = comm.size, comm.rank
    B = int(params.bucket_slots)
    n_total = comm.allreduce_sum(len(keys))
    cur_k, cur_v = keys, vals
    meta, owned = [], []
    for l in range(int(params.layers)):
        n_l = comm.allreduce_sum(len(cur_k))
        if n_l == 0:
            meta.append((0, 0, 0, 0, 0))
            owned.append(None)
            continue
        geo = engine.geometry(n_l, l)
        K = geo["partitions"]
        part_first = [g * K // R for g in range(R + 1)]
        ks, vs, counts = engine.route(cur_k, cur_v, r, l, n_l, part_first)
        rk, rv = comm.alltoallv(ks, vs, counts)
        lo, hi = part_first[rank], part_first[rank + 1]
        thr, z, bk, bv = engine.build_layer(rk, rv, r, l, n_l, lo, hi)
        b_lo, b_hi, s_lo, s_hi = owned_range(geo, B, lo, hi)
        owned.append((_codes_of(_host(thr).view(np.uint64), b_lo, b_hi),
                      _host(z).view(np.uint64)[(s_lo // 64) * r:(s_hi // 64) * r].copy()))
        meta.append((n_l, geo["m"], K, geo["buckets"], comm.allreduce_sum(len(bk))))
        cur_k, cur_v = bk, bv
    rest = comm.gather((cur_k, cur_v))
    parts = comm.gather(pickle.dumps(owned))
    if rank != 0:
        return None
    base_k = _cat([x[0] for x in rest])
    base_v = _cat([x[1] for x in rest])
    fz, fm, fseed, fatt = engine.build_base(base_k, base_v, r)
    owned_all = [pickle.loads(p) for p in parts]
    return _export_bytes(params, r, n_total, meta, owned_all, len(base_k), fm, fseed, fatt, _host(fz).view(np.uint64))


def _export_bytes(params, r, n, meta, owned_all, fn, fm, fseed, fatt, fz) -> bytes:
    """The canonical export (include/burr.h, version 1: 2-bit thresholds)."""
    out = [struct.pack("<10I", MAGIC, 1, r, int(params.ribbon_width), int(params.bucket_slots), int(params.layers),
                       *[int(x) for x in params.levels]),
           struct.pack("<Q", int(params.seed)), struct.pack("<d", float(params.load_factor)),
           struct.pack("<QQ", n, int(params.partition_slots))]
    for mt in meta:
        out.append(struct.pack("<5Q", *mt))
    out.append(struct.pack("<4Q", fn, fm, fseed, fatt))
    for l, mt in enumerate(meta):
        if mt[0] == 0:
            continue
        codes = np.concatenate([o[l][0] for o in owned_all if o[l] is not None])
        z = np.concatenate([o[l][1] for o in owned_all if o[l] is not None])
        assert len(codes) == mt[3] and len(z) == (mt[1] // 64) * r
        out.append(_pack_codes(codes).astype("<u8").tobytes())
        out.append(z.astype("<u8").tobytes())
    out.append(np.asarray(fz, dtype="<u8").tobytes())
    return b"".join(out)


def build_sharded_virtual(keys_per_rank, vals_per_rank, r: int, engine=None, params=None, **kw) -> bytes:
    """The sharded build with len(keys_per_rank) ranks as threads of this
    process (e.g. shards of one GPU); returns the export."""
    if engine is None:
        engine = GpuEngine(params, **kw)
    params = engine.params
    comm = ThreadComm(len(keys_per_rank))
    out = comm.run(lambda c, k, v: build_sharded_rank(c, engine, k, v, r, params), keys_per_rank, vals_per_rank)
    return out[0]
