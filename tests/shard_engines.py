"""A rank-local engine for the sharded build made of the oracle's steps (CPU,
test infrastructure): routing by the oracle's hash, each rank's partitions
built by the oracle's layer build with the layer's cut list, the base case by
its retries.  With it the sharded orchestration (routing, exchange,
ownership, export assembly) runs and is checked without a GPU."""
import types

import numpy as np

from oracle import oracle as O


def params(**kw):
    """The build parameters the orchestration reads, under the library's names."""
    p = dict(ribbon_width=64, bucket_slots=128, layers=4, levels=(0, 32, 64, 128), load_factor=1.015,
             partition_slots=65536, lower_partition_slots=4096, min_partition_slots=4096, seed=0x5EED5EED5EED5EED,
             fallback_slack=0.1, fallback_max_retries=16)
    p.update(kw)
    return types.SimpleNamespace(**p)


def oracle_kwargs(p):
    return dict(B=p.bucket_slots, levels=tuple(p.levels), alpha=p.load_factor, layers=p.layers,
                partition_slots=p.partition_slots, lower_partition_slots=p.lower_partition_slots,
                min_partition_slots=p.min_partition_slots, seed=p.seed)


def _np(x, dtype):
    import torch
    if isinstance(x, torch.Tensor):
        x = x.numpy()
    return np.ascontiguousarray(x).view(dtype) if np.asarray(x).dtype.itemsize == np.dtype(dtype).itemsize \
        else np.ascontiguousarray(x, dtype=dtype)


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a))


class OracleEngine:
    """Keys travel as int64 CPU tensors, values as int32 CPU tensors."""

    def __init__(self, p, threads=1):
        self.params = p
        self.threads = threads

    def geometry(self, n_layer, layer):
        p = self.params
        m = O.layer_slots(n_layer, p.load_factor)
        P = p.partition_slots if layer == 0 or not p.lower_partition_slots else p.lower_partition_slots
        return dict(n=n_layer, m=m, buckets=O.num_buckets(m, 64, p.bucket_slots),
                    partitions=O.num_partitions(m, P, p.min_partition_slots), partition_slots=P, seed_index=layer)

    def route(self, keys, vals, r, layer, n_layer, part_first):
        g = self.geometry(n_layer, layer)
        k = _np(keys, np.uint64)
        starts, _ = O.hash_many(k, O.layer_seed(self.params.seed, layer), g["m"])
        part = np.minimum(starts // np.uint64(g["partition_slots"]), np.uint64(g["partitions"] - 1)).astype(np.int64)
        owner = np.searchsorted(np.asarray(part_first, dtype=np.int64), part, side="right") - 1
        order = np.argsort(owner, kind="stable")
        counts = np.bincount(owner, minlength=len(part_first) - 1).tolist()
        return _t(k[order].view(np.int64)), _t(_np(vals, np.int32)[order]), counts

    def build_layer(self, keys, vals, r, layer, n_layer, part_lo, part_hi):
        p, g = self.params, self.geometry(n_layer, layer)
        P, K = g["partition_slots"], g["partitions"]
        res = O.build_layer(_np(keys, np.uint64), _np(vals, np.uint32), r, g["m"],
                            O.layer_seed(p.seed, layer), cuts=[j * P for j in range(1, K)],
                            levels=tuple(p.levels), B=p.bucket_slots, threads=self.threads)
        assert res.status == 0
        return res.thresh, res.z, _t(res.bumped_keys.view(np.int64)), _t(res.bumped_vals.view(np.int32))

    def build_base(self, keys, vals, r):
        p = self.params
        k, v = _np(keys, np.uint64), _np(vals, np.uint32)
        if len(k) == 0:
            return np.zeros(0, np.uint64), 0, p.layers, 0
        for a in range(p.fallback_max_retries + 1):
            m = O.fallback_slots(len(k), p.fallback_slack, 64, a)
            res = O.build_layer(k, v, r, m, O.layer_seed(p.seed, p.layers + a), fallback=True,
                                levels=tuple(p.levels), B=p.bucket_slots)
            if res.status == 0:
                return res.z, m, p.layers + a, a
        raise RuntimeError("base case unsolvable")
