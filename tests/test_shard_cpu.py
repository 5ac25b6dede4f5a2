"""Sharded construction (Sec. 3: partitions are independent once the cuts are
placed) on CPU: ranks own contiguous ranges of each layer's partitions, keys
are routed by start bucket and exchanged once per layer, every rank builds
its partitions alone, rank 0 builds the base case and writes the export.  The
export must equal the single-process oracle build of all keys, byte for
byte, for any number of ranks and any split of the keys.  The rank-local
steps are the oracle's (tests/shard_engines.py); the communicators are the
library's: threads of one process, and gloo processes (world size 2)."""
import os
import socket

import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_12365_gb300 import inputs as I
from paper_2411_12365_gb300 import shard
from tests import shard_engines as E

torch = pytest.importorskip("torch")


def _want(k, v, r, p):
    s = O.build(k, v.astype(np.uint32), r=r, **E.oracle_kwargs(p))
    assert s.ok
    return s.export()


def _split(k, v, ranks, how):
    if how == "strided":
        return [k[g::ranks] for g in range(ranks)], [v[g::ranks] for g in range(ranks)]
    cut = np.sort(np.random.default_rng(ranks).choice(len(k) + 1, ranks - 1))     # uneven, maybe empty
    idx = np.split(np.arange(len(k)), cut)
    return [k[i] for i in idx], [v[i] for i in idx]


CASES = [
    (200_000, 8, dict(partition_slots=4096), 2, "strided"),
    (200_000, 8, dict(partition_slots=4096), 3, "uneven"),
    (300_007, 16, dict(partition_slots=8192, lower_partition_slots=1024, min_partition_slots=1024), 5, "uneven"),
    (150_000, 1, dict(partition_slots=1024, min_partition_slots=0), 4, "strided"),
    (60_000, 8, dict(partition_slots=384, min_partition_slots=0, load_factor=1.6), 3, "strided"),  # heavy bumping
    (20_000, 8, {}, 4, "strided"),          # one partition per layer: three ranks own nothing
    (1, 8, {}, 2, "strided"),
    (0, 8, {}, 2, "strided"),
]


@pytest.mark.parametrize("n,r,pk,ranks,how", CASES)
def test_sharded_threads_equal_single_build(n, r, pk, ranks, how):
    p = E.params(**pk)
    k = I.keys_np(n, seed=n + 11)
    v = I.values_np(k, r).astype(np.uint32)
    ks, vs = _split(k, v, ranks, how)
    got = shard.build_sharded_virtual([torch.from_numpy(x.view(np.int64)) for x in ks],
                                      [torch.from_numpy(x.view(np.int32)) for x in vs], r,
                                      engine=E.OracleEngine(p))
    assert got == _want(k, v, r, p)


def test_owned_ranges_tile_the_layer():
    geo = dict(partitions=7, partition_slots=4096, m=30016, buckets=(30016 - 64 + 128) // 128)
    R = 3
    pf = [g * 7 // R for g in range(R + 1)]
    rs = [shard.owned_range(geo, 128, pf[g], pf[g + 1]) for g in range(R)]
    assert rs[0][0] == 0 and rs[0][2] == 0 and rs[-1][1] == geo["buckets"] and rs[-1][3] == geo["m"]
    for a, b in zip(rs, rs[1:]):
        assert a[1] == b[0] and a[3] == b[2]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _gloo_rank(rank, world, port, n, r, q):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from paper_2411_12365_gb300 import inputs as I
    from paper_2411_12365_gb300 import shard
    from tests import shard_engines as E
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = E.params(partition_slots=2048, lower_partition_slots=1024, min_partition_slots=1024)
    k = I.keys_np(n, seed=3)
    v = I.values_np(k, r).astype(np.uint32)
    mine = slice(rank * n // world, (rank + 1) * n // world)
    out = shard.build_sharded_rank(shard.TorchComm(), E.OracleEngine(p), torch.from_numpy(k[mine].view(np.int64)),
                                   torch.from_numpy(v[mine].view(np.int32)), r, p)
    if rank == 0:
        q.put(out == _want(k, v, r, p))
    dist.destroy_process_group()


def test_sharded_gloo_world2_equals_single_build():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_gloo_rank, args=(g, 2, port, 120_000, 8, q)) for g in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(300)
        assert p.exitcode == 0
    assert q.get(timeout=10) is True
