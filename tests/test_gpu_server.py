"""Build/query server: continuous batching of independent builds with resident
structures and queries that overlap the builds.

Each structure the server builds, whatever else shared its batch, must be
bit-identical to the serial CPU oracle's structure for its keys with the
server's parameters (and so to a solo burr_build); queries return the stored
values, and for keys outside the set the oracle's values.
"""
import threading
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_12365_gb300 import inputs as I
from tests.export_format import describe_difference

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_12365_gb300 import burr  # noqa: E402

P = 4096
PARAMS = dict(partition_slots=P, min_partition_slots=P)


def _estimate(n, r, alpha=1.015):
    """The server's documented admission estimate of one build, in bytes."""
    vb = 1 if r <= 8 else (2 if r <= 16 else 4)
    m = 0 if n == 0 else ((-(-n * 1000 // int(alpha * 1000)) + 64 + 63) // 64) * 64
    return n * (8 + vb) * 4 + m * (8 + vb) * 2 + (m // 64) * r * 8 + (1 << 20)


def _request(i, n, r):
    keys = I.keys_np(n, seed=I.KEY_SEED + 1000 * i)
    return keys, I.values_np(keys, r)


def _oracle(keys, vals, r, **params):
    ref = O.build(keys, vals.astype(np.uint32), r=r, **{**PARAMS, **params})
    assert ref.ok
    return ref


@pytest.mark.parametrize("staging", [1 << 30, 600_000, 0])
def test_server_mix_equals_oracle_with_overlapping_queries(staging):
    rng = np.random.default_rng(11)
    sizes = [int(x) for x in np.exp(rng.uniform(np.log(50), np.log(60_000), size=48))]
    sizes[5], sizes[9] = 0, 1
    rs = [int(x) for x in rng.choice([1, 4, 8, 13, 16, 32], size=len(sizes))]
    reqs = [_request(i, n, r) for i, (n, r) in enumerate(zip(sizes, rs))]
    tickets = [None] * len(reqs)
    queries = {}
    with burr.Server(8 << 30, host_staging_bytes=staging, **PARAMS) as srv:
        def client(ids):
            for i in ids:
                k, v = reqs[i]
                tickets[i] = srv.submit_build(k, v, rs[i])
                # queued before the structure exists: runs once it is resident
                neg = I.keys_np(777, seed=I.KEY_SEED + 1000 * i, offset=1 << 40)
                queries[i] = (srv.submit_query(tickets[i], k), srv.submit_query(tickets[i], neg), neg)

        th = [threading.Thread(target=client, args=(list(range(c, len(reqs), 4)),)) for c in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for i, (k, v) in enumerate(reqs):
            srv.wait(tickets[i])
            got = srv.handle(tickets[i]).export()
            ref = _oracle(k, v, rs[i])
            want = ref.export()
            assert got == want, f"request {i} (n={sizes[i]}, r={rs[i]}): {describe_difference(got, want)}"
            qpos, qneg, neg = queries[i]
            out, ms = srv.wait(qpos)
            assert ms >= 0 and np.array_equal(out, v)
            out, _ = srv.wait(qneg)
            assert np.array_equal(out.astype(np.uint32), ref.query(neg))
        st = srv.stats()
        assert st["resident_structures"] == len(reqs) and st["batched_structures"] == len(reqs)
        total = st["staged_requests"] + st["pageable_requests"]
        assert total == 3 * len(reqs)
        if staging == 0:
            assert st["staged_requests"] == 0
        elif staging == 1 << 30:
            assert st["pageable_requests"] == 0
        else:
            assert st["staged_requests"] > 0 and st["pageable_requests"] > 0
        assert st["queued_builds"] == 0 and st["queued_queries"] == 0 and st["bytes_inflight"] == 0
        for t in tickets:
            srv.release(t)
        assert srv.stats()["bytes_resident"] == 0


def test_server_large_structure_takes_the_solo_path():
    # above the batched build's 64*1024 buckets per structure
    n, r = 9_000_000, 8
    keys, vals = _request(3, n, r)
    with burr.Server(8 << 30, **PARAMS) as srv:
        t_big = srv.submit_build(keys, vals, r)
        small = _request(4, 30_000, 8)
        t_small = srv.submit_build(*small, 8)
        srv.wait(t_big)
        srv.wait(t_small)
        got = srv.handle(t_big).export()
        want = _oracle(keys, vals, r).export()
        assert got == want, describe_difference(got, want)
        assert srv.handle(t_small).export() == _oracle(*small, 8).export()
        sel = np.random.default_rng(0).choice(n, 200_000, replace=False)
        out, _ = srv.wait(srv.submit_query(t_big, keys[sel]))
        assert np.array_equal(out, vals[sel])


def test_server_budget_admission_waits_for_release():
    n, r = 20_000, 8
    a, x = _request(20, n, r), _request(21, n, r)
    budget = _estimate(n, r) + 1000      # one build in flight; a resident one leaves no room
    with burr.Server(budget, **PARAMS) as srv:
        ta = srv.submit_build(*a, r)
        srv.wait(ta)
        resident = srv.stats()["bytes_resident"]
        assert resident > 1000
        tx = srv.submit_build(*x, r)
        tq = srv.submit_query(tx, x[0])
        time.sleep(0.3)
        st = srv.stats()
        assert st["queued_builds"] == 1 and st["bytes_inflight"] == 0 and st["queued_queries"] == 1
        with pytest.raises(burr.BurrError) as e:
            srv.release(tx)                   # still pending
        assert e.value.code == burr.ERR_INVALID
        srv.release(ta)                       # frees the room: x is admitted
        srv.wait(tx)
        out, _ = srv.wait(tq)
        assert np.array_equal(out, x[1])
        assert srv.handle(tx).export() == _oracle(*x, r).export()
        with pytest.raises(burr.BurrError) as e:
            srv.submit_build(*_request(22, 4 * n, r), r)   # larger than the whole budget
        assert e.value.code == burr.ERR_OOM


def test_server_failed_build_is_isolated():
    params = dict(PARAMS, fallback_max_retries=2)
    good1, good2 = _request(30, 40_000, 8), _request(31, 25_000, 8)
    dk, dv = _request(32, 10_000, 8)
    dk[5], dv[5] = dk[9], dv[9]               # a duplicate key: unsolvable
    with burr.Server(8 << 30, **params) as srv:
        t1 = srv.submit_build(*good1, 8)
        td = srv.submit_build(dk, dv, 8)
        t2 = srv.submit_build(*good2, 8)
        tq = srv.submit_query(td, dk[:10])
        with pytest.raises(burr.BurrError) as e:
            srv.wait(td)
        assert e.value.code == burr.ERR_UNSOLVABLE
        with pytest.raises(burr.BurrError) as e:
            srv.wait(tq)
        assert e.value.code == burr.ERR_INVALID
        for t, (k, v) in ((t1, good1), (t2, good2)):
            srv.wait(t)
            assert srv.handle(t).export() == _oracle(k, v, 8, fb_max_retries=2).export()
        srv.release(td)                       # a failed build's ticket is released like any other
        assert srv.stats()["resident_structures"] == 2


def test_server_destroy_with_pending_work():
    srv = burr.Server(8 << 30, **PARAMS)
    for i in range(16):
        t = srv.submit_build(*_request(40 + i, 50_000, 8), 8)
        srv.submit_query(t, I.keys_np(100))
    srv.close()                               # finishes the running batch, fails the queued ones
    with burr.Server(8 << 30, **PARAMS) as srv2:
        k, v = _request(60, 1000, 8)
        t = srv2.submit_build(k, v, 8)
        srv2.wait(t)
        out, _ = srv2.wait(srv2.submit_query(t, k))
        assert np.array_equal(out, v)


def test_server_1plus_thresholds():
    params = dict(PARAMS, threshold_mode=burr.THRESH_1PLUS)
    reqs = [_request(70 + i, n, 8) for i, n in enumerate((500, 20_000, 60_000, 3_000))]
    with burr.Server(8 << 30, **params) as srv:
        ts = [srv.submit_build(k, v, 8) for k, v in reqs]
        for t, (k, v) in zip(ts, reqs):
            srv.wait(t)
            assert srv.handle(t).export() == _oracle(k, v, 8, threshold_mode=O.THRESH_1PLUS).export()
            out, _ = srv.wait(srv.submit_query(t, k))
            assert np.array_equal(out, v)


@pytest.mark.parametrize("workers", [1, 3])
def test_batches_overlap_and_equal_the_oracle(workers):
    """Continuous batching: builds submitted while a batch is on the device are
    taken by an idle build worker at once (their own stream), so batches
    overlap; every structure still equals the oracle's for its keys."""
    big = _request(40, 3_000_000, 8)
    small = [_request(41 + i, int(n), 8) for i, n in enumerate([5000, 70_000, 1, 0, 20_000, 150_000])]
    with burr.Server(16 << 30, build_workers=workers, **PARAMS) as srv:
        tb = srv.submit_build(*big, 8)
        for _ in range(2000):                      # the big build is admitted and running
            st = srv.stats()
            if st["queued_builds"] == 0 and st["bytes_inflight"] > 0:
                break
            time.sleep(0.001)
        ts = [srv.submit_build(k, v, 8) for k, v in small]
        for t in [tb] + ts:
            srv.wait(t)
        st = srv.stats()
        if workers == 1:
            assert st["max_concurrent_batches"] == 1
        else:
            assert st["max_concurrent_batches"] >= 2
        for t, (k, v) in zip(ts, small):
            got, want = srv.handle(t).export(), _oracle(k, v, 8).export()
            assert got == want, describe_difference(got, want)
        sel = np.random.default_rng(1).choice(len(big[0]), 100_000, replace=False)
        out, _ = srv.wait(srv.submit_query(tb, big[0][sel]))
        assert np.array_equal(out, big[1][sel])
