#!/usr/bin/env python3
"""Benchmark of the GB300 BuRR hot path: one step = construction of a BuRR
structure of n keys (hash, sort by bucket, band + bump with partition cuts,
back-substitution, recursion into the next layers and the base case) through
the C ABI of libburr.so.

Default workload: 10^9 uniform-random 64-bit keys, r = 8 (8-bit filter
values), w = 64, 2-bit thresholds, partitions of 2^16 slots in layer 0 and
4096 in deeper layers.  Queries (n keys, half members) are timed apart, and
the same construction at r = 1 and r = 16 gives the per-stage split.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl burr|reference]

Prints one JSON line (rank 0).  `value` is constructed keys per second with
device-resident inputs; `e2e` is the construction from page-locked host keys
and values with the structure read back to the host, copies inside the timed
region; `roofline` is the dominant kernel (layer-0 band + bump) against the
measured HBM bandwidth; `cpu_baseline` is the CPU oracle on a bounded sample,
serial and with its partitions spread over the host's cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BuRR construction Mkeys/s and % HBM roofline at 1 GB300 (plain vs batched/served)"
UNIT = "Mkeys/s"
FALLBACK_HBM_GBS = 6800.0


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="burr", choices=["burr", "reference"])
    ap.add_argument("--keys", type=int, default=1_000_000_000, help="keys per structure")
    ap.add_argument("--r", type=int, default=8)
    ap.add_argument("--partition-slots", type=int, default=65536)
    ap.add_argument("--lower-partition-slots", type=int, default=4096)
    ap.add_argument("--cut-search", default="none", choices=["none", "minbump", "maxprev", "diff"],
                    help="cut-point search (Sec. 3) over --cut-search-range buckets from each nominal cut")
    ap.add_argument("--cut-search-range", type=int, default=50)
    ap.add_argument("--thresholds", default="2bit", choices=["2bit", "1plus"],
                    help="threshold storage: 2-bit levels or 1+-bit (bit per bucket + exact thresholds)")
    ap.add_argument("--min-partition-slots", type=int, default=4096)
    ap.add_argument("--cpu-sample", type=int, default=1 << 24,
                    help="keys of the serial oracle sample (about 10 s of CPU work)")
    ap.add_argument("--cpu-sample-mt", type=int, default=1 << 26,
                    help="keys of the threaded oracle sample (all host cores)")
    ap.add_argument("--ref-sample", type=int, default=1 << 24, help="keys per reference-arm step")
    ap.add_argument("--ref-threads", type=int, default=0,
                    help="host threads of the reference arm's oracle (0 = all cores)")
    ap.add_argument("--split-r", default="1,16",
                    help="value widths whose construction split (sort/band/back-substitution) is also reported")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile-steps", action="store_true",
                    help="only run warmup+steps (for ncu launch lists), skip extras")
    ap.add_argument("--workload", default="plain", choices=["plain", "batched", "serve"],
                    help="plain: one structure of --keys keys; batched: many independent structures")
    ap.add_argument("--structures", type=int, default=10_000, help="batched: number of structures")
    ap.add_argument("--plain-sample", type=int, default=300,
                    help="batched: structures also built one call each, for the comparison")
    ap.add_argument("--serve-builds", type=int, default=600, help="serve: build requests per load point")
    ap.add_argument("--serve-loads", default="0.5,0.75,0.9",
                    help="serve: offered load points as fractions of the measured saturated capacity")
    ap.add_argument("--serve-budget-gb", type=float, default=40.0, help="serve: admission budget")
    ap.add_argument("--serve-staging-gb", type=float, default=4.0, help="serve: page-locked payload region")
    ap.add_argument("--serve-workers", type=int, default=1,
                    help="serve: build workers (batches that overlap on the device); the other of 1 and 2 is also "
                         "measured at 0.75 load")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def ncu_band_summary(kernel_src: str, path: str | None = None):
    """DRAM bytes and warp instructions of the captured layer-0 band launches
    (2-bit thresholds, 1-byte values) and their layer-0 key count, from the
    committed ncu summary, if it was taken on the current kernel source; else
    None.  Both grow in proportion to the keys of the launch."""
    path = path or os.path.join(ROOT, "profiles", "k_band_1e9_r8_traffic.txt")
    try:
        kv = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        src_hash = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
        if kv.get("kernel_source_sha256_16") != src_hash:
            return None
        inst = kv.get("warp_instructions_captured")
        return {"dram_bytes": float(kv["dram_bytes_per_launch_captured"]),
                "warp_instructions": float(inst) if inst else None,
                "keys": float(kv["n_keys_captured"])}
    except Exception:
        return None


def issue_roofline(warp_instructions, band_ms, sms, sm_max_mhz):
    """Warp instructions per second of the band launch against the issue peak:
    four schedulers per SM, one warp instruction each per cycle, at the SM clock."""
    peak = sms * 4 * sm_max_mhz * 1e6
    achieved = warp_instructions / (band_ms / 1e3)
    return {"warp_instructions": warp_instructions, "achieved": achieved, "peak": peak,
            "unit": "warp instructions/s", "frac": achieved / peak,
            "peak_derivation": f"{sms} SMs x 4 schedulers x 1 warp instruction/cycle x {sm_max_mhz:.0f} MHz"}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.p is None:
            return
        time.sleep(0.25)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return ws, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x: float) -> float:
    if pg is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def oracle_sample(n_s: int, r: int, P: int, minP: int = 4096, lowP: int = 4096, mode: int = 0, cut: int = 0,
                  cut_range: int = 50, threads: int = 1):
    """CPU oracle: construction of n_s keys of the workload (serial, or with each
    layer's partitions over `threads` host threads); returns seconds."""
    import numpy as np

    from oracle import oracle as O
    from paper_2411_12365_gb300 import inputs as I
    k = I.keys_np(n_s)
    v = I.values_np(k, r).astype(np.uint32)
    t0 = time.perf_counter()
    s = O.build(k, v, r=r, partition_slots=P, min_partition_slots=minP, lower_partition_slots=lowP,
                threshold_mode=mode, cut_search=cut, cut_search_range=cut_range, threads=threads)
    dt = time.perf_counter() - t0
    sel = np.arange(0, n_s, max(1, n_s // 4096))
    assert s.ok and np.array_equal(s.query(k[sel]), v[sel])
    oracle_sample.xor_steps_per_row = s.stats.xor_steps / max(s.stats.inserted, 1)
    return dt


def run_reference(a, ws, rank, pg):
    if rank != 0:
        return
    from oracle import oracle as O
    O.build_lib()
    n_s = a.ref_sample
    cores, model = cpu_info()
    threads = a.ref_threads or cores
    dt = 0.0
    for i in range(a.warmup + a.steps):
        t = oracle_sample(n_s, a.r, a.partition_slots, a.min_partition_slots, a.lower_partition_slots, tmode(a),
                          cmode(a), a.cut_search_range, threads=threads)
        if i >= a.warmup:
            dt += t
    dt /= max(a.steps, 1)
    value = n_s / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": workload_config(a),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"C oracle with each layer's partitions spread over {threads} host threads: "
                                   f"construction of {n_s} keys per step (of the {a.keys}-key workload)",
                         "nproc": cores, "cpu_model": model},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def tmode(a) -> int:
    return 1 if a.thresholds == "1plus" else 0


def cmode(a) -> int:
    return ["none", "minbump", "maxprev", "diff"].index(a.cut_search)


def workload_config(a):
    tdesc = "1+-bit thresholds" if a.thresholds == "1plus" else "2-bit thresholds"
    if a.cut_search != "none":
        tdesc += f", {a.cut_search} cut search over {a.cut_search_range} buckets"
    return {"workload": f"construction of one structure of {a.keys} uniform-random 64-bit keys, r={a.r}, w=64, "
                        f"{tdesc}, partition size {a.partition_slots} slots in layer 0 and "
                        f"{a.lower_partition_slots} in deeper layers, 4 layers + base case, plain build",
            "n_keys": a.keys, "r": a.r, "ribbon_width": 64, "bucket_slots": 128,
            "partition_slots": a.partition_slots, "lower_partition_slots": a.lower_partition_slots,
            "min_partition_slots": a.min_partition_slots, "load_factor": 1.015, "layers": 4,
            "thresholds": a.thresholds, "cut_search": a.cut_search, "cut_search_range": a.cut_search_range,
            "l2_flush": "inputs larger than L2 (keys 8n bytes)", "parallelism": "one independent structure per GPU"}


def batched_sizes(count: int, seed: int = 2024):
    """Structure sizes log-uniform in [100, 10^6] keys and value widths uniform
    in {1, 2, 3, 4, 8} (the many-small-structures workload)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(100), np.log(1_000_000), size=count)).astype(np.int64)
    rs = rng.choice([1, 2, 3, 4, 8], size=count)
    return sizes, rs


def run_batched(a, ws, rank, local, pg):
    import numpy as np
    import torch

    from paper_2411_12365_gb300 import burr
    from paper_2411_12365_gb300 import inputs as I

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sizes, rs = batched_sizes(a.structures, seed=2024 + rank)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    N = int(offs[-1])
    keys = I.keys_torch(N, dev, seed=I.KEY_SEED + rank * 0x100000000)
    vals = I.values_torch(keys, 8)
    params = burr.default_params(partition_slots=0, flags=burr.FLAG_TIMING)
    chosen = [None]

    def step():
        hs = burr.build_batch(keys, vals, offs, rs, params=params)
        chosen[0] = hs[0].export()[64:72]
        burr.free_all(hs)

    for _ in range(a.warmup):
        step()
    # correctness of the timed configuration: a few structures answer their values
    hs = burr.build_batch(keys, vals, offs, rs, params=params)
    for s in (0, len(hs) // 2, len(hs) - 1):
        k = keys[offs[s]:offs[s + 1]]
        got = hs[s].query(k).to(torch.int64) & ((1 << int(rs[s])) - 1)
        want = vals[offs[s]:offs[s + 1]].to(torch.int64) & ((1 << int(rs[s])) - 1)
        assert torch.equal(got, want)
    P = int(np.frombuffer(hs[0].export()[64:72], dtype=np.uint64)[0])
    del hs
    torch.cuda.synchronize()
    barrier(pg)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record()
        for _ in range(a.steps):
            step()
        ev1.record()
        torch.cuda.synchronize()
    ms = max_over_ranks(pg, ev0.elapsed_time(ev1) / a.steps)
    value = ws * N / (ms / 1e3) / 1e6
    # equal output, one call per structure: a sample built both ways
    q = min(a.plain_sample, a.structures)
    sample = np.random.default_rng(7).choice(a.structures, size=q, replace=False)
    sub_sizes, sub_rs = sizes[sample], rs[sample]
    sub_offs = np.concatenate([[0], np.cumsum(sub_sizes)]).astype(np.int64)
    sub_keys = torch.cat([keys[offs[s]:offs[s + 1]] for s in sample])
    sub_vals = torch.cat([vals[offs[s]:offs[s + 1]] for s in sample])
    pp = burr.default_params(partition_slots=P, min_partition_slots=P)
    t0 = time.perf_counter()
    hs = burr.build_batch(sub_keys, sub_vals, sub_offs, sub_rs, params=pp)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    ex_batch = [h.export() for h in hs]
    del hs
    t0 = time.perf_counter()
    solo = []
    for i in range(q):
        k = sub_keys[sub_offs[i]:sub_offs[i + 1]]
        v = sub_vals[sub_offs[i]:sub_offs[i + 1]]
        solo.append(burr.build(k, v, int(sub_rs[i]), params=pp))
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    equal = all(solo[i].export() == ex_batch[i] for i in range(q))
    n_sub = int(sub_offs[-1])
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": f"batched build of {a.structures} independent structures, sizes log-uniform "
                                   f"in [100, 10^6] keys, r uniform in {{1,2,3,4,8}}, one launch per stage "
                                   f"and layer, partition size autotuned",
                       "structures": a.structures, "total_keys": N, "partition_slots_autotuned": P,
                       "l2_flush": "inputs larger than L2", "parallelism": "independent structures"},
            "breakdown": {"sample_structures": q, "sample_keys": n_sub,
                          "batched_sample_mkeys_s": n_sub / t_batch / 1e6,
                          "plain_one_call_per_structure_sample_mkeys_s": n_sub / t_plain / 1e6,
                          "sample_exports_equal": equal},
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)


def serve_requests(count: int, pool: int, seed: int):
    """Seeded request stream: builds with sizes log-uniform in [10^3, 10^7] keys
    (r = 8), each a slice of a key pool, and as many query batches with sizes
    log-uniform in [10^4, 10^6] keys on one of the 16 most recent builds.
    Returns ([(kind, n, pool offset, build index)], mean build size)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    b_sizes = np.exp(rng.uniform(np.log(1e3), np.log(1e7), size=count)).astype(np.int64)
    b_offs = rng.integers(0, pool - b_sizes + 1)
    events = []
    for i in range(count):
        events.append(("build", int(b_sizes[i]), int(b_offs[i]), i))
        t = int(rng.integers(max(0, i - 15), i + 1))
        q = int(min(np.exp(rng.uniform(np.log(1e4), np.log(1e6))), b_sizes[t]))
        events.append(("query", q, int(b_offs[t] + rng.integers(0, b_sizes[t] - q + 1)), t))
    return events, float(b_sizes.mean())


def serve_run(srv, events, keys, vals, rate_builds_s, seed):
    """Open loop: builds arrive as a Poisson process of the given rate (queries
    right behind the build they follow); a collector waits for every request
    in arrival order, checks query results and releases structures that fall
    out of the 64 most recent.  rate None = everything at once (saturation).
    Every structure is released at the end."""
    import queue
    import threading
    import numpy as np
    rng = np.random.default_rng(seed)
    fifo = queue.Queue()
    res = {"build_ms": [], "query_ms": [], "bad": 0, "keys": 0, "errors": []}
    st0 = srv.stats()
    tickets = {}
    resident = []
    batch_dev = {}

    def collector():
        while True:
            item = fifo.get()
            if item is None:
                return
            kind, t, info = item
            try:
                if kind == "build":
                    res["build_ms"].append(srv.wait(t))
                    hs = srv.handle(t).stats()
                    # structures of one batch share its device time and stage times
                    batch_dev[round(hs["total_ms"], 5)] = hs["stage_ms"]
                    resident.append(t)
                    if len(resident) > 64:
                        srv.release(resident.pop(0))
                else:
                    out, ms = srv.wait(t)
                    res["query_ms"].append(ms)
                    off, q = info
                    res["bad"] += int(np.count_nonzero(out != vals[off:off + q]))
            except Exception as e:                      # recorded, reported in the line
                res["errors"].append(str(e))

    th = threading.Thread(target=collector)
    th.start()
    t0 = time.perf_counter()
    t_next = t0
    for kind, n, off, idx in events:
        if kind == "build":
            if rate_builds_s:
                t_next += rng.exponential(1.0 / rate_builds_s)
                d = t_next - time.perf_counter()
                if d > 0:
                    time.sleep(d)
            tickets[idx] = srv.submit_build(keys[off:off + n], vals[off:off + n], 8)
            res["keys"] += n
            fifo.put(("build", tickets[idx], None))
        else:
            fifo.put(("query", srv.submit_query(tickets[idx], keys[off:off + n]), (off, n)))
    t_submitted = time.perf_counter()
    fifo.put(None)
    th.join()
    t_end = time.perf_counter()
    st = {k: v - st0[k] for k, v in srv.stats().items()}
    for t in resident:
        srv.release(t)
    pct = lambda xs, p: float(np.percentile(xs, p)) if xs else None  # noqa: E731
    return {"offered_builds_per_s": rate_builds_s, "submit_s": t_submitted - t0, "makespan_s": t_end - t0,
            "served_mkeys_s": res["keys"] / (t_end - t0) / 1e6,
            "build_p50_ms": pct(res["build_ms"], 50), "build_p99_ms": pct(res["build_ms"], 99),
            "query_p50_ms": pct(res["query_ms"], 50), "query_p99_ms": pct(res["query_ms"], 99),
            "batches": st["batches"], "batched_structures": st["batched_structures"],
            "staged_requests": st["staged_requests"], "pageable_requests": st["pageable_requests"],
            "build_worker_busy_ms": st["build_busy_ms"], "query_worker_busy_ms": st["query_busy_ms"],
            "build_device_ms": sum(batch_dev), "builds_device_ms_by_stage": [
                round(sum(sm[l][k] for sm in batch_dev.values()), 2) for l in range(5) for k in range(3)],
            "query_value_mismatches": res["bad"], "errors": res["errors"][:3]}


def run_served(a, ws, rank, local, pg):
    import numpy as np
    import torch

    from paper_2411_12365_gb300 import burr
    from paper_2411_12365_gb300 import inputs as I

    torch.cuda.set_device(local)
    pool = 1 << 26
    kd = I.keys_torch(pool, torch.device("cuda", local), seed=I.KEY_SEED + rank * 0x100000000)
    vals = I.values_torch(kd, 8).cpu().numpy()
    keys = kd.cpu().numpy().view(np.uint64)
    del kd
    torch.cuda.empty_cache()
    budget = int(a.serve_budget_gb * (1 << 30))
    def server(workers):
        return burr.Server(budget, host_staging_bytes=int(a.serve_staging_gb * (1 << 30)), build_workers=workers,
                           partition_slots=a.partition_slots, min_partition_slots=a.min_partition_slots,
                           lower_partition_slots=a.lower_partition_slots, flags=burr.FLAG_TIMING)

    srv = server(a.serve_workers)
    # warm-up (library load, pools, first launches), then saturated capacity
    ev, _ = serve_requests(max(8, a.serve_builds // 20), pool, seed=99)
    serve_run(srv, ev, keys, vals, None, 0)
    events, mean_n = serve_requests(a.serve_builds, pool, seed=2025 + rank)
    with ClockSampler(local) as clk:
        sat = serve_run(srv, events, keys, vals, None, 1)
        cap_builds_s = sat["served_mkeys_s"] * 1e6 / mean_n
        points = []
        for i, f in enumerate(float(x) for x in a.serve_loads.split(",")):
            r = serve_run(srv, events, keys, vals, f * cap_builds_s, 10 + i)
            r["load"] = f
            points.append(r)
    # equal output: a sample of the stream's builds, served and built one call each
    pp = burr.default_params(partition_slots=a.partition_slots, min_partition_slots=a.min_partition_slots,
                             lower_partition_slots=a.lower_partition_slots)
    sample = [e for e in events if e[0] == "build"][:12]
    st = [srv.submit_build(keys[off:off + n], vals[off:off + n], 8) for _, n, off, _ in sample]
    equal = True
    for t, (_, n, off, _) in zip(st, sample):
        srv.wait(t)
        h = burr.build(keys[off:off + n], vals[off:off + n], 8, params=pp)
        equal = equal and srv.handle(t).export() == h.export()
        h.free()
        srv.release(t)
    srv.close()
    # the same build requests, one burr_build call each (host keys and values, as the server gets them)
    builds = [e for e in events if e[0] == "build"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _, n, off, _ in builds:
        h = burr.build(keys[off:off + n], vals[off:off + n], 8, params=pp)
        h.free()
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    plain = {"builds": len(builds), "keys": int(sum(e[1] for e in builds)), "seconds": plain_s,
             "mkeys_s": sum(e[1] for e in builds) / plain_s / 1e6,
             "note": "the stream's build requests back to back, one burr_build call each, from host memory"}
    # the other worker count (one: batches never overlap; two: a new batch starts while one runs)
    # at the 0.75 load point, for the latency comparison
    other_w = 2 if a.serve_workers == 1 else 1
    s1 = server(other_w)
    serve_run(s1, ev, keys, vals, None, 0)
    other = serve_run(s1, events, keys, vals, 0.75 * cap_builds_s, 11)
    other["load"] = 0.75
    other["build_workers"] = other_w
    s1.close()
    head = min(points, key=lambda r: abs(r["load"] - 0.75))
    value = max_over_ranks(pg, -head["served_mkeys_s"]) * -1 * ws if ws > 1 else head["served_mkeys_s"]
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": len(points), "warmup": 1,
            "ms_per_step": head["makespan_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"served builds and queries: {a.serve_builds} builds per load point, Poisson "
                                   f"arrivals, sizes log-uniform in [10^3, 10^7] keys (r=8), one query batch "
                                   f"of 10^4..10^6 keys per build on one of the 16 latest builds, admission "
                                   f"budget {a.serve_budget_gb:g} GB, page-locked staging "
                                   f"{a.serve_staging_gb:g} GB, 64 most recent structures resident; "
                                   f"value = served throughput at the load point nearest 0.75 of capacity",
                       "partition_slots": a.partition_slots, "mean_build_keys": mean_n,
                       "l2_flush": "inputs larger than L2", "parallelism": "independent structures"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                    "note": "every request is host to device: this line is end to end"},
            "serving": {"build_workers": a.serve_workers, "saturated": sat, "points": points,
                        "other_build_workers_at_0.75": other,
                        "plain_one_call_per_build": plain,
                        "served_saturated_over_plain": sat["served_mkeys_s"] / plain["mkeys_s"],
                        "sample_exports_equal_served_vs_plain": equal},
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)


def cpu_info():
    """Host cores and CPU model (for the CPU-baseline record)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if not model.isdigit():
                    break
    except Exception:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return os.cpu_count() or 1, model


def stage_split(stats_list, layers):
    """Mean device ms per layer and stage (sort, band + bump, back-substitution)
    over several builds, and the layer-0 stages."""
    avg = lambda f: statistics.mean(f(s) for s in stats_list)  # noqa: E731
    per_layer = [[round(avg(lambda s, l=l, k=k: s["stage_ms"][l][k]), 4) for k in range(3)]
                 for l in range(layers + 1)]
    return {"build_ms": avg(lambda s: s["total_ms"]),
            "layer0_ms": {"sort": per_layer[0][0], "band_bump": per_layer[0][1], "backsub": per_layer[0][2]},
            "stage_ms_per_layer [sort, band+bump, backsub]": per_layer}


def compulsory_build_bytes(st, r):
    """Compulsory bytes of a build (the model of the roofline): per layer-l key
    read (key, value) and one partition-order round trip, bumped keys written
    into the next layer, the table written once."""
    vb = 1 if r <= 8 else (2 if r <= 16 else 4)
    layers = st["layers"]
    ln, lm = st["layer_n"], st["layer_m"]
    return (sum(ln[:layers + 1]) * 3 * (8 + vb) + sum(ln[1:layers + 1]) * (8 + vb)
            + sum(lm[:layers + 1]) * r // 8)


def run_plain(a, ws, rank, local, pg):
    import numpy as np
    import torch

    from paper_2411_12365_gb300 import burr
    from paper_2411_12365_gb300 import inputs as I

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, r, P = a.keys, a.r, a.partition_slots
    vb = 1 if r <= 8 else (2 if r <= 16 else 4)
    seed = I.KEY_SEED + rank * 0x100000000        # independent structure per rank
    keys = I.keys_torch(n, dev, seed=seed)
    vals = I.values_torch(keys, r)

    def params_for(flags=burr.FLAG_TIMING):
        return burr.default_params(partition_slots=P, min_partition_slots=a.min_partition_slots,
                                   lower_partition_slots=a.lower_partition_slots, threshold_mode=tmode(a),
                                   cut_search=cmode(a), cut_search_range=a.cut_search_range, flags=flags)

    params = params_for()
    torch.cuda.synchronize()
    stats_acc = []
    launches = [0]

    def step():
        # one construction: hash, sort, band + bump, back-substitution of every
        # layer and the base case; the handle is released right after
        h = burr.build(keys, vals, r, params=params)
        st = h.stats()
        stats_acc.append(st)
        launches[0] += st["kernel_launches"]
        h.free()

    for _ in range(a.warmup):
        step()
    # correctness of the timed configuration: query(x) = f(x) for every key
    h = burr.build(keys, vals, r, params=params)
    assert torch.equal(h.query(keys), vals), "query(x) != f(x)"
    h.free()
    stats_acc.clear()
    launches[0] = 0
    torch.cuda.synchronize()
    barrier(pg)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        w0 = time.perf_counter()
        ev0.record()
        for _ in range(a.steps):
            step()
        ev1.record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
    barrier(pg)
    ms = max_over_ranks(pg, ev0.elapsed_time(ev1) / a.steps)
    value = ws * n / (ms / 1e3) / 1e6
    if a.profile_steps:
        if rank == 0:
            print(json.dumps({"ms_per_step": ms, "value": value}))
        return

    # end to end through the C ABI (measured first, on a quiet pool): keys and values in page-locked host memory,
    # the structure read back into page-locked host memory, copies inside the timed region
    e2e_line = None
    if not a.no_e2e:
        hk = keys.cpu().pin_memory()
        hv = vals.cpu().pin_memory()
        hk_np, hv_np = hk.numpy().view(np.uint64), hv.numpy()
        p2 = params_for(0)
        h = burr.build(hk_np, hv_np, r, params=p2)
        ex_len = h.export_size()
        h.free()
        hx = torch.empty(ex_len, dtype=torch.uint8).pin_memory()
        out_len = [0]

        def e2e_step():
            h = burr.build(hk_np, hv_np, r, params=p2)
            out_len[0] = h.export(out=hx)
            h.free()

        for _ in range(max(1, min(a.warmup, 3))):
            e2e_step()
        torch.cuda.synchronize()
        barrier(pg)
        t0 = time.perf_counter()
        marks = []
        for _ in range(a.steps):
            e2e_step()
            marks.append(time.perf_counter())
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(pg, (time.perf_counter() - t0) / a.steps)
        per = [1e3 * (b - a_) for a_, b in zip([t0] + marks[:-1], marks)]
        e2e_line = {"value": ws * n / e2e_s / 1e6, "unit": UNIT, "ms_per_step": e2e_s * 1e3,
                    "step_ms_min_median_max": [min(per), statistics.median(per), max(per)],
                    "h2d_bytes_per_step": n * 8 + n * vb, "d2h_bytes_per_step": out_len[0],
                    "step": "burr_build from page-locked host keys and values, burr_export of the "
                            "structure into page-locked host memory, burr_free"}
        del hk, hv, hx

    st0 = stats_acc[-1]
    layers = st0["layers"]
    split = stage_split(stats_acc, layers)
    band0 = split["layer0_ms"]["band_bump"]
    build_ms = split["build_ms"]
    n0, m0 = st0["layer_n"][0], st0["layer_m"][0]
    nb0 = (m0 - 64 + 128) // 128
    bump0 = st0["layer_bumped"][0]
    # algorithmic bytes of the layer-0 band launch: read the bucket-sorted
    # (key, value) records, write the bumped ones, write the thresholds
    band_bytes = n0 * (8 + vb) + bump0 * (8 + vb) + ((nb0 + 31) // 32) * 8
    peak, peak_kind = measured_peaks()
    achieved = band_bytes / (band0 / 1e3) / 1e9
    # the ncu figures belong to the captured instantiation: 2-bit thresholds, 1-byte values
    summ = (ncu_band_summary(os.path.join(ROOT, "paper_2411_12365_gb300", "csrc", "burr_band.cu"))
            if tmode(a) == 0 and vb == 1 else None)
    scale = n0 / summ["keys"] if summ else None
    traffic = summ["dram_bytes"] * scale if summ else None
    overhead = (st0["table_bytes"] - 64) * 8 / (r * n) - 1
    build_bytes = compulsory_build_bytes(st0, r)

    # queries, timed apart from construction: n keys, half members
    half = n // 2
    qkeys = torch.cat([keys[:half], I.keys_torch(n - half, dev, seed=seed, offset=n)])
    qout = torch.empty(n, dtype=burr.value_torch_dtype(r), device=dev)
    h = burr.build(keys, vals, r, params=params)
    qsteps = max(3, min(a.steps, 10))
    for _ in range(2):
        h.query(qkeys, out=qout)
    torch.cuda.synchronize()
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q0.record()
    for _ in range(qsteps):
        h.query(qkeys, out=qout)
    q1.record()
    torch.cuda.synchronize()
    query_ms = q0.elapsed_time(q1) / qsteps
    assert torch.equal(qout[:half], vals[:half]), "query(x) != f(x)"
    visits = sum(st0["layer_n"][:layers + 1]) / max(n0, 1)
    query_bytes = n * (8 + vb) + n * visits * (32 + -(-2 * r * 8 // 32) * 32)
    h.free()
    del qkeys, qout
    torch.cuda.empty_cache()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": workload_config(a), "wall_s_timed": wall,
        "breakdown": {
            "step": "one burr_build of n device-resident keys (all layers and the base case), then burr_free",
            "build_ms_device": build_ms, "build_mkeys_s": n / build_ms / 1e3,
            **split,
            "layer_n": st0["layer_n"], "layer_m": st0["layer_m"], "layer_parts": st0["layer_parts"],
            "space_overhead": overhead,
            "query": {"keys": n, "members": half, "ms": query_ms, "mkeys_s": n / query_ms / 1e3,
                      "compulsory_bytes": query_bytes, "frac": query_bytes / (query_ms / 1e3) / 1e9 / peak,
                      "note": "timed apart from construction; 32-byte sectors counted as if from DRAM"},
            "roofline_by_stage": {
                "peak_gbs": peak, "peak_kind": peak_kind,
                "build": {"compulsory_bytes": build_bytes,
                          "achieved_gbs": build_bytes / (ms / 1e3) / 1e9,
                          "frac": build_bytes / (ms / 1e3) / 1e9 / peak,
                          "model": "per layer-l key 3(8+v) bytes, bumped keys (8+v) into the next layer, "
                                   "the table once; over the timed step"}},
            "paper_cpu_context": "67.8 Mkeys/s construction, 1e8 keys, 64 threads on EPYC 7551P (Fig. 7)",
        },
        "roofline": {"bound": "hbm", "kernel": "k_band (layer 0)", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "algorithmic_bytes": band_bytes,
                     "algorithmic_model": "read n0 sorted (key, value) records, write the bumped ones, "
                                          "write the 2-bit thresholds",
                     "note": "band+bump is latency-bound (dependent GF(2) elimination chains); see issue"},
        "gpu_launches": launches[0],
    }
    line["clocks"] = clk.summary()
    if e2e_line:
        line["e2e"] = e2e_line
    if summ and summ["warp_instructions"]:
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = line["clocks"].get("sm_max_mhz") or 2070.0
        line["roofline"]["issue"] = issue_roofline(summ["warp_instructions"] * scale, band0, sms, mhz)

    # the sort/band/back-substitution split at other value widths (r = 1, 16)
    if a.split_r and rank == 0:
        other = {}
        for rr in (int(x) for x in a.split_r.split(",") if x):
            v2 = I.values_torch(keys, rr)
            acc = []
            for i in range(3 + 5):
                h = burr.build(keys, v2, rr, params=params)
                if i >= 3:
                    acc.append(h.stats())
                h.free()
            sp = stage_split(acc, acc[-1]["layers"])
            sp["build_mkeys_s"] = n / sp["build_ms"] * 1e-3
            sp["space_overhead"] = (acc[-1]["table_bytes"] - 64) * 8 / (rr * n) - 1
            other[f"r{rr}"] = sp
            del v2
        line["breakdown"]["split_by_r"] = other
        torch.cuda.empty_cache()

    if not a.no_cpu and rank == 0:
        cores, model = cpu_info()
        dt = oracle_sample(a.cpu_sample, r, P, a.min_partition_slots, a.lower_partition_slots, tmode(a),
                           cmode(a), a.cut_search_range)
        xor_steps = oracle_sample.xor_steps_per_row
        dtm = oracle_sample(a.cpu_sample_mt, r, P, a.min_partition_slots, a.lower_partition_slots, tmode(a),
                            cmode(a), a.cut_search_range, threads=cores)
        line["cpu_baseline"] = {
            "value": a.cpu_sample / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"serial C oracle: construction of {a.cpu_sample} keys of the same workload "
                      f"(same r, P, load; {dt:.1f} s)",
            "threaded": {"value": a.cpu_sample_mt / dtm / 1e6, "unit": UNIT, "cores": cores,
                         "sample": f"the same oracle with each layer's partitions spread over {cores} host "
                                   f"threads: construction of {a.cpu_sample_mt} keys ({dtm:.1f} s)"},
            "nproc": cores, "cpu_model": model}
        # the dependent chain behind the band kernel's latency bound: row XORs
        # per insertion attempt of the serial elimination
        line["breakdown"]["oracle_xor_steps_per_row"] = xor_steps
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    a = args_()
    ws, rank, local, pg = dist_setup()
    if a.impl == "reference":
        run_reference(a, ws, rank, pg)
        return
    if a.workload == "batched":
        run_batched(a, ws, rank, local, pg)
        return
    if a.workload == "serve":
        run_served(a, ws, rank, local, pg)
        return
    run_plain(a, ws, rank, local, pg)


if __name__ == "__main__":
    main()
