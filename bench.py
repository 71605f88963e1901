#!/usr/bin/env python3
"""Benchmark: exact short-pattern search throughput on GB300.

Workload (default ``sweep``, the pattern-length sweep): three synthetic texts of
n = 256 MiB each — sigma=4 uniform DNA-like, sigma=20 uniform protein-like,
sigma=64 natural-language-like (Zipf s=1.1 with a 15% space symbol) — and for
each text 100 patterns per m in {2, 4, 8, 16, 32}, half copied from random text
offsets and half drawn i.i.d. from the text's symbol distribution.  One step
searches every (text, pattern) pair: 1500 searches, 402.7 GB of text.  Each
search produces its count and all sorted uint64 start positions.

Metric: text GB/s (bytes of text scanned / second), device-timed with the
texts resident in HBM.  ``e2e`` is the same metric through the public C entry
point that takes HOST buffers (epsm_search_host), with the texts' host->device
copies and the positions' device->host copies inside the timed region.

``--impl reference`` times the CPU oracle (brute-force scan) on the host cores
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

GiB = 1 << 30
MiB = 1 << 20
METRIC = "text GB/s (pattern-length sweep, m=2..32)"
UNIT = "GB/s"
KINDS = ("dna", "protein", "nl64")
MS = (2, 4, 8, 16, 32)
PATS_PER_M = 100
TEXT_N = 256 * MiB
L2_BYTES = 129 * 10**6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="epsm", choices=["epsm", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--patterns", type=int, default=PATS_PER_M,
                    help="patterns per (text, m); the workload uses 100")
    ap.add_argument("--case", default=None,
                    help="KIND:M[:VARIANT[:N[:count]]] — time one search of an N-byte text "
                         "(default 256 MiB; 'count': count only) and exit (the small case "
                         "used for ncu captures)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--sample", action="store_true",
                    help="one search per (text, m) of the sweep (15 launches) and exit; the "
                         "launches an ncu traffic capture measures")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-pairs", type=int, default=8192)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-rates", default="2000,5000,10000,20000,50000",
                    help="Poisson arrival rates (queries/s) of the served workload")
    ap.add_argument("--serve-secs", type=float, default=1.0,
                    help="arrival window per rate for the serving engine")
    ap.add_argument("--serve-pq-secs", type=float, default=0.25,
                    help="arrival window per rate for the per-query path (it saturates early)")
    return ap.parse_args()


def run_case(args):
    """One search configuration, timed with CUDA events (for profiling)."""
    import torch
    import gen
    import paper_1209_6449_gb300 as epsm
    parts = args.case.split(":")
    kind, m = parts[0], int(parts[1])
    variant = int(parts[2]) if len(parts) > 2 else 0
    n = int(parts[3]) if len(parts) > 3 else TEXT_N
    count_only = len(parts) > 4 and parts[4] == "count"
    ctx = epsm.Context(0)
    t = torch.empty(n, dtype=torch.uint8, device="cuda")
    gen.TextSpec(kind, 0).device(n, t.data_ptr(), torch.cuda.current_stream().cuda_stream)
    pat = gen.planted_patterns(gen.TextSpec(kind, 0), n, m, 1)[0]
    cap = 0 if count_only else n // 3
    out = torch.empty(max(cap, 1), dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    times = []
    for _ in range(args.reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.search_async(t, pat, out, cap, cnt, variant=variant)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    st = ctx.sync()
    print(json.dumps({"case": args.case, "n": n, "count": int(cnt.item()), "status": st,
                      "ms": [round(x, 4) for x in times],
                      "gbs_best": round(n / min(times) / 1e6, 1)}), flush=True)
    ctx.close()
    return 0 if st == 0 else 1


def workload_patterns(npat):
    import gen
    out = []
    for kind in KINDS:
        spec = gen.TextSpec(kind, 0)
        for m in MS:
            for p in gen.mixed_patterns(spec, TEXT_N, m, npat):
                out.append((kind, m, p))
    return out


def config(npat, ngpus):
    return {"workload": "pattern-length sweep: 3 texts x 256 MiB (sigma 4 DNA-like, sigma 20 "
                        "protein-like, sigma 64 Zipf natural-language-like), m in {2,4,8,16,32}, "
                        f"{npat} patterns per (text, m), half planted half i.i.d.",
            "text_bytes": TEXT_N, "texts": list(KINDS), "m": list(MS),
            "patterns_per_text_and_m": npat, "searches_per_step": len(KINDS) * len(MS) * npat,
            "l2": "inputs larger than L2 (256 MiB text vs 129 MB L2); no flush",
            "parallelism": f"replicas x{ngpus}" if ngpus > 1 else "single GPU"}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [l for (t, l) in self.lines if t0 - 0.15 <= t <= t1 + 0.15] or [l for _, l in self.lines]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [x.strip() for x in r.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for name, val in zip(names, f[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# reference arm / CPU baseline: the oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_sample(budget_s, texts_host):
    """Time the oracle on a bounded sample: the first 8 MiB of each text, two
    patterns per (text, m), repeated until about budget_s seconds."""
    import gen
    import oracle
    cores = os.cpu_count() or 1
    sample_n = 8 * MiB
    jobs = []
    for kind in KINDS:
        spec = gen.TextSpec(kind, 0)
        t = texts_host[kind][:sample_n] if texts_host else spec.host(sample_n)
        for m in MS:
            for p in gen.mixed_patterns(spec, TEXT_N, m, 2):
                jobs.append((t, p))
    scanned, t0 = 0, time.perf_counter()
    rounds = 0
    while True:
        for t, p in jobs:
            oracle.count(t, p, threads=cores)
            scanned += t.size
        rounds += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": round(scanned / dt / 1e9, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{rounds} round(s) of {len(jobs)} searches (3 texts x 5 m x 2 patterns) "
                      f"over the first 8 MiB of each text, brute-force C oracle on {cores} threads"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import gen
    import oracle
    cores = os.cpu_count() or 1
    sample_n = 4 * MiB
    jobs = []
    for kind in KINDS:
        spec = gen.TextSpec(kind, 0)
        t = spec.host(sample_n)
        for m in MS:
            p = gen.mixed_patterns(spec, TEXT_N, m, 2)[0]
            jobs.append((t, p))

    def step():
        tot = 0
        for t, p in jobs:
            oracle.count(t, p, threads=cores)
            tot += t.size
        return tot

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    tot = 0
    for _ in range(args.steps):
        tot += step()
    dt = time.perf_counter() - t0
    v = tot / dt / 1e9
    sample = (f"each step: 15 searches (3 texts x 5 m x 1 pattern) over the first 4 MiB of each "
              f"text, brute-force C oracle on {cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": config(args.patterns, args.gpus),
            "cpu_baseline": {"value": round(v, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# roofline inputs
# ---------------------------------------------------------------------------

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1209_6449_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    return d


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_sample(args):
    """One search per (text, m) of the sweep, with the first (planted) pattern:
    the launches the committed DRAM-traffic capture covers."""
    import torch
    import gen
    import paper_1209_6449_gb300 as epsm
    ctx = epsm.Context(0)
    stream = torch.cuda.current_stream()
    cap = TEXT_N // 8
    out = torch.empty(cap, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    rows = []
    for kind in KINDS:
        t = torch.empty(TEXT_N, dtype=torch.uint8, device="cuda")
        gen.TextSpec(kind, 0).device(TEXT_N, t.data_ptr(), stream.cuda_stream)
        for m in MS:
            p = gen.mixed_patterns(gen.TextSpec(kind, 0), TEXT_N, m, args.patterns)[0]
            ctx.search_async(t, p, out, cap, cnt, stream=stream)
            torch.cuda.synchronize()
            c = int(cnt.item())
            rows.append({"text": kind, "m": m, "count": c, "alg_bytes": TEXT_N + 8 * c + 8})
        del t
    st = ctx.sync()
    print(json.dumps({"sample": rows, "mean_alg_bytes": sum(r["alg_bytes"] for r in rows) / len(rows),
                      "status": st}), flush=True)
    ctx.close()
    return 0 if st == 0 else 1


def run_batched(ctx, torch, npairs):
    """The batched-uneven workload: npairs (text, pattern) pairs, text lengths
    log-uniform in 1 KiB..32 MiB over sigma in {4, 20, 64}, m uniform in 1..32,
    half planted; one batched launch per step against one launch per pair."""
    import gen
    from paper_1209_6449_gb300 import epsm_search_async
    pairs = gen.batch_pairs(npairs, seed=0)
    tot = sum(p.n for p in pairs)
    buf = torch.empty(tot + 16 * npairs, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    texts, off = [], 0
    for p in pairs:
        p.spec.device(p.n, buf.data_ptr() + off, s)
        texts.append((buf.data_ptr() + off, p.n))
        off += (p.n + 15) // 16 * 16
    pats = [p.pattern for p in pairs]
    cap = 1 << 28
    times = []
    offs = None
    for rep in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        offs, out = ctx.search_batch(texts, pats, cap)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        del out
    batched = min(times[1:])
    cnts = torch.zeros(npairs, dtype=torch.int64, device="cuda")
    out2 = torch.empty(cap, dtype=torch.int64, device="cuda")
    ptimes = []
    for rep in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i, (ptr, n) in enumerate(texts):
            epsm_search_async(ctx.handle, ptr, n, pats[i], len(pats[i]), out2.data_ptr(), cap,
                              cnts.data_ptr() + 8 * i, s)
        torch.cuda.synchronize()
        ptimes.append(time.perf_counter() - t0)
    per_pair = min(ptimes)
    agree = bool((np.diff(offs.astype(np.int64)) == cnts.cpu().numpy()).all())
    del buf, out2
    torch.cuda.empty_cache()
    return {"workload": f"{npairs} pairs, n log-uniform 1 KiB..32 MiB ({tot / 2**30:.2f} GiB), "
                        "sigma in {4,20,64}, m uniform 1..32, half planted",
            "queries_per_s": round(npairs / batched, 1), "text_gbs": round(tot / batched / 1e9, 1),
            "ms": round(batched * 1e3, 3), "per_pair_queries_per_s": round(npairs / per_pair, 1),
            "per_pair_ms": round(per_pair * 1e3, 3), "speedup_vs_per_pair": round(per_pair / batched, 2),
            "graph_replay": ctx.batch_uses_graph, "counts_agree_with_per_pair": agree,
            "timing": "wall clock around the synchronous batched call (upload, launch, offsets "
                      "download) vs one asynchronous launch per pair and a final synchronize"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.case:
        return run_case(args)
    if args.sample:
        return run_sample(args)

    import torch
    import gen
    import paper_1209_6449_gb300 as epsm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    else:
        torch.cuda.set_device(0)
    dev = torch.device(f"cuda:{local if world > 1 else 0}")
    ctx = epsm.Context(dev.index)
    stream = torch.cuda.current_stream()

    # texts resident in HBM, generated on the device
    texts = {}
    for kind in KINDS:
        t = torch.empty(TEXT_N, dtype=torch.uint8, device=dev)
        gen.TextSpec(kind, 0).device(TEXT_N, t.data_ptr(), stream.cuda_stream)
        texts[kind] = t
    pats = workload_patterns(args.patterns)
    nsearch = len(pats)
    cap = TEXT_N // 8
    out = torch.empty(cap, dtype=torch.int64, device=dev)
    counts = torch.zeros(nsearch, dtype=torch.int64, device=dev)
    torch.cuda.synchronize()

    def step():
        for i, (kind, m, p) in enumerate(pats):
            ctx.search_async(texts[kind], p, out, cap, counts[i:i + 1], stream=stream)

    launches0 = ctx.launch_count
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = ctx.sync()
    if st != 0:
        raise SystemExit(f"device status {st} after warm-up")
    occ = counts.cpu().numpy()
    assert int(occ.max()) <= cap, "output capacity exceeded"

    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches_before = ctx.launch_count
    t_wall0 = time.time()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    if dist:
        dist.barrier()
    launches = ctx.launch_count - launches_before
    elapsed_ms = e0.elapsed_time(e1)
    clocks.stop()
    st = ctx.sync()
    if st != 0:
        raise SystemExit(f"device status {st} after timed region")
    if dist:
        tt = torch.tensor([elapsed_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed_ms = float(tt.item())

    bytes_per_step = nsearch * TEXT_N
    value = world * bytes_per_step * args.steps / (elapsed_ms / 1e3) / 1e9
    occ_total = int(occ.sum())
    # roofline of one search (the filter kernel and its emission kernel):
    # algorithmic bytes = text read + 8 B per written position + 8 B count;
    # duration = timed region / searches
    alg_bytes_per_launch = (bytes_per_step + 8 * occ_total + 8 * nsearch) / nsearch
    per_launch_s = elapsed_ms / 1e3 / max(args.steps * nsearch, 1)
    achieved = alg_bytes_per_launch / per_launch_s / 1e9
    peak, peak_kind = measured_peaks()
    traffic = profiled_traffic()

    e2e = None
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = oracle_sample(12.0, None)
    if not args.no_e2e:
        e2e = run_e2e(ctx, pats, args, torch, dev, dist)
    batched = None
    if not args.no_batch:
        del texts, out
        torch.cuda.empty_cache()
        batched = run_batched(ctx, torch, args.batch_pairs)
    served = None
    if not args.no_serve and world == 1:
        torch.cuda.empty_cache()
        served = run_served(torch, args)

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(elapsed_ms / args.steps, 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
                "config": config(args.patterns, world),
                "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                             "unit": "GB/s", "frac": round(achieved / peak, 4),
                             "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                             "kernel": "stream_kernel + stream_emit_kernel, per search (all variants; "
                                       "algorithmic bytes = n + 8*occ + 8 per search)",
                             "traffic": traffic.get("bytes_per_launch") if traffic else None,
                             "traffic_note": (traffic.get("note") if traffic else
                                              "null: no ncu capture of the current kernel sources")},
                "cpu_baseline": cpu,
                "e2e": e2e,
                "batched": batched,
                "served": served,
                "gpu_launches": launches,
                "clocks": clocks.summary(t_wall0, t_wall1),
                "occurrences_per_step": occ_total}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    ctx.close()
    return 0


def run_served(torch, args):
    """The served workload: 4 corpora of 1 GiB resident in HBM (sigma 4, 20,
    64 Zipf, 96-symbol order-2 Markov), a Poisson stream of queries (corpus
    uniform, pattern from a pool of 1024 per corpus with m uniform in 2..32,
    half copied from the corpus, half i.i.d.), 1% of requests uploading a new
    16..256 MiB text (admitted against a 16 GiB upload budget, least recently
    used uploads evicted).  Each rate is replayed through the serving engine
    (continuous batching, two launches in flight) and through the per-query
    path (one single-search launch per query); latency = result published -
    scheduled arrival."""
    import gen
    import paper_1209_6449_gb300 as epsm
    n = 1 << 30
    kinds = ("dna", "protein", "nl64", "markov96")
    stream = torch.cuda.current_stream().cuda_stream
    bufs, specs = [], []
    for i, k in enumerate(kinds):
        b = torch.empty(n + 16, dtype=torch.uint8, device="cuda")
        sp = gen.TextSpec(k, 900 + i)
        sp.device(n, b.data_ptr(), stream)
        bufs.append(b)
        specs.append(sp)
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    pool = []
    for c, sp in enumerate(specs):
        for k in range(1024):
            m = int(rng.integers(2, 33))
            p = (gen.planted_patterns(sp, n, m, 1, stream_seed=k)[0] if k % 2
                 else gen.random_patterns(sp, m, 1, stream_seed=k)[0])
            pool.append((c, p))
    uploads = [gen.TextSpec("protein", 77).host(u) for u in (16 << 20, 64 << 20, 128 << 20, 256 << 20)]

    def stream_for(rate, secs, seed):
        r = np.random.default_rng(seed)
        cnt = int(rate * secs)
        at = np.cumsum(r.exponential(1e9 / rate, size=cnt)).astype(np.int64)
        kind = (r.random(cnt) < 0.01).astype(np.uint32)
        idx = r.integers(0, len(pool), size=cnt)
        corp = np.array([pool[i][0] for i in idx], dtype=np.uint32)
        pay = [uploads[int(r.integers(0, 4))] if kind[j] else pool[idx[j]][1] for j in range(cnt)]
        return at, kind, corp, pay

    def replay(per_query, rate, secs):
        srv = epsm.Server(0, max_batch=1024, inflight=2, per_query=per_query,
                          upload_budget=16 << 30, out_capacity=1 << 29)
        for b in bufs:
            srv.add_corpus((b.data_ptr(), n))
        at, kind, corp, pay = stream_for(rate, args.serve_secs, 11)
        cnt = int(rate * secs)
        res = srv.replay(at[:cnt], kind[:cnt], corp[:cnt], pay[:cnt])
        stats = srv.stats()
        srv.close()
        q = kind[:cnt] == 0
        lat = res["latency_ns"][q] / 1e6
        return ({"offered_qps": rate, "queries": int(q.sum()), "uploads": int((~q).sum()),
                 "qps": round(float(q.sum()) / res["elapsed_s"], 1),
                 "p50_ms": round(float(np.percentile(lat, 50)), 3),
                 "p99_ms": round(float(np.percentile(lat, 99)), 3),
                 "all_ok": bool((res["status"] == 0).all()),
                 "batches": stats["batches"], "evictions": stats["evictions"]},
                res["counts"])

    out = []
    for rate in [int(x) for x in args.serve_rates.split(",")]:
        srv, c1 = replay(False, rate, args.serve_secs)
        pq, c2 = replay(True, rate, min(args.serve_secs, args.serve_pq_secs))
        out.append({"served": srv, "per_query": pq,
                    "same_counts": bool((c1[:len(c2)] == c2).all()),
                    "qps_ratio": round(srv["qps"] / pq["qps"], 2)})
    del bufs
    torch.cuda.empty_cache()
    return {"workload": "4 resident 1 GiB corpora (sigma 4, 20, 64 Zipf, 96 order-2 Markov); Poisson "
                        "queries, m uniform 2..32 from a 1024-pattern pool per corpus (half planted); "
                        "1% uploads of 16..256 MiB texts under a 16 GiB budget",
            "engine": "epsm_server (continuous batching, 2 launches in flight, up to 1024 queries "
                      "per batch) vs per-query (one single-search launch per query)",
            "latency": "result published - scheduled arrival",
            "rates": out}


def run_e2e(ctx, pats, args, torch, dev, dist):
    """Same workload through epsm_search_host: host texts in, host positions out."""
    import gen
    from paper_1209_6449_gb300 import epsm_search_host
    hosts = {}
    for kind in KINDS:
        h = torch.empty(TEXT_N, dtype=torch.uint8, pin_memory=True)
        h.numpy()[:] = gen.TextSpec(kind, 0).host(TEXT_N)
        hosts[kind] = h.numpy()
    groups = {k: [p for (kk, m, p) in pats if kk == k] for k in KINDS}
    # capacity per call: the largest per-text total seen on the device path
    caps = {}
    for k in KINDS:
        st, offs = epsm_search_host(ctx.handle, hosts[k], groups[k],
                                    np.zeros(0, dtype=np.uint64))
        caps[k] = int(offs[-1])
    cap = max(caps.values())
    pos_host = torch.empty(max(cap, 1), dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    d2h = 0

    def step():
        nonlocal d2h
        d2h = 0
        for k in KINDS:
            st, offs = epsm_search_host(ctx.handle, hosts[k], groups[k], pos_host[:cap])
            if st != 0:
                raise SystemExit(f"epsm_search_host status {st}")
            d2h += int(offs[-1]) * 8 + offs.size * 8
    for _ in range(max(1, args.warmup)):
        step()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    if dist:
        tt = torch.tensor([dt], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dt = float(tt.item())
    world = dist.get_world_size() if dist else 1
    scanned = len(pats) * TEXT_N * args.steps * world
    h2d = len(KINDS) * TEXT_N + sum(len(p) for (_, _, p) in pats)
    return {"value": round(scanned / dt / 1e9, 2), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "api": "epsm_search_host (one call per text, "
                                              "pinned host buffers)"}


if __name__ == "__main__":
    sys.exit(main())
