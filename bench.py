#!/usr/bin/env python3
"""Benchmark: exact short-pattern search throughput on GB300.

Workload (default, the large single-GPU scan): three synthetic texts of
n = 16 GiB each, resident in HBM -- sigma=4 uniform DNA-like bytes, an order-2
Markov chain over 96 printable ASCII bytes with seeded transition rows, and
the DNA-like text with seeded runs of ``A`` covering about 5% of its bytes.
For the DNA-like and Markov texts, m in {2,3,4,6,8,12,16,24,32} with one
pattern copied from a random text offset and one drawn i.i.d. from the text's
symbol distribution; for the runs text the adversarial periodic pattern A^m
for every m.  One step searches every (text, pattern) pair: 45 searches,
773 GB of text.  Each search produces its count and all sorted uint64 start
positions.

Metric: text GB/s (bytes of text scanned / second), device-timed with the
texts resident in HBM (inputs far larger than the 129 MB L2).  ``per_text_m``
breaks it down per (text, m) from a separate pass with CUDA events between
searches, with the fraction of the measured HBM peak taken on the algorithmic
bytes (n + 8 per position + 8).  ``e2e`` is the same metric through the public
C entry point that takes HOST buffers (epsm_search_host: one call per text,
its single searches, the text's host->device copy and the positions'
device->host copy inside the timed region).  ``sweep`` is the pattern-length
sweep (three 256 MiB texts, m in {2,4,8,16,32}, 100 patterns each);
``batched`` and ``served`` are the batched and served workloads against the
plain per-pair / per-query launch path.

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
UNIT = "GB/s"
L2_BYTES = 129 * 10**6
# large single-GPU scan (the headline)
METRIC = "text GB/s (large single-GPU scan, m=2..32, 16 GiB texts)"
SCAN_KINDS = ("dna", "markov96", "dna_runs")
SCAN_MS = (2, 3, 4, 6, 8, 12, 16, 24, 32)
SCAN_N = 16 * GiB
# pattern-length sweep
SWEEP_METRIC = "text GB/s (pattern-length sweep, m=2..32, 256 MiB texts)"
KINDS = ("dna", "protein", "nl64")
MS = (2, 4, 8, 16, 32)
PATS_PER_M = 100
TEXT_N = 256 * MiB


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="epsm", choices=["epsm", "reference"])
    ap.add_argument("--workload", default="scan", choices=["scan", "sweep"],
                    help="headline workload: the large single-GPU scan (default) or the "
                         "pattern-length sweep")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the sweep's extra key")
    ap.add_argument("--patterns", type=int, default=PATS_PER_M,
                    help="sweep: patterns per (text, m); the workload uses 100")
    ap.add_argument("--case", default=None,
                    help="KIND:M[:VARIANT[:N[:MODE]]] -- time one search of an N-byte text "
                         "(default 256 MiB; a count-only search first sizes the output) and "
                         "exit (the small cases of ncu captures); MODE "
                         "'count': count only; 'iid': an i.i.d. pattern instead of a planted "
                         "one; 'runs': the pattern A^m")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--sample", action="store_true",
                    help="one search per (text, m) of the sweep (15 launches) and exit")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-pairs", type=int, default=8192)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-rates", default="2000,5000,10000,20000,50000",
                    help="Poisson arrival rates (queries/s) of the served workload")
    ap.add_argument("--serve-secs", type=float, default=1.0,
                    help="arrival window per rate for the serving engine")
    ap.add_argument("--serve-pq-secs", type=float, default=0.25,
                    help="arrival window per rate for the per-query path (it saturates early)")
    ap.add_argument("--served-only", action="store_true",
                    help="run the served workload alone and print its JSON (the main run starts "
                         "it this way, in a child process with a time limit)")
    ap.add_argument("--serve-timeout", type=float, default=300.0,
                    help="seconds the served workload's child process may take")
    return ap.parse_args()


def run_case(args):
    """One search configuration, timed with CUDA events (for profiling)."""
    import torch
    import gen
    import paper_1209_6449_gb300 as epsm
    parts = args.case.split(":")
    kind, m = parts[0], int(parts[1])
    variant = int(parts[2]) if len(parts) > 2 and parts[2] else 0
    n = int(parts[3]) if len(parts) > 3 and parts[3] else TEXT_N
    mode = parts[4] if len(parts) > 4 else ""
    ctx = epsm.Context(0, text_class=KIND_CLASS.get(kind, "mixed"))
    spec = gen.TextSpec(kind, 0)
    t = torch.empty(n, dtype=torch.uint8, device="cuda")
    spec.device(n, t.data_ptr(), torch.cuda.current_stream().cuda_stream)
    if mode == "runs":
        pat = b"A" * m
    elif mode == "iid":
        pat = gen.random_patterns(spec, m, 1)[0]
    else:
        pat = gen.planted_patterns(spec, n, m, 1)[0]
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    # a count-only search first sizes the output (the first launch of a case)
    ctx.search_async(t, pat, cnt, 0, cnt, variant=variant)
    torch.cuda.synchronize()
    cap = 0 if mode == "count" else int(cnt.item()) + 1024
    out = torch.empty(max(cap, 1), dtype=torch.int64, device="cuda")
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
    c = int(cnt.item())
    best = min(times)
    print(json.dumps({"case": args.case, "n": n, "count": c, "status": st,
                      "ms": [round(x, 4) for x in times],
                      "gbs_best": round(n / best / 1e6, 1),
                      "alg_gbs_best": round((n + 8 * c + 8) / best / 1e6, 1)}), flush=True)
    ctx.close()
    return 0 if st == 0 else 1


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def scan_patterns():
    """(text, m, kind of pattern, pattern) of one step of the large scan."""
    import gen
    out = []
    for kind in ("dna", "markov96"):
        spec = gen.TextSpec(kind, 0)
        for m in SCAN_MS:
            out.append((kind, m, "planted", gen.planted_patterns(spec, SCAN_N, m, 1)[0]))
            out.append((kind, m, "iid", gen.random_patterns(spec, m, 1)[0]))
    for m in SCAN_MS:
        out.append(("dna_runs", m, "runs", b"A" * m))
    return out


def scan_config(ngpus):
    return {"workload": "large single-GPU scan: 16 GiB sigma-4 uniform DNA-like text, 16 GiB "
                        "order-2 Markov text over 96 printable bytes, 16 GiB DNA-like text with "
                        "5% runs of A; m in {2,3,4,6,8,12,16,24,32}: one planted and one i.i.d. "
                        "pattern per (text, m) on the first two, A^m on the runs text",
            "text_bytes": SCAN_N, "texts": list(SCAN_KINDS), "m": list(SCAN_MS),
            "searches_per_step": 2 * 2 * len(SCAN_MS) + len(SCAN_MS),
            "l2": "inputs larger than L2 (16 GiB texts vs 129 MB L2); no flush",
            "parallelism": f"replicas x{ngpus}" if ngpus > 1 else "single GPU"}


def sweep_patterns(npat):
    import gen
    out = []
    for kind in KINDS:
        spec = gen.TextSpec(kind, 0)
        for m in MS:
            for i, p in enumerate(gen.mixed_patterns(spec, TEXT_N, m, npat)):
                out.append((kind, m, "planted" if i < npat - npat // 2 else "iid", p))
    return out


def sweep_config(npat, ngpus):
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

def oracle_jobs(workload, sample_n):
    """A bounded sample of the workload for the oracle: the first sample_n
    bytes of each text, one pattern per (text, m)."""
    import gen
    if workload == "scan":
        texts = {k: gen.TextSpec(k, 0).host_parallel(sample_n) for k in SCAN_KINDS}
        pats = [(k, m, p) for (k, m, kind, p) in scan_patterns() if kind != "iid"]
        desc = "3 texts x 9 m x 1 pattern (planted; A^m on the runs text)"
    else:
        texts = {k: gen.TextSpec(k, 0).host(sample_n) for k in KINDS}
        pats = [(k, m, gen.mixed_patterns(gen.TextSpec(k, 0), TEXT_N, m, 2)[0])
                for k in KINDS for m in MS]
        desc = "3 texts x 5 m x 1 pattern (planted)"
    return [(texts[k], p) for (k, m, p) in pats], desc


def oracle_rate(jobs, threads, budget_s):
    """Rounds of the oracle over the jobs until about budget_s seconds."""
    import oracle
    scanned, rounds = 0, 0
    t0 = time.perf_counter()
    while True:
        for t, p in jobs:
            oracle.search(t, p, threads=threads)
            scanned += t.size
        rounds += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return scanned / dt / 1e9, rounds


def cpu_baseline(workload, budget_s=10.0):
    """The oracle (count and all positions) timed on all host cores and on one
    core, on a bounded sample of the workload."""
    cores = os.cpu_count() or 1
    sample_n = 16 * MiB if workload == "scan" else 8 * MiB
    jobs, desc = oracle_jobs(workload, sample_n)
    v_all, r_all = oracle_rate(jobs, cores, budget_s)
    v_one, r_one = oracle_rate(jobs, 1, budget_s)
    sample = (f"{len(jobs)} searches ({desc}) over the first {sample_n // MiB} MiB of each text, "
              f"brute-force C oracle returning all positions")
    return {"value": round(v_all, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{r_all} round(s) of {sample} on {cores} threads",
            "single_thread": {"value": round(v_one, 4), "unit": UNIT, "cores": 1,
                              "sample": f"{r_one} round(s) of {sample} on 1 thread"}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    cores = os.cpu_count() or 1
    sample_n = 8 * MiB if args.workload == "scan" else 4 * MiB
    jobs, desc = oracle_jobs(args.workload, sample_n)

    def step():
        tot = 0
        for t, p in jobs:
            oracle.search(t, p, threads=cores)
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
    sample = (f"each step: {len(jobs)} searches ({desc}) over the first {sample_n // MiB} MiB of "
              f"each text, brute-force C oracle returning all positions, on {cores} threads")
    cfg = scan_config(args.gpus) if args.workload == "scan" else sweep_config(args.patterns, args.gpus)
    line = {"impl": "reference", "metric": METRIC if args.workload == "scan" else SWEEP_METRIC,
            "value": round(v, 4), "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": cfg,
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


# the files the single search's kernels and their launch choices come from
# (the batched and served forms, and the host runtime, do not change them)
SINGLE_SEARCH_SOURCES = ("csrc/epsm_kernels.cuh", "csrc/epsm_scan.cuh", "csrc/epsm_stream.cuh",
                         "csrc/epsm_tile.cuh", "tuning.json")


def kernel_source_hash():
    h = hashlib.sha256()
    pkg = os.path.join(ROOT, "paper_1209_6449_gb300")
    for f in SINGLE_SEARCH_SOURCES:
        with open(os.path.join(pkg, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload):
    """DRAM bytes per search from the committed ncu summary of this workload,
    if it was taken on the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", f"traffic_{workload}.json")
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
    """One search per (text, m) of the sweep, with the first (planted) pattern."""
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


# alphabet class of each text kind (rows of the tuning table a context uses)
KIND_CLASS = {"dna": "dna", "dna_runs": "dna", "protein": "protein", "nl64": "text",
              "markov96": "text"}


class Contexts:
    """One library context per alphabet class of the workload's texts, each
    with its class's rows of the tuning table."""

    def __init__(self, epsm, device, kinds):
        self.by_class = {c: epsm.Context(device, text_class=c)
                         for c in sorted({KIND_CLASS[k] for k in kinds})}

    def __getitem__(self, kind):
        return self.by_class[KIND_CLASS[kind]]

    @property
    def launch_count(self):
        return sum(c.launch_count for c in self.by_class.values())

    def sync(self):
        st = 0
        for c in self.by_class.values():
            st = st or c.sync()
        return st

    def close(self):
        for c in self.by_class.values():
            c.close()


def make_texts(torch, dev, kinds, n, stream):
    import gen
    texts = {}
    for kind in kinds:
        t = torch.empty(n, dtype=torch.uint8, device=dev)
        gen.TextSpec(kind, 0).device(n, t.data_ptr(), stream.cuda_stream)
        texts[kind] = t
    return texts


def measure(ctx, torch, texts, pats, steps, warmup, stream, dist=None, clocks_index=None):
    """Times `steps` passes over all (text, pattern) searches (after `warmup`
    untimed passes): device time with CUDA events on the launching stream,
    max over ranks.  Then one more pass with an event between searches gives
    the per-search times.  Returns a dict of the measurements."""
    n_by = {k: t.numel() for k, t in texts.items()}
    nsearch = len(pats)
    counts = torch.zeros(nsearch, dtype=torch.int64, device=stream.device)
    # output room: the densest search of the workload (from a count-only pass)
    for i, (kind, m, _, p) in enumerate(pats):
        ctx[kind].search_async(texts[kind], p, counts, 0, counts[i:i + 1], stream=stream)
    torch.cuda.synchronize()
    if ctx.sync() != 0:
        raise SystemExit("device status after the count pass")
    occ = counts.cpu().numpy().copy()
    cap = int(occ.max()) + 1024
    out = torch.empty(cap, dtype=torch.int64, device=stream.device)

    def step():
        for i, (kind, m, _, p) in enumerate(pats):
            ctx[kind].search_async(texts[kind], p, out, cap, counts[i:i + 1], stream=stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if ctx.sync() != 0:
        raise SystemExit("device status after warm-up")
    if not np.array_equal(counts.cpu().numpy(), occ):
        raise SystemExit("counts differ between the count pass and the searches")

    clocks = ClockSampler(clocks_index if clocks_index is not None else 0)
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
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    if dist:
        dist.barrier()
    launches = ctx.launch_count - launches_before
    elapsed_ms = e0.elapsed_time(e1)
    clocks.stop()
    if ctx.sync() != 0:
        raise SystemExit("device status after the timed region")
    if dist:
        tt = torch.tensor([elapsed_ms], dtype=torch.float64, device=stream.device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed_ms = float(tt.item())
    # per-search times: one more pass with an event after every search
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(nsearch + 1)]
    evs[0].record(stream)
    for i, (kind, m, _, p) in enumerate(pats):
        ctx[kind].search_async(texts[kind], p, out, cap, counts[i:i + 1], stream=stream)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    per = [evs[i].elapsed_time(evs[i + 1]) for i in range(nsearch)]
    del out
    text_bytes = sum(n_by[k] for (k, _, _, _) in pats)
    alg_bytes = text_bytes + 8 * int(occ.sum()) + 8 * nsearch
    return {"elapsed_ms": elapsed_ms, "steps": steps, "launches": launches, "occ": occ,
            "per_search_ms": per, "text_bytes_per_step": text_bytes,
            "alg_bytes_per_step": alg_bytes, "clocks": clocks.summary(t_wall0, t_wall1),
            "n_by": n_by}


def breakdown(pats, res, peak):
    """Per (text, m, pattern kind): text GB/s and algorithmic GB/s of the
    per-search pass (summed over that group's patterns), and the fraction of
    the HBM peak on the algorithmic bytes."""
    acc = {}
    for i, (kind, m, pk, p) in enumerate(pats):
        a = acc.setdefault((kind, m, pk), [0.0, 0, 0, 0])
        n = res["n_by"][kind]
        occ = int(res["occ"][i])
        a[0] += res["per_search_ms"][i]
        a[1] += occ
        a[2] += n
        a[3] += n + 8 * occ + 8
    rows = {}
    for (kind, m, pk), (ms, occ, nb, alg) in acc.items():
        rows.setdefault(kind, {})[f"{m}/{pk}"] = {
            "ms": round(ms, 3), "occ": occ, "text_gbs": round(nb / ms / 1e6, 1),
            "alg_gbs": round(alg / ms / 1e6, 1), "frac": round(alg / ms / 1e6 / peak, 3)}
    return rows


def _mem_available():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def run_e2e(ctx, torch, texts, pats, steps, warmup, occ, dist=None):
    """The same workload through epsm_search_host (host text in, host positions
    out): every step copies each text from pinned host memory to the device,
    runs its single searches and copies all positions back.  One call per text
    with all its patterns when the pinned buffers fit in 55% of the host's
    available memory; otherwise a text's patterns are split over several calls
    (each uploads the text again, counted in h2d_bytes_per_step)."""
    from paper_1209_6449_gb300 import epsm_search_host
    kinds = list(dict.fromkeys(k for (k, _, _, _) in pats))
    text_bytes = sum(texts[k].numel() for k in kinds)
    budget = max(_mem_available() * 11 // 20 - text_bytes, 1 << 30)
    cap = max(int(occ.max()) + 1024, min(budget // 8, int(occ.sum()) + 1024))
    calls = []  # (text kind, patterns)
    for k in kinds:
        cur, tot = [], 0
        for i, (kk, _, _, p) in enumerate(pats):
            if kk != k:
                continue
            if cur and tot + int(occ[i]) > cap - 1024:
                calls.append((k, cur))
                cur, tot = [], 0
            cur.append(p)
            tot += int(occ[i])
        calls.append((k, cur))
    hosts = {}
    for k in kinds:
        h = torch.empty(texts[k].numel(), dtype=torch.uint8, pin_memory=True)
        h.copy_(texts[k])
        hosts[k] = h.numpy()
    pos_host = torch.empty(cap, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)

    def step():
        d2h = 0
        for k, group in calls:
            st, offs = epsm_search_host(ctx[k].handle, hosts[k], group, pos_host)
            if st != 0:
                raise SystemExit(f"epsm_search_host status {st}")
            d2h += int(offs[-1]) * 8
        return d2h

    for _ in range(warmup):
        step()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(steps):
        d2h = step()
    dt = time.perf_counter() - t0
    if dist:
        tt = torch.tensor([dt], dtype=torch.float64, device=texts[kinds[0]].device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dt = float(tt.item())
    world = dist.get_world_size() if dist else 1
    scanned = sum(texts[k].numel() for (k, _, _, _) in pats) * steps * world
    h2d = sum(texts[k].numel() + sum(len(p) for p in g) for k, g in calls)
    del hosts, pos_host
    return {"value": round(scanned / dt / 1e9, 2), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": steps, "calls_per_step": len(calls),
            "api": "epsm_search_host (host text in, host positions out; its single searches "
                   "run the same kernels as the device-timed value), pinned host buffers, "
                   "wall clock"}


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


def run_served_child(args):
    """The served workload in a child process with a time limit, so that a
    stalled serving engine cannot hold up the rest of the report."""
    cmd = [sys.executable, os.path.abspath(__file__), "--served-only", "--serve-rates", args.serve_rates,
           "--serve-secs", str(args.serve_secs), "--serve-pq-secs", str(args.serve_pq_secs)]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=args.serve_timeout)
    except subprocess.TimeoutExpired:
        return {"unavailable": f"served workload did not finish within {args.serve_timeout:.0f} s"}
    lines = [x for x in r.stdout.strip().splitlines() if x.startswith("{")]
    if r.returncode != 0 or not lines:
        return {"unavailable": f"served workload failed (exit {r.returncode}): {r.stderr.strip()[-300:]}"}
    return json.loads(lines[-1])


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


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.case:
        return run_case(args)
    if args.served_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(run_served(torch, args)), flush=True)
        return 0
    if args.sample:
        return run_sample(args)

    import torch
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
    ctx = Contexts(epsm, dev.index, SCAN_KINDS + KINDS)
    stream = torch.cuda.current_stream()
    peak, peak_kind = measured_peaks()

    if args.workload == "scan":
        pats = scan_patterns()
        texts = make_texts(torch, dev, SCAN_KINDS, SCAN_N, stream)
        cfg, metric = scan_config(world), METRIC
    else:
        pats = sweep_patterns(args.patterns)
        texts = make_texts(torch, dev, KINDS, TEXT_N, stream)
        cfg, metric = sweep_config(args.patterns, world), SWEEP_METRIC
    torch.cuda.synchronize()
    res = measure(ctx, torch, texts, pats, args.steps, args.warmup, stream, dist, dev.index)
    value = world * res["text_bytes_per_step"] * args.steps / (res["elapsed_ms"] / 1e3) / 1e9
    nsearch = len(pats)
    per_launch_s = res["elapsed_ms"] / 1e3 / max(args.steps * nsearch, 1)
    alg_per_launch = res["alg_bytes_per_step"] / nsearch
    achieved = alg_per_launch / per_launch_s / 1e9
    traffic = profiled_traffic(args.workload)
    rows = breakdown(pats, res, peak)

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(ctx, torch, texts, pats, min(args.steps, 5), 1, res["occ"], dist)
    del texts
    torch.cuda.empty_cache()
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(args.workload)
    sweep = None
    if args.workload == "scan" and not args.no_sweep:
        spats = sweep_patterns(args.patterns)
        stexts = make_texts(torch, dev, KINDS, TEXT_N, stream)
        sres = measure(ctx, torch, stexts, spats, max(1, args.steps // 2), args.warmup, stream, dist,
                       dev.index)
        del stexts
        torch.cuda.empty_cache()
        s_nsearch = len(spats)
        s_alg = sres["alg_bytes_per_step"] / s_nsearch
        s_per = sres["elapsed_ms"] / 1e3 / (sres["steps"] * s_nsearch)
        sweep = {"metric": SWEEP_METRIC, "config": sweep_config(args.patterns, world),
                 "value": round(world * sres["text_bytes_per_step"] * sres["steps"] /
                                (sres["elapsed_ms"] / 1e3) / 1e9, 2),
                 "unit": UNIT, "steps": sres["steps"],
                 "ms_per_step": round(sres["elapsed_ms"] / sres["steps"], 3),
                 "roofline": {"bound": "hbm", "achieved": round(s_alg / s_per / 1e9, 1),
                              "peak": peak, "unit": "GB/s",
                              "frac": round(s_alg / s_per / 1e9 / peak, 4)},
                 "per_text_m": {k: {mk: v for mk, v in d.items()}
                                for k, d in breakdown(spats, sres, peak).items()},
                 "clocks": sres["clocks"]}
    batched = None
    if not args.no_batch:
        batched = run_batched(ctx["dna"], torch, args.batch_pairs)
    served = None
    if not args.no_serve and world == 1:
        torch.cuda.empty_cache()
        served = run_served_child(args)

    if rank == 0:
        line = {"metric": metric, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(res["elapsed_ms"] / args.steps, 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
                "config": cfg,
                "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                             "unit": "GB/s", "frac": round(achieved / peak, 4),
                             "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs: copy "
                                            "bandwidth, burst)",
                             "kernel": "one search (stream_kernel filter + stream_emit_kernel), "
                                       "all variants; algorithmic bytes = n + 8*occ + 8 per search",
                             "alg_bytes_per_launch": round(alg_per_launch),
                             "traffic": traffic.get("bytes_per_launch") if traffic else None,
                             "traffic_note": (traffic.get("note") if traffic else
                                              "null: no ncu capture of the current kernel sources")},
                "per_text_m": rows,
                "cpu_baseline": cpu,
                "e2e": e2e,
                "sweep": sweep,
                "batched": batched,
                "served": served,
                "gpu_launches": res["launches"],
                "clocks": res["clocks"],
                "occurrences_per_step": int(res["occ"].sum())}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
