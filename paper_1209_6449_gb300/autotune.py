"""Autotuner of the single search (the EPSM dispatcher of Section 3 picks its
procedure by m; on the GPU the choice is measured, not fixed).

For every text-length bucket of the context's tuning table, every alphabet
class and every pattern length m it times each candidate configuration --
a kernel variant that covers m, a launch shape of the filter kernel (ring
depth and blocks per SM) and, for the block fingerprint variants, the
fingerprint width k (Section 3.4 takes k = 11) -- on texts made by the
workloads' own generators with half planted and half i.i.d. patterns, and
keeps the fastest.  The table is written as JSON; ``apply`` installs the rows
of one alphabet class (or the rows that are best over all classes, "mixed")
into a context.  ``Context`` loads ``tuning.json`` next to this file when it
exists.

Run on the target GPU:  python -m paper_1209_6449_gb300.autotune [out.json]
"""
from __future__ import annotations

import json
import os
import sys
import time

from ._native import (BUCKET_MIN, SHAPES, TEXT_BUCKETS, VARIANT_ADAPT, VARIANT_BLOCK4, VARIANT_BLOCK8,
                      VARIANT_BLOCK8S, VARIANT_CODE2, VARIANT_DIRECT, VARIANT_NAMES, VARIANT_PREFIX4,
                      VARIANT_PREFIX8)

COVER = {VARIANT_DIRECT: range(1, 5), VARIANT_PREFIX4: range(4, 16),
         VARIANT_PREFIX8: range(8, 16), VARIANT_BLOCK8: range(15, 33), VARIANT_BLOCK4: range(7, 17),
         VARIANT_CODE2: range(2, 17), VARIANT_ADAPT: range(5, 17), VARIANT_BLOCK8S: range(23, 33)}
BLOCK_VARIANTS = (VARIANT_BLOCK8, VARIANT_BLOCK8S)
KBITS = (11, 14)            # fingerprint widths tried for the block variants
DEFAULT_KBITS = 14
DEFAULT_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")
# alphabet classes and the generator kinds they are measured on (the DNA-like
# class includes the text with runs of A, searched also with A^m, so that its
# rows hold up on periodic stretches)
CLASSES = {"dna": ("dna", "dna_runs"), "protein": ("protein",), "text": ("nl64", "markov96")}
# one text length per bucket of the tuning table
BUCKET_N = (4 << 20, 128 << 20, 1 << 30)


def variants_for(m: int):
    return [v for v, r in COVER.items() if m in r]


def candidates(m: int):
    """(variant, shape, kbits) configurations tried for pattern length m."""
    out = []
    for v in variants_for(m):
        for sh in range(SHAPES):
            for kb in (KBITS if v in BLOCK_VARIANTS else (DEFAULT_KBITS,)):
                out.append((v, sh, kb))
    return out


def _time_config(ctx, torch, texts, pats, cfg, bucket, m, reps, out, cap, cnt):
    v, sh, kb = cfg
    ctx.set_tuning(bucket, m, v, sh, kb)
    for t, ps in zip(texts, pats):          # warm-up
        for p in ps:
            ctx.search_async(t, p, out, cap, cnt)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        for t, ps in zip(texts, pats):
            for p in ps:
                ctx.search_async(t, p, out, cap, cnt)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(ctx, ms=range(1, 33), buckets=range(TEXT_BUCKETS), classes=tuple(CLASSES),
             bucket_n=BUCKET_N, reps: int = 3, patterns: int = 2, seed: int = 0) -> dict:
    """Measure every candidate configuration; returns the tuning table."""
    import torch
    import gen
    table = {"version": 2, "bucket_min": list(BUCKET_MIN), "bucket_n": {}, "classes": {},
             "ms": {}, "kinds": {c: list(CLASSES[c]) for c in classes}}
    for b in buckets:
        n = bucket_n[b]
        table["bucket_n"][str(b)] = n
        cap = n // 2
        out = torch.empty(cap, dtype=torch.int64, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        for cls in classes:
            texts, specs = [], []
            for kind in CLASSES[cls]:
                spec = gen.TextSpec(kind, seed)
                t = torch.empty(n, dtype=torch.uint8, device="cuda")
                spec.device(n, t.data_ptr(), torch.cuda.current_stream().cuda_stream)
                texts.append(t)
                specs.append(spec)
            rows = table["classes"].setdefault(cls, {}).setdefault(str(b), {})
            times = table["ms"].setdefault(cls, {}).setdefault(str(b), {})
            for m in ms:
                pats = [gen.mixed_patterns(sp, n, m, patterns, stream_seed=7) +
                        ([b"A" * m] if sp.kind == "dna_runs" else []) for sp in specs]
                res = {}
                for cfg in candidates(m):
                    res[cfg] = _time_config(ctx, torch, texts, pats, cfg, b, m, reps, out, cap, cnt)
                best = min(res, key=res.get)
                rows[str(m)] = {"variant": best[0], "shape": best[1], "kbits": best[2],
                                "name": VARIANT_NAMES[best[0]]}
                times[str(m)] = {f"{VARIANT_NAMES[v]}/{sh}/{kb}": round(t, 4)
                                 for (v, sh, kb), t in res.items()}
            del texts
        del out
        torch.cuda.empty_cache()
    if ctx.sync() != 0:
        raise RuntimeError("device error during autotuning")
    table["classes"]["mixed"] = mixed_rows(table)
    table["when"] = time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())
    return table


def mixed_rows(table: dict) -> dict:
    """Per (bucket, m): the configuration whose time, relative to each class's
    best, is smallest summed over the classes (for texts of unknown class)."""
    rows = {}
    for b, by_m in next(iter(table["ms"].values())).items():
        for m in by_m:
            score = {}
            for cls, tb in table["ms"].items():
                res = tb[b][m]
                best = min(res.values())
                for key, t in res.items():
                    score[key] = score.get(key, 0.0) + t / best
            key = min(score, key=score.get)
            name, sh, kb = key.split("/")
            v = next(v for v, nm in VARIANT_NAMES.items() if nm == name)
            rows.setdefault(b, {})[m] = {"variant": v, "shape": int(sh), "kbits": int(kb), "name": name}
    return rows


def apply(ctx, table: dict, text_class: str = "mixed") -> None:
    """Installs the rows of one alphabet class (every bucket and m) into a context."""
    rows = table["classes"][text_class]
    for b, by_m in rows.items():
        for m, r in by_m.items():
            ctx.set_tuning(int(b), int(m), int(r["variant"]), int(r["shape"]), int(r["kbits"]))


def load(path: str = DEFAULT_PATH):
    if not os.path.exists(path):
        return None
    with open(path) as f:
        t = json.load(f)
    return t if t.get("version") == 2 else None


if __name__ == "__main__":
    from . import Context
    ctx = Context(0, tuning=None)
    res = autotune(ctx)
    out = sys.argv[1] if len(sys.argv) > 1 else DEFAULT_PATH
    with open(out, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps({c: {b: {m: r["name"] for m, r in bm.items()} for b, bm in rows.items()}
                      for c, rows in res["classes"].items()}))
