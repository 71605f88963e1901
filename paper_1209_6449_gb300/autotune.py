"""Autotuner for the per-m kernel variant (the EPSM dispatcher of Section 3
chooses its procedure by m; on the GPU the choice is measured, not fixed).

For every pattern length m it times each variant that covers m on texts over
the workloads' alphabets (uniform random bytes over the DNA letters ACGT, the
20 amino-acid letters and a 64-symbol natural-language set, with patterns
copied from the text) and keeps the variant with the smallest total time.  The
table is written as JSON and installed into a context with ``apply``.
``Context`` loads ``tuning.json`` next to this file when it exists.

Run on the target GPU:  python -m paper_1209_6449_gb300.autotune [out.json]
"""
from __future__ import annotations

import json
import os
import sys
import time

from ._native import (VARIANT_ADAPT, VARIANT_BLOCK4, VARIANT_BLOCK8, VARIANT_BLOCK8S, VARIANT_CODE2,
                      VARIANT_DIRECT, VARIANT_NAMES, VARIANT_PREFIX4, VARIANT_PREFIX8)

COVER = {VARIANT_DIRECT: range(1, 5), VARIANT_PREFIX4: range(4, 16),
         VARIANT_PREFIX8: range(8, 16), VARIANT_BLOCK8: range(15, 33), VARIANT_BLOCK4: range(7, 17),
         VARIANT_CODE2: range(2, 17), VARIANT_ADAPT: range(5, 17), VARIANT_BLOCK8S: range(23, 33)}
DEFAULT_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")


def variants_for(m: int):
    return [v for v, r in COVER.items() if m in r]


ALPHABETS = (b"ACGT", b"ACDEFGHIKLMNPQRSTVWY",
             b" abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ0123456789.")


def autotune(ctx, n: int = 64 << 20, alphabets=ALPHABETS, ms=range(1, 33), reps: int = 3,
             patterns: int = 4, seed: int = 0) -> dict:
    """Measure every (m, variant) and return the tuning table."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    texts = []
    for alpha in alphabets:
        sym = torch.tensor(list(alpha), dtype=torch.uint8)
        idx = torch.randint(0, len(alpha), (n,), generator=g)
        texts.append(sym[idx].cuda())
    cap = n // 2
    out = torch.empty(cap, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    table, detail = {}, {}
    for m in ms:
        best, best_t = None, None
        times = {}
        for v in variants_for(m):
            total = 0.0
            for t in texts:
                offs = torch.randint(0, n - m, (patterns,), generator=g).tolist()
                pats = [bytes(t[o:o + m].cpu().numpy()) for o in offs]
                for p in pats:  # warm-up
                    ctx.search_async(t, p, out, cap, cnt, variant=v)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    for p in pats:
                        ctx.search_async(t, p, out, cap, cnt, variant=v)
                e1.record()
                torch.cuda.synchronize()
                total += e0.elapsed_time(e1) / (reps * len(pats))
            times[VARIANT_NAMES[v]] = round(total, 4)
            if best_t is None or total < best_t:
                best, best_t = v, total
        table[m] = best
        detail[m] = times
    if ctx.sync() != 0:
        raise RuntimeError("device error during autotuning")
    return {"variant": {str(m): v for m, v in table.items()},
            "names": {str(m): VARIANT_NAMES[v] for m, v in table.items()},
            "ms_per_search": {str(m): d for m, d in detail.items()},
            "text_bytes": n, "alphabets": [a.decode() for a in alphabets], "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}


def apply(ctx, table: dict) -> None:
    for m, v in table["variant"].items():
        ctx.set_variant(int(m), int(v))


def load(path: str = DEFAULT_PATH):
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


if __name__ == "__main__":
    from . import Context
    ctx = Context(0)
    res = autotune(ctx)
    out = sys.argv[1] if len(sys.argv) > 1 else DEFAULT_PATH
    with open(out, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res["names"]))
