"""Hand-built test texts (seeded) that the generators do not make."""
import numpy as np

import gen


def periodic_runs_text(n, seed):
    """A DNA-like text in which runs of a periodic string (period 1..10, the
    runs of varying length and phase) cover about a third of the bytes."""
    rng = np.random.default_rng(seed)
    host = gen.TextSpec("dna", seed).host(n).copy()
    units = [b"A", b"AC", b"ACG", b"ACGT", b"AACG", b"ACGTT", b"AACCGG", b"ACGTACG", b"AACGTTGC",
             b"ACGTTGCAT", b"ACGGTACCAT"]
    pos = 0
    while pos < n:
        pos += int(rng.integers(0, 400))
        u = units[int(rng.integers(0, len(units)))]
        ln = int(rng.integers(1, 200))
        run = np.frombuffer((u * (ln // len(u) + 2))[int(rng.integers(0, len(u))):][:ln], dtype=np.uint8)
        k = min(run.size, n - pos)
        if k > 0:
            host[pos:pos + k] = run[:k]
        pos += ln
    return host, units
