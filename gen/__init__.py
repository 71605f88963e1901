"""Seeded synthetic inputs shaped like the paper's workloads (Section 4).

This module serves the tests and the benchmark.  It holds none of the string
matching arithmetic: it only makes texts and patterns.  The byte streams are
defined in ``textgen.h`` (SplitMix64 in counter mode) and are produced either on
the host (``libgen_host.so``, gcc) or directly in device memory
(``libgen_cuda.so``, nvcc) with identical results, so multi-GiB texts never
cross the host-device link.

Text kinds (the paper searched 4 MB genome, protein and English texts; these
synthetic stand-ins take their alphabets and symbol statistics):

``dna``       i.i.d. uniform over ``ACGT`` (sigma = 4)
``protein``   i.i.d. uniform over the 20 amino-acid letters
``nl64``      64 symbols: space with p = 0.15, 63 symbols ``a-z A-Z 0-9 .``
              with p proportional to rank**-1.1 (Zipf s = 1.1), rank order
              fixed by the seed
``markov96``  order-2 Markov chain over the 95 printable ASCII bytes plus
              ``\\n``; each of the 96*96 contexts has a seeded row of
              exponential-variate weights; generated in independent 64 KiB
              segments
``dna_runs``  ``dna`` with seeded runs of ``A`` covering about 5% of bytes
``bytes256``  i.i.d. uniform over all 256 byte values
``binary``    i.i.d. uniform over two byte values (0x00 and 0xFF)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_HOST_LIB = os.path.join(_HERE, "libgen_host.so")
_CUDA_LIB = os.path.join(_HERE, "libgen_cuda.so")
_lock = threading.Lock()
_host = None
_cuda = None

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15

DNA = b"ACGT"
PROTEIN = b"ACDEFGHIKLMNPQRSTVWY"
NL63 = b"abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ0123456789."
MARKOV96 = bytes(range(0x20, 0x7F)) + b"\n"
RUN_BLOCK = 1240       # one run per 1240-byte block ...
RUN_MAXLEN = 127       # ... of length uniform in [1, 127]: about 5% of bytes
STREAM_TEXT = 1
STREAM_RUNS = 2
STREAM_PAT_OFFSET = 3
STREAM_PAT_RANDOM = 4
STREAM_TABLE = 5
STREAM_BATCH = 6


# ---------------------------------------------------------------------------
# builds
# ---------------------------------------------------------------------------

def _newer(out, *srcs):
    return os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(s) for s in srcs)


def build(cuda: bool = True, force: bool = False) -> None:
    """Compile the host generator (gcc) and, if requested, the device one (nvcc)."""
    hdr = os.path.join(_HERE, "textgen.h")
    src = os.path.join(_HERE, "gen_host.c")
    if force or not _newer(_HOST_LIB, src, hdr):
        tmp = _HOST_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, _HOST_LIB)
    if cuda:
        csrc = os.path.join(_HERE, "gen_cuda.cu")
        if force or not _newer(_CUDA_LIB, csrc, hdr):
            tmp = _CUDA_LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                                   "-shared", "-Xcompiler", "-fPIC", "-o", tmp, csrc])
            os.replace(tmp, _CUDA_LIB)


def _host_lib():
    global _host
    with _lock:
        if _host is None:
            build(cuda=False)
            lib = ctypes.CDLL(_HOST_LIB)
            vp, u64 = ctypes.c_void_p, ctypes.c_uint64
            lib.gen_fill_iid.argtypes = [vp, u64, u64, u64, vp]
            lib.gen_fill_markov.argtypes = [vp, u64, u64, u64, vp, vp, vp]
            lib.gen_apply_runs.argtypes = [vp, u64, u64, u64, u64, ctypes.c_uint32, ctypes.c_uint8]
            for f in (lib.gen_fill_iid, lib.gen_fill_markov, lib.gen_apply_runs):
                f.restype = None
            _host = lib
    return _host


def _cuda_lib():
    global _cuda
    with _lock:
        if _cuda is None:
            build(cuda=True)
            lib = ctypes.CDLL(_CUDA_LIB)
            vp, u64 = ctypes.c_void_p, ctypes.c_uint64
            lib.gen_fill_iid_device.argtypes = [vp, u64, u64, u64, vp, vp]
            lib.gen_fill_markov_device.argtypes = [vp, u64, u64, u64, vp, vp, vp, vp]
            lib.gen_apply_runs_device.argtypes = [vp, u64, u64, u64, u64, ctypes.c_uint32,
                                                  ctypes.c_uint8, vp]
            for f in (lib.gen_fill_iid_device, lib.gen_fill_markov_device,
                      lib.gen_apply_runs_device):
                f.restype = ctypes.c_int
            _cuda = lib
    return _cuda


# ---------------------------------------------------------------------------
# SplitMix64 in Python (same definition as textgen.h) for keys and small draws
# ---------------------------------------------------------------------------

def mix64(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def key(seed: int, stream: int) -> int:
    return mix64(mix64(seed + GOLDEN) ^ ((stream * 0xD1B54A32D192ED03 + 1) & MASK64))


def draw(k: int, i: int) -> int:
    return mix64(k + ((i + 1) * GOLDEN & MASK64))


def draws(k: int, idx: np.ndarray) -> np.ndarray:
    """Vectorised ``draw`` over an index array (uint64 arithmetic wraps)."""
    with np.errstate(over="ignore"):
        z = np.uint64(k) + (idx.astype(np.uint64) + np.uint64(1)) * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform01(k: int, idx: np.ndarray) -> np.ndarray:
    """Floats in (0, 1) from the top 53 bits of each draw."""
    return ((draws(k, idx) >> np.uint64(11)).astype(np.float64) + 0.5) / float(1 << 53)


# ---------------------------------------------------------------------------
# symbol tables
# ---------------------------------------------------------------------------

def _quantise(probs: np.ndarray, total: int) -> np.ndarray:
    """Integer counts per row summing to ``total`` (largest-remainder rounding,
    ties broken by symbol order)."""
    probs = np.asarray(probs, dtype=np.float64)
    probs = probs / probs.sum(axis=1, keepdims=True)
    raw = probs * total
    base = np.floor(raw).astype(np.int64)
    short = total - base.sum(axis=1)
    order = np.argsort(-(raw - base), axis=1, kind="stable")
    ranks = np.empty_like(order)
    np.put_along_axis(ranks, order, np.broadcast_to(np.arange(probs.shape[1]), probs.shape).copy(),
                      axis=1)
    return base + (ranks < short[:, None]).astype(np.int64)


def _table_from_counts(symbols: bytes, counts: np.ndarray, size: int) -> np.ndarray:
    t = np.repeat(np.frombuffer(symbols, dtype=np.uint8), counts)
    assert t.size == size
    return t


def uniform_table(alphabet: bytes) -> np.ndarray:
    """65536-entry table: entry u maps to alphabet[(u * sigma) >> 16]."""
    u = np.arange(65536, dtype=np.uint64)
    a = np.frombuffer(alphabet, dtype=np.uint8)
    return a[(u * np.uint64(len(alphabet))) >> np.uint64(16)].copy()


def nl64_probs(seed: int):
    """Symbols and probabilities of the 64-symbol natural-language-like alphabet."""
    k = key(seed, STREAM_TABLE)
    perm = list(NL63)
    for i in range(len(perm) - 1, 0, -1):   # seeded Fisher-Yates: rank -> symbol
        j = draw(k, i) % (i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    ranks = np.arange(1, 64, dtype=np.float64)
    w = ranks ** -1.1
    probs = np.concatenate([[0.15], 0.85 * w / w.sum()])
    return bytes([0x20]) + bytes(perm), probs


def nl64_table(seed: int) -> np.ndarray:
    syms, probs = nl64_probs(seed)
    counts = _quantise(probs[None, :], 65536)[0]
    return _table_from_counts(syms, counts, 65536)


@dataclass
class MarkovTables:
    start: np.ndarray      # 65536-entry start-symbol table (uniform over 96)
    rows: np.ndarray       # [96*96*1024] next-symbol tables per context
    sym_index: np.ndarray  # 256-entry byte -> symbol index


def markov_tables(seed: int) -> MarkovTables:
    k = key(seed, STREAM_TABLE)
    nsym = len(MARKOV96)
    u = uniform01(k, np.arange(nsym * nsym * nsym, dtype=np.uint64)).reshape(nsym * nsym, nsym)
    weights = -np.log(u)                       # exponential variates
    counts = _quantise(weights, 1024)
    syms = np.frombuffer(MARKOV96, dtype=np.uint8)
    rows = np.repeat(np.tile(syms, nsym * nsym), counts.reshape(-1)).astype(np.uint8)
    assert rows.size == nsym * nsym * 1024
    sym_index = np.zeros(256, dtype=np.uint8)
    sym_index[syms] = np.arange(nsym, dtype=np.uint8)
    return MarkovTables(uniform_table(MARKOV96), rows, sym_index)


# ---------------------------------------------------------------------------
# text specifications
# ---------------------------------------------------------------------------

KINDS = ("dna", "protein", "nl64", "markov96", "dna_runs", "bytes256", "binary")


@dataclass(frozen=True)
class TextSpec:
    kind: str
    seed: int = 0

    def __post_init__(self):
        if self.kind not in KINDS:
            raise ValueError(f"unknown text kind {self.kind!r}")

    @property
    def sigma(self) -> int:
        return {"dna": 4, "protein": 20, "nl64": 64, "markov96": 96, "dna_runs": 4,
                "bytes256": 256, "binary": 2}[self.kind]

    def symbol_table(self) -> np.ndarray:
        """65536-entry table of the i.i.d. symbol distribution (also used for
        random patterns)."""
        if self.kind in ("dna", "dna_runs"):
            return uniform_table(DNA)
        if self.kind == "protein":
            return uniform_table(PROTEIN)
        if self.kind == "nl64":
            return nl64_table(self.seed)
        if self.kind == "bytes256":
            return uniform_table(bytes(range(256)))
        if self.kind == "binary":
            return uniform_table(b"\x00\xff")
        return uniform_table(MARKOV96)

    # -- host ---------------------------------------------------------------
    def host(self, n: int, start: int = 0, out: np.ndarray | None = None) -> np.ndarray:
        """Bytes [start, start+n) of the text, made on the host (into ``out``,
        a contiguous uint8 array of n bytes, when given)."""
        lib = _host_lib()
        if out is None:
            out = np.empty(n, dtype=np.uint8)
        assert out.size == n and out.dtype == np.uint8 and out.flags["C_CONTIGUOUS"]
        if n == 0:
            return out
        k = key(self.seed, STREAM_TEXT)
        if self.kind == "markov96":
            mt = _markov_cached(self.seed)
            lib.gen_fill_markov(out.ctypes.data, start, n, k, mt.start.ctypes.data,
                                mt.rows.ctypes.data, mt.sym_index.ctypes.data)
        else:
            tab = _table_cached(self)
            lib.gen_fill_iid(out.ctypes.data, start, n, k, tab.ctypes.data)
            if self.kind == "dna_runs":
                lib.gen_apply_runs(out.ctypes.data, start, n, key(self.seed, STREAM_RUNS),
                                   RUN_BLOCK, RUN_MAXLEN, ord("A"))
        return out

    def host_parallel(self, n: int, start: int = 0, threads: int | None = None,
                      piece: int = 16 << 20) -> np.ndarray:
        """``host`` made by several threads, each filling pieces of ``piece``
        bytes (the byte streams are counter-based, so any range can be made
        on its own; the C generator runs without the interpreter lock)."""
        from concurrent.futures import ThreadPoolExecutor
        out = np.empty(n, dtype=np.uint8)
        if n == 0:
            return out
        if self.kind == "markov96":
            _markov_cached(self.seed)   # build the tables once, before the threads
        else:
            _table_cached(self)

        def work(a):
            b = min(n, a + piece)
            self.host(b - a, start=start + a, out=out[a:b])

        with ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 1) as ex:
            list(ex.map(work, range(0, n, piece)))
        return out

    # -- device -------------------------------------------------------------
    def device(self, n: int, dst_ptr: int, stream_ptr: int = 0, start: int = 0) -> None:
        """Write bytes [start, start+n) of the text to device memory at dst_ptr."""
        import torch
        lib = _cuda_lib()
        if n == 0:
            return
        k = key(self.seed, STREAM_TEXT)
        dev = torch.device("cuda")
        if self.kind == "markov96":
            mt = _markov_cached(self.seed)
            tabs = _device_cached(("markov", self.seed),
                                  lambda: [torch.from_numpy(a).to(dev) for a in
                                           (mt.start, mt.rows, mt.sym_index)])
            rc = lib.gen_fill_markov_device(dst_ptr, start, n, k, tabs[0].data_ptr(),
                                            tabs[1].data_ptr(), tabs[2].data_ptr(), stream_ptr)
        else:
            tab = _device_cached((self.kind, self.seed),
                                 lambda: [torch.from_numpy(_table_cached(self)).to(dev)])
            rc = lib.gen_fill_iid_device(dst_ptr, start, n, k, tab[0].data_ptr(), stream_ptr)
            if rc == 0 and self.kind == "dna_runs":
                rc = lib.gen_apply_runs_device(dst_ptr, start, n, key(self.seed, STREAM_RUNS),
                                               RUN_BLOCK, RUN_MAXLEN, ord("A"), stream_ptr)
        if rc != 0:
            raise RuntimeError(f"device text generation failed (cuda error {rc})")

    def device_tensor(self, n: int, pad: int = 0):
        """A fresh uint8 CUDA tensor holding the text (plus ``pad`` zero bytes)."""
        import torch
        t = torch.zeros(n + pad, dtype=torch.uint8, device="cuda")
        self.device(n, t.data_ptr(), torch.cuda.current_stream().cuda_stream)
        return t[:n] if pad == 0 else t


_tables = {}
_markovs = {}
_devtabs = {}


def _table_cached(spec: TextSpec) -> np.ndarray:
    k = (spec.kind, spec.seed)
    if k not in _tables:
        _tables[k] = np.ascontiguousarray(spec.symbol_table())
    return _tables[k]


def _markov_cached(seed: int) -> MarkovTables:
    if seed not in _markovs:
        _markovs[seed] = markov_tables(seed)
    return _markovs[seed]


def _device_cached(k, make):
    if k not in _devtabs:
        _devtabs[k] = make()
    return _devtabs[k]


# ---------------------------------------------------------------------------
# patterns
# ---------------------------------------------------------------------------

def planted_offsets(spec: TextSpec, n: int, m: int, count: int, stream_seed: int = 0) -> list:
    k = key(spec.seed * 1000003 + m * 7919 + stream_seed, STREAM_PAT_OFFSET)
    span = n - m + 1
    return [draw(k, i) % span for i in range(count)] if span > 0 else []


def planted_patterns(spec: TextSpec, n: int, m: int, count: int, stream_seed: int = 0) -> list:
    """Patterns copied from uniformly random offsets of the text."""
    return [bytes(spec.host(m, start=o)) for o in planted_offsets(spec, n, m, count, stream_seed)]


def random_patterns(spec: TextSpec, m: int, count: int, stream_seed: int = 0) -> list:
    """Patterns drawn i.i.d. from the text's symbol distribution."""
    tab = _table_cached(spec)
    k = key(spec.seed * 1000003 + m * 7919 + stream_seed, STREAM_PAT_RANDOM)
    out = []
    for i in range(count):
        idx = np.arange(i * m, (i + 1) * m, dtype=np.uint64)
        u = (draws(k, idx) & np.uint64(0xFFFF)).astype(np.int64)
        out.append(bytes(tab[u]))
    return out


def mixed_patterns(spec: TextSpec, n: int, m: int, count: int, stream_seed: int = 0) -> list:
    """Half planted, half i.i.d. (planted first), as in the pattern-length sweep."""
    half = count // 2
    return (planted_patterns(spec, n, m, count - half, stream_seed)
            + random_patterns(spec, m, half, stream_seed))


# ---------------------------------------------------------------------------
# batched-workload pair table (uneven n and m)
# ---------------------------------------------------------------------------

@dataclass
class Pair:
    spec: TextSpec
    n: int
    pattern: bytes


def batch_pairs(npairs: int, seed: int = 0, n_lo_log2: int = 10, n_hi_log2: int = 25,
                m_lo: int = 1, m_hi: int = 32) -> list:
    """(text, pattern) pairs: n log-uniform in [2^lo, 2^hi], alphabet uniform over
    {dna, protein, nl64}, m uniform in [m_lo, m_hi], half planted / half i.i.d."""
    k = key(seed, STREAM_BATCH)
    kinds = ("dna", "protein", "nl64")
    pairs = []
    for i in range(npairs):
        d0, d1, d2 = draw(k, 4 * i), draw(k, 4 * i + 1), draw(k, 4 * i + 2)
        u = ((d0 >> 11) + 0.5) / float(1 << 53)
        n = int(round(2.0 ** (n_lo_log2 + (n_hi_log2 - n_lo_log2) * u)))
        spec = TextSpec(kinds[d1 % 3], seed=seed * 100003 + i)
        m = m_lo + int(d2 % (m_hi - m_lo + 1))
        if (d2 >> 32) & 1 and n >= m:
            pat = planted_patterns(spec, n, m, 1)[0]
        else:
            pat = random_patterns(spec, m, 1)[0]
        pairs.append(Pair(spec, n, pat))
    return pairs
