"""CPU oracle for exact short-pattern string matching — TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline
and reference legs) may import this package.  The GPU library never imports,
links or executes anything here, and nothing here imports the GPU library.

The oracle computes the plain definition of the exact string matching problem
(Section 1; notation of Section 2): every start position ``s`` with
``0 <= s <= n - m`` and ``t[s + i] == p[i]`` for all ``i < m``, ascending,
overlaps included, bytes compared unsigned.  The brute-force scan lives in
``epsm_oracle.c`` (plain C, built with gcc); ``paper.py`` restates the paper's
packed-word primitives and its three procedures for small cross-checks.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "epsm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/liboracle.so`` with gcc."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u8p = ctypes.c_void_p
            lib.oracle_search.argtypes = [u8p, ctypes.c_uint64, u8p, ctypes.c_uint32,
                                          ctypes.c_void_p, ctypes.c_uint64]
            lib.oracle_search.restype = ctypes.c_uint64
            lib.oracle_search_mt.argtypes = [u8p, ctypes.c_uint64, u8p, ctypes.c_uint32,
                                             ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int]
            lib.oracle_search_mt.restype = ctypes.c_uint64
            lib.oracle_count.argtypes = [u8p, ctypes.c_uint64, u8p, ctypes.c_uint32]
            lib.oracle_count.restype = ctypes.c_uint64
            lib.oracle_kmp_count.argtypes = [u8p, ctypes.c_uint64, u8p, ctypes.c_uint32]
            lib.oracle_kmp_count.restype = ctypes.c_uint64
            _lib = lib
    return _lib


def _as_u8(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(x), dtype=np.uint8)
    a = np.ascontiguousarray(x)
    if a.dtype != np.uint8:
        raise TypeError("oracle inputs must be bytes or uint8 arrays")
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data if a.size else None


def search(text, pattern, threads: int = 1) -> np.ndarray:
    """All occurrence start positions of ``pattern`` in ``text`` (uint64, ascending)."""
    lib = _load()
    t = _as_u8(text)
    p = _as_u8(pattern)
    n, m = int(t.size), int(p.size)
    if m == 0 or m > n:
        return np.zeros(0, dtype=np.uint64)
    if threads > 1:
        cnt = lib.oracle_search_mt(_ptr(t), n, _ptr(p), m, None, 0, threads)
    else:
        cnt = lib.oracle_count(_ptr(t), n, _ptr(p), m)
    out = np.empty(int(cnt), dtype=np.uint64)
    if cnt:
        if threads > 1:
            got = lib.oracle_search_mt(_ptr(t), n, _ptr(p), m, _ptr(out), int(cnt), threads)
        else:
            got = lib.oracle_search(_ptr(t), n, _ptr(p), m, _ptr(out), int(cnt))
        assert got == cnt
    return out


def count(text, pattern, threads: int = 1) -> int:
    lib = _load()
    t = _as_u8(text)
    p = _as_u8(pattern)
    n, m = int(t.size), int(p.size)
    if m == 0 or m > n:
        return 0
    if threads > 1:
        return int(lib.oracle_search_mt(_ptr(t), n, _ptr(p), m, None, 0, threads))
    return int(lib.oracle_count(_ptr(t), n, _ptr(p), m))


def kmp_count(text, pattern) -> int:
    """Occurrence count by the Knuth-Morris-Pratt automaton (independent algorithm)."""
    lib = _load()
    t = _as_u8(text)
    p = _as_u8(pattern)
    n, m = int(t.size), int(p.size)
    if m == 0 or m > n:
        return 0
    return int(lib.oracle_kmp_count(_ptr(t), n, _ptr(p), m))
