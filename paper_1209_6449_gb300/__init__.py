"""GB300 exact short-pattern matching (Faro & Kulekci, "Fast Packed String
Matching for Short Patterns").

Python binding of the C ABI in ``include/epsm.h``.  The functions named
``epsm_*`` mirror the C entry points one to one (argument marshalling only);
``Context`` wraps them for torch tensors.  Every step of a search runs in the
sm_103a kernels of ``lib/libepsm.so``; importing this package without the
built library raises ImportError (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np

from . import _native
from ._native import (MAX_M, MAX_M_LONG, STATIC_MAX_TEXT, STATUS_NAMES, VARIANT_AUTO, VARIANT_BLOCK4, VARIANT_BLOCK8,
                      VARIANT_ADAPT, VARIANT_BLOCK8S, VARIANT_CODE2, VARIANT_DIRECT, VARIANT_NAMES,
                      VARIANT_PREFIX4, VARIANT_PREFIX8)

__all__ = ["Context", "EpsmError", "Server", "epsm_create", "epsm_destroy", "epsm_status_str",
           "epsm_search", "epsm_search_async", "epsm_search_variant", "epsm_sync",
           "epsm_search_batch", "epsm_search_host", "epsm_variant_for", "epsm_set_variant",
           "epsm_launch_count", "epsm_search_static", "epsm_set_tuning", "epsm_get_tuning", "epsm_wait_probe", "STATIC_MAX_TEXT", "MAX_M", "MAX_M_LONG", "VARIANT_AUTO", "VARIANT_DIRECT", "VARIANT_PREFIX4",
           "VARIANT_PREFIX8", "VARIANT_BLOCK8", "VARIANT_BLOCK4", "VARIANT_CODE2", "VARIANT_ADAPT", "VARIANT_BLOCK8S",
           "VARIANT_NAMES"]

_lib = _native.load()

from .serve import Server  # noqa: E402  (needs the loaded library)


class EpsmError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}{' (' + detail + ')' if detail else ''}")


def _buf(b: bytes):
    return ctypes.c_char_p(b)


# ---------------------------------------------------------------------------
# C-named entry points (same names and argument order as include/epsm.h;
# pointers are plain integers, patterns are bytes)
# ---------------------------------------------------------------------------

def epsm_create(device: int = 0, flags: int = 0) -> int:
    h = ctypes.c_void_p()
    st = _lib.epsm_create(ctypes.byref(h), device, flags)
    if st != 0:
        raise EpsmError(st, "epsm_create")
    return h.value


def epsm_destroy(ctx: int) -> int:
    return _lib.epsm_destroy(ctx)


def epsm_status_str(status: int) -> str:
    return _lib.epsm_status_str(status).decode()


def epsm_search(ctx: int, text: int, n: int, pattern: bytes, m: int, positions: int,
                capacity: int, stream: int = 0):
    """Returns (status, count)."""
    cnt = ctypes.c_uint64(0)
    st = _lib.epsm_search(ctx, text, n, _buf(pattern), m, positions, capacity,
                          ctypes.byref(cnt), stream)
    return st, cnt.value


def epsm_search_async(ctx: int, text: int, n: int, pattern: bytes, m: int, positions: int,
                      capacity: int, count_dev: int, stream: int = 0) -> int:
    return _lib.epsm_search_async(ctx, text, n, _buf(pattern), m, positions, capacity,
                                  count_dev, stream)


def epsm_search_variant(ctx: int, variant: int, text: int, n: int, pattern: bytes, m: int,
                        positions: int, capacity: int, count_dev: int, stream: int = 0) -> int:
    return _lib.epsm_search_variant(ctx, variant, text, n, _buf(pattern), m, positions,
                                    capacity, count_dev, stream)


def epsm_sync(ctx: int, stream: int = 0) -> int:
    return _lib.epsm_sync(ctx, stream)


def epsm_wait_probe(ctx: int, limit_ns: int, stream: int = 0) -> int:
    """Diagnostic of the bounded device waits (see include/epsm.h)."""
    return _lib.epsm_wait_probe(ctx, limit_ns, stream)


def _pattern_table(patterns: Sequence[bytes]):
    """One buffer holding all patterns and the array of their addresses."""
    blob = b"".join(patterns)
    buf = np.frombuffer(blob, dtype=np.uint8) if blob else np.zeros(1, dtype=np.uint8)
    ms = np.fromiter((len(p) for p in patterns), dtype=np.uint32, count=len(patterns))
    starts = np.zeros(len(patterns), dtype=np.uint64)
    if len(patterns) > 1:
        np.cumsum(ms[:-1], dtype=np.uint64, out=starts[1:])
    ptrs = starts + np.uint64(buf.ctypes.data)
    return buf, ptrs, ms


def epsm_search_batch(ctx: int, texts: Sequence[int], ns: Sequence[int],
                      patterns: Sequence[bytes], positions: int, capacity: int,
                      stream: int = 0):
    """Returns (status, offsets ndarray[npairs+1])."""
    npairs = len(patterns)
    t_arr = np.ascontiguousarray(texts, dtype=np.uint64)
    n_arr = np.ascontiguousarray(ns, dtype=np.uint64)
    keep, p_arr, m_arr = _pattern_table(patterns)
    offs = np.zeros(npairs + 1, dtype=np.uint64)
    st = _lib.epsm_search_batch(ctx, npairs, t_arr.ctypes.data, n_arr.ctypes.data, p_arr.ctypes.data,
                                m_arr.ctypes.data, positions, capacity, offs.ctypes.data, stream)
    del keep
    return st, offs


def epsm_search_host(ctx: int, text: np.ndarray, patterns: Sequence[bytes],
                     positions: np.ndarray):
    """Host buffers in, host buffers out.  Returns (status, offsets)."""
    text = np.ascontiguousarray(text, dtype=np.uint8)
    cat = b"".join(patterns)
    ms = np.ascontiguousarray([len(p) for p in patterns], dtype=np.uint32)
    offs = np.zeros(len(patterns) + 1, dtype=np.uint64)
    st = _lib.epsm_search_host(ctx, text.ctypes.data if text.size else None, text.size,
                               _buf(cat), ms.ctypes.data, len(patterns),
                               positions.ctypes.data if positions.size else None,
                               positions.size, offs.ctypes.data)
    return st, offs


def epsm_variant_for(ctx: int, m: int) -> int:
    return _lib.epsm_variant_for(ctx, m)


def epsm_set_variant(ctx: int, m: int, variant: int) -> int:
    return _lib.epsm_set_variant(ctx, m, variant)


def epsm_set_tuning(ctx: int, bucket: int, m: int, variant: int = 0, shape: int = -1,
                    kbits: int = 0) -> int:
    return _lib.epsm_set_tuning(ctx, bucket, m, variant, shape, kbits)


def epsm_get_tuning(ctx: int, bucket: int, m: int):
    """Returns (status, variant, shape, kbits)."""
    v, sh, kb = ctypes.c_int(), ctypes.c_int(), ctypes.c_uint32()
    st = _lib.epsm_get_tuning(ctx, bucket, m, ctypes.byref(v), ctypes.byref(sh), ctypes.byref(kb))
    return st, v.value, sh.value, kb.value


def epsm_launch_count(ctx: int) -> int:
    return _lib.epsm_launch_count(ctx)


def epsm_search_static(text: int, n: int, pattern: bytes, m: int, positions: int,
                       capacity: int, result_dev: int, stream: int = 0) -> int:
    """Search with no allocation: scratch is the library's fixed device array.
    ``result_dev`` points to two device uint64 (count, device error bits)."""
    return _lib.epsm_search_static(text, n, _buf(pattern), m, positions, capacity, result_dev,
                                   stream)


# ---------------------------------------------------------------------------
# torch-facing wrapper
# ---------------------------------------------------------------------------

class Context:
    """One library context on one CUDA device (not thread-safe)."""

    def __init__(self, device: int = 0, tuning: str | None = "default", text_class: str = "mixed"):
        """``tuning``: "default" installs the measured tuning table shipped
        next to this file (if present); a path installs that table; None keeps
        the library's built-in choice.  ``text_class`` picks the table's rows
        for an alphabet class ("dna", "protein", "text") or the rows best over
        all classes ("mixed")."""
        import torch
        self._torch = torch
        self.device = device
        self.handle = epsm_create(device)
        self._count = torch.zeros(1, dtype=torch.int64, device=f"cuda:{device}")
        if tuning is not None:
            from . import autotune
            table = autotune.load() if tuning == "default" else autotune.load(tuning)
            if table is not None:
                autotune.apply(self, table, text_class)

    def close(self):
        if self.handle:
            epsm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, where):
        if st != 0:
            detail = _lib.epsm_last_error(self.handle).decode()
            raise EpsmError(st, where, detail)

    @staticmethod
    def _stream(stream):
        import torch
        if stream is None:
            return torch.cuda.current_stream().cuda_stream
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)

    def search(self, text, pattern: bytes, capacity: int | None = None, stream=None,
               variant: int = VARIANT_AUTO):
        """All start positions of ``pattern`` in the uint8 CUDA tensor ``text``.

        Returns (count, positions) with positions an int64 CUDA tensor of the
        sorted starts (length == count).  If ``capacity`` is None a first guess
        is used and the search is repeated with the exact size on overflow."""
        torch = self._torch
        n = text.numel()
        m = len(pattern)
        cap = capacity if capacity is not None else max(1024, min(n, n // 64 + 4096))
        for _ in range(2):
            out = torch.empty(max(cap, 1), dtype=torch.int64, device=text.device)
            cnt = self.search_into(text, pattern, out, cap, stream=stream, variant=variant)
            if cnt <= cap or capacity is not None:
                return cnt, out[:min(cnt, cap)]
            cap = cnt
        return cnt, out[:cnt]

    def search_into(self, text, pattern: bytes, out, capacity: int, stream=None,
                    variant: int = VARIANT_AUTO) -> int:
        """Synchronous search into a preallocated int64/uint64 CUDA tensor."""
        s = self._stream(stream)
        n = text.numel()
        pos_ptr = out.data_ptr() if capacity else 0
        st = _lib.epsm_search_variant(self.handle, variant, text.data_ptr() if n else 0, n,
                                      _buf(pattern), len(pattern), pos_ptr, capacity,
                                      self._count.data_ptr(), s)
        self._check(st, "epsm_search_variant")
        st = _lib.epsm_sync(self.handle, s)
        if st not in (0, _native.ERR_CAPACITY):
            self._check(st, "epsm_sync")
        return int(self._count.item())

    def count(self, text, pattern: bytes, stream=None, variant: int = VARIANT_AUTO) -> int:
        return self.search_into(text, pattern, self._count, 0, stream=stream, variant=variant)

    def search_async(self, text, pattern: bytes, out, capacity: int, count_out, stream=None,
                     variant: int = VARIANT_AUTO) -> None:
        """Enqueue a search; the count lands in ``count_out`` (a CUDA tensor
        element) when the stream reaches it.  No host synchronisation."""
        s = self._stream(stream)
        n = text.numel()
        st = _lib.epsm_search_variant(self.handle, variant, text.data_ptr() if n else 0, n,
                                      _buf(pattern), len(pattern),
                                      out.data_ptr() if capacity else 0, capacity,
                                      count_out.data_ptr(), s)
        self._check(st, "epsm_search_variant")

    def sync(self, stream=None) -> int:
        return _lib.epsm_sync(self.handle, self._stream(stream))

    def search_batch(self, texts, patterns: Sequence[bytes], capacity: int, stream=None):
        """Batched search.  ``texts`` are uint8 CUDA tensors (or (ptr, n) tuples).
        Returns (offsets ndarray[npairs+1], positions int64 CUDA tensor)."""
        torch = self._torch
        ptrs = [t[0] if isinstance(t, tuple) else (t.data_ptr() if t.numel() else 0) for t in texts]
        ns = [t[1] if isinstance(t, tuple) else t.numel() for t in texts]
        out = torch.empty(max(capacity, 1), dtype=torch.int64, device=f"cuda:{self.device}")
        st, offs = epsm_search_batch(self.handle, ptrs, ns, patterns,
                                     out.data_ptr() if capacity else 0, capacity,
                                     self._stream(stream))
        if st not in (0, _native.ERR_CAPACITY):
            self._check(st, "epsm_search_batch")
        return offs, out

    def search_host(self, text: np.ndarray, patterns: Sequence[bytes], capacity: int):
        """End-to-end search from host memory.  Returns (offsets, positions ndarray)."""
        pos = np.zeros(capacity, dtype=np.uint64)
        st, offs = epsm_search_host(self.handle, text, patterns, pos)
        if st not in (0, _native.ERR_CAPACITY):
            self._check(st, "epsm_search_host")
        return offs, pos

    def set_tuning(self, bucket: int, m: int, variant: int = 0, shape: int = -1, kbits: int = 0):
        """One entry of the tuning table (bucket -1: every text-length bucket)."""
        self._check(epsm_set_tuning(self.handle, bucket, m, variant, shape, kbits), "epsm_set_tuning")

    def get_tuning(self, bucket: int, m: int):
        """(variant, shape, kbits) of one entry of the tuning table."""
        st, v, sh, kb = epsm_get_tuning(self.handle, bucket, m)
        self._check(st, "epsm_get_tuning")
        return v, sh, kb

    def variant_for(self, m: int) -> int:
        return epsm_variant_for(self.handle, m)

    def set_variant(self, m: int, variant: int) -> None:
        self._check(epsm_set_variant(self.handle, m, variant), "epsm_set_variant")

    @property
    def launch_count(self) -> int:
        return epsm_launch_count(self.handle)

    @property
    def batch_uses_graph(self) -> bool:
        return bool(_lib.epsm_batch_uses_graph(self.handle))
