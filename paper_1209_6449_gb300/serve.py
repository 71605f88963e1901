"""Python binding of the serving engine declared in include/epsm_serve.h
(argument marshalling only: batching, admission and the searches run in the
native engine and its CUDA kernels)."""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np

from . import _native

_lib = _native.load()


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_uint32), ("inflight", ctypes.c_uint32),
                ("per_query", ctypes.c_uint32), ("small_batch", ctypes.c_uint32),
                ("upload_budget", ctypes.c_uint64), ("reserve", ctypes.c_uint64),
                ("out_capacity", ctypes.c_uint64)]


class Result(ctypes.Structure):
    _fields_ = [("request", ctypes.c_uint64), ("status", ctypes.c_int32), ("corpus", ctypes.c_uint32),
                ("count", ctypes.c_uint64), ("positions", ctypes.c_void_p),
                ("submit_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in
                ("batches", "queries", "uploads", "evictions", "reruns", "max_batch_seen")]


# epsm_replay_item: int64 at_ns, uint32 kind, uint32 corpus, pointer data, uint64 len
REPLAY_DTYPE = np.dtype([("at_ns", "<i8"), ("kind", "<u4"), ("corpus", "<u4"),
                         ("data", "<u8"), ("len", "<u8")])


class ServerError(RuntimeError):
    def __init__(self, status: int, where: str):
        name = _native.STATUS_NAMES[status] if 0 <= status < len(_native.STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}")
        self.status = status


def _check(st: int, where: str):
    if st != 0:
        raise ServerError(st, where)


class Server:
    """A serving engine on one CUDA device: resident corpora, queries batched
    as they arrive, uploads admitted by device memory."""

    def __init__(self, device: int = 0, max_batch: int = 1024, inflight: int = 2,
                 per_query: bool = False, upload_budget: int = 0, reserve: int = 0,
                 out_capacity: int = 0, small_batch: int = 0):
        cfg = ServerConfig(max_batch, inflight, 1 if per_query else 0, small_batch, upload_budget,
                           reserve, out_capacity)
        h = ctypes.c_void_p()
        _check(_lib.epsm_server_create(ctypes.byref(h), device, ctypes.byref(cfg)), "epsm_server_create")
        self.handle = h
        self._keep = []     # device tensors of registered corpora
        self._uploads = {}  # request -> host array kept alive until the upload completes

    def close(self):
        if self.handle:
            _lib.epsm_server_destroy(self.handle)
            self.handle = None
            self._keep = []
            self._uploads = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_corpus(self, text) -> int:
        """Registers a resident corpus: a uint8 CUDA tensor, or (device pointer, n)."""
        if isinstance(text, tuple):
            ptr, n = text
        else:
            self._keep.append(text)
            ptr, n = text.data_ptr(), text.numel()
        cid = ctypes.c_uint32()
        _check(_lib.epsm_server_add_corpus(self.handle, ptr, n, ctypes.byref(cid)), "epsm_server_add_corpus")
        return cid.value

    def upload(self, host: np.ndarray) -> int:
        """Uploads a host text (uint8 array) as a new corpus; returns the request id."""
        host = np.ascontiguousarray(host, dtype=np.uint8)
        rid = ctypes.c_uint64()
        _check(_lib.epsm_server_upload(self.handle, host.ctypes.data, host.size, ctypes.byref(rid)),
               "epsm_server_upload")
        self._uploads[rid.value] = host
        return rid.value

    def submit(self, corpus: int, pattern: bytes) -> int:
        rid = ctypes.c_uint64()
        _check(_lib.epsm_server_submit(self.handle, corpus, pattern, len(pattern), ctypes.byref(rid)),
               "epsm_server_submit")
        return rid.value

    def poll(self, max_results: int = 256, timeout_s: float = 0.0) -> list:
        buf = (Result * max_results)()
        k = _lib.epsm_server_poll(self.handle, buf, max_results, int(timeout_s * 1e9))
        out = []
        for i in range(k):
            r = buf[i]
            self._uploads.pop(r.request, None)
            out.append({"request": r.request, "status": r.status, "corpus": r.corpus, "count": r.count,
                        "positions": r.positions, "submit_ns": r.submit_ns, "done_ns": r.done_ns})
        return out

    def read(self, request: int, count: int) -> np.ndarray:
        """The positions of a completed, unreleased query (copied to the host)."""
        out = np.empty(count, dtype=np.uint64)
        _check(_lib.epsm_server_read(self.handle, request, out.ctypes.data, count), "epsm_server_read")
        return out

    def release(self, request: int):
        _check(_lib.epsm_server_release(self.handle, request), "epsm_server_release")

    FAULT_ALLOC, FAULT_ADMIT, FAULT_UPLOAD = 0, 1, 2

    def inject_fault(self, kind: int, count: int = 1):
        """Arms `count` host-side failures of one kind (see epsm_server_inject_fault)."""
        _check(_lib.epsm_server_inject_fault(self.handle, kind, count), "epsm_server_inject_fault")

    def stats(self) -> dict:
        s = Stats()
        _check(_lib.epsm_server_stats_get(self.handle, ctypes.byref(s)), "epsm_server_stats_get")
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def replay(self, at_ns: np.ndarray, kinds: np.ndarray, corpora: np.ndarray,
               payloads: Sequence) -> dict:
        """Replays a request stream at the given arrival offsets: payloads[i] is
        a pattern (bytes) for a query, a host uint8 array for an upload."""
        n = len(payloads)
        items = np.zeros(n, dtype=REPLAY_DTYPE)
        items["at_ns"] = at_ns
        items["kind"] = kinds
        items["corpus"] = corpora
        keep = []
        pats = [p for p, k in zip(payloads, kinds) if k == 0]
        blob = np.frombuffer(b"".join(pats) or b"\0", dtype=np.uint8)
        keep.append(blob)
        off = 0
        base = blob.ctypes.data
        for i, (p, k) in enumerate(zip(payloads, kinds)):
            if k == 0:
                items["data"][i] = base + off
                items["len"][i] = len(p)
                off += len(p)
            else:
                a = np.ascontiguousarray(p, dtype=np.uint8)
                keep.append(a)
                items["data"][i] = a.ctypes.data
                items["len"][i] = a.size
        lat = np.zeros(n, dtype=np.int64)
        cnt = np.zeros(n, dtype=np.uint64)
        st = np.zeros(n, dtype=np.int32)
        el = ctypes.c_int64()
        _check(_lib.epsm_server_replay(self.handle, n, items.ctypes.data, lat.ctypes.data, cnt.ctypes.data,
                                       st.ctypes.data, ctypes.byref(el)), "epsm_server_replay")
        del keep
        return {"latency_ns": lat, "counts": cnt, "status": st, "elapsed_s": el.value / 1e9}
