"""ctypes binding of the C ABI declared in include/epsm.h (argument marshalling
only; every step of the search runs in the CUDA kernels of libepsm.so)."""
from __future__ import annotations

import ctypes
import os

import os as _os

_LIB = _os.path.join(_os.path.dirname(_os.path.abspath(__file__)), "lib", "libepsm.so")

_lib = None

OK, ERR_ARG, ERR_CAPACITY, ERR_CUDA, ERR_NOMEM, ERR_TIMEOUT = range(6)
STATUS_NAMES = ["EPSM_OK", "EPSM_ERR_ARG", "EPSM_ERR_CAPACITY", "EPSM_ERR_CUDA",
                "EPSM_ERR_NOMEM", "EPSM_ERR_TIMEOUT"]
(VARIANT_AUTO, VARIANT_DIRECT, VARIANT_PREFIX4, VARIANT_PREFIX8, VARIANT_BLOCK8, VARIANT_BLOCK4, VARIANT_CODE2,
 VARIANT_ADAPT, VARIANT_BLOCK8S) = range(9)
VARIANT_NAMES = {1: "direct", 2: "prefix4", 3: "prefix8", 4: "block8", 5: "block4", 6: "code2", 7: "adapt", 8: "block8s"}
MAX_M = 32
MAX_M_LONG = 4096  # single-search entry points only

EXPORTS = ["epsm_create", "epsm_destroy", "epsm_status_str", "epsm_last_error",
           "epsm_search", "epsm_search_async", "epsm_search_variant", "epsm_sync",
           "epsm_search_batch", "epsm_search_host", "epsm_variant_for", "epsm_set_variant",
           "epsm_launch_count", "epsm_search_static", "epsm_batch_uses_graph",
           "epsm_set_tuning", "epsm_get_tuning",
           "epsm_server_create", "epsm_server_destroy", "epsm_server_add_corpus",
           "epsm_server_upload", "epsm_server_submit", "epsm_server_poll", "epsm_server_read",
           "epsm_server_release", "epsm_server_replay", "epsm_server_stats_get",
           "epsm_server_inject_fault"]
STATIC_MAX_TEXT = 64 << 20
TEXT_BUCKETS = 3
BUCKET_MIN = (0, 16 << 20, 512 << 20)   # first text length of each tuning-table bucket
KBITS_MIN, KBITS_MAX = 8, 14
SHAPES = 2


def text_bucket(n: int) -> int:
    """Bucket of the tuning table a text of n bytes falls in."""
    return 0 if n < BUCKET_MIN[1] else (1 if n < BUCKET_MIN[2] else 2)


def lib_path() -> str:
    return _LIB


def load(path: str | None = None):
    """Load libepsm.so.  Raises ImportError when it has not been built: there is
    no fallback implementation."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _LIB
    if not os.path.exists(p):
        raise ImportError(f"libepsm.so is not built ({p}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(p)
    vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    st = ctypes.c_int
    lib.epsm_create.argtypes = [ctypes.POINTER(vp), i32, u64]
    lib.epsm_create.restype = st
    lib.epsm_destroy.argtypes = [vp]
    lib.epsm_destroy.restype = st
    lib.epsm_status_str.argtypes = [st]
    lib.epsm_status_str.restype = ctypes.c_char_p
    lib.epsm_last_error.argtypes = [vp]
    lib.epsm_last_error.restype = ctypes.c_char_p
    lib.epsm_search.argtypes = [vp, vp, u64, vp, u32, vp, u64, ctypes.POINTER(u64), vp]
    lib.epsm_search.restype = st
    lib.epsm_search_async.argtypes = [vp, vp, u64, vp, u32, vp, u64, vp, vp]
    lib.epsm_search_async.restype = st
    lib.epsm_search_variant.argtypes = [vp, i32, vp, u64, vp, u32, vp, u64, vp, vp]
    lib.epsm_search_variant.restype = st
    lib.epsm_sync.argtypes = [vp, vp]
    lib.epsm_wait_probe.argtypes = [vp, u64, vp]
    lib.epsm_wait_probe.restype = st
    lib.epsm_sync.restype = st
    lib.epsm_search_batch.argtypes = [vp, u32, vp, vp, vp, vp, vp, u64, vp, vp]
    lib.epsm_search_batch.restype = st
    lib.epsm_search_host.argtypes = [vp, vp, u64, vp, vp, u32, vp, u64, vp]
    lib.epsm_search_host.restype = st
    lib.epsm_variant_for.argtypes = [vp, u32]
    lib.epsm_variant_for.restype = i32
    lib.epsm_set_variant.argtypes = [vp, u32, i32]
    lib.epsm_set_variant.restype = st
    lib.epsm_set_tuning.argtypes = [vp, i32, u32, i32, i32, u32]
    lib.epsm_set_tuning.restype = st
    lib.epsm_get_tuning.argtypes = [vp, i32, u32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                    ctypes.POINTER(u32)]
    lib.epsm_get_tuning.restype = st
    lib.epsm_launch_count.argtypes = [vp]
    lib.epsm_launch_count.restype = u64
    lib.epsm_batch_uses_graph.argtypes = [vp]
    lib.epsm_batch_uses_graph.restype = i32
    lib.epsm_search_static.argtypes = [vp, u64, vp, u32, vp, u64, vp, vp]
    lib.epsm_search_static.restype = st
    i64 = ctypes.c_int64
    lib.epsm_server_create.argtypes = [ctypes.POINTER(vp), i32, vp]
    lib.epsm_server_create.restype = st
    lib.epsm_server_destroy.argtypes = [vp]
    lib.epsm_server_destroy.restype = st
    lib.epsm_server_add_corpus.argtypes = [vp, vp, u64, ctypes.POINTER(u32)]
    lib.epsm_server_add_corpus.restype = st
    lib.epsm_server_upload.argtypes = [vp, vp, u64, ctypes.POINTER(u64)]
    lib.epsm_server_upload.restype = st
    lib.epsm_server_submit.argtypes = [vp, u32, vp, u32, ctypes.POINTER(u64)]
    lib.epsm_server_submit.restype = st
    lib.epsm_server_poll.argtypes = [vp, vp, u32, i64]
    lib.epsm_server_poll.restype = u32
    lib.epsm_server_read.argtypes = [vp, u64, vp, u64]
    lib.epsm_server_read.restype = st
    lib.epsm_server_release.argtypes = [vp, u64]
    lib.epsm_server_release.restype = st
    lib.epsm_server_replay.argtypes = [vp, u32, vp, vp, vp, vp, vp]
    lib.epsm_server_replay.restype = st
    lib.epsm_server_stats_get.argtypes = [vp, vp]
    lib.epsm_server_stats_get.restype = st
    lib.epsm_server_inject_fault.argtypes = [vp, i32, u32]
    lib.epsm_server_inject_fault.restype = st
    if path is None:
        _lib = lib
    return lib
