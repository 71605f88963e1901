"""The oracle's pins catch plausible mistakes: each test plants one mistake in a
temporary copy of the C oracle (on the CPU), builds it, and requires at least
one pin of tests/_pins.py to fail against it."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from tests import _pins

SRC = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "epsm_oracle.c")

MUTANTS = {
    # the last valid start n-m is dropped
    "drops_last_start": ("return scan_range(t, n, p, m, 0, n - m + 1, out, cap);",
                         "return scan_range(t, n, p, m, 0, n - m, out, cap);"),
    # the last pattern byte is never compared
    "drops_last_byte": ("while (i < m && t[s + i] == p[i]) ++i;\n        if (i == m) {",
                        "while (i + 1 < m && t[s + i] == p[i]) ++i;\n        if (i + 1 >= m) {"),
    # text index shifted by one
    "shifted_index": ("t[s + i] == p[i]", "t[s + i + 1 - (s + i + 1 >= n)] == p[i]"),
    # overlapping occurrences skipped
    "no_overlaps": ("if (count < cap) out[count] = s;\n            ++count;",
                    "if (count < cap) out[count] = s;\n            ++count; s += m - 1;"),
    # first start skipped
    "skips_zero": ("for (uint64_t s = s_begin; s < s_end; ++s) {",
                   "for (uint64_t s = s_begin + (s_begin == 0); s < s_end; ++s) {"),
}


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, name
    mut = src.replace(old, new, 1)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(mut)
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-pthread", "-o", str(so), str(c)])
    lib = ctypes.CDLL(str(so))
    lib.oracle_search.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                  ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint64]
    lib.oracle_search.restype = ctypes.c_uint64

    def search(t, p):
        tb = np.frombuffer(t + b"\0", dtype=np.uint8)
        pb = np.frombuffer(p, dtype=np.uint8)
        n, m = len(t), len(p)
        cnt = lib.oracle_search(tb.ctypes.data, n, pb.ctypes.data, m, None, 0)
        out = np.zeros(max(int(cnt), 1), dtype=np.uint64)
        lib.oracle_search(tb.ctypes.data, n, pb.ctypes.data, m, out.ctypes.data, int(cnt))
        return [int(x) for x in out[:cnt]]
    return search


CHECKS = [_pins.check_closed_form_runs, _pins.check_periodic, _pins.check_edges,
          lambda s: _pins.check_exhaustive_binary(s, nmax=7, mmax=3)]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    search = _build(tmp_path, name, *MUTANTS[name])
    failures = 0
    for chk in CHECKS:
        try:
            chk(search)
        except AssertionError:
            failures += 1
    assert failures >= 1, f"no pin caught mutant {name}"


def test_unmutated_copy_passes(tmp_path):
    search = _build(tmp_path, "identity", "#include <stdint.h>", "#include <stdint.h>")
    for chk in CHECKS:
        chk(search)
