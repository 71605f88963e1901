"""Pins for the oracle: checks against facts the paper and mathematics fix.

Each check takes a ``search(text: bytes, pattern: bytes) -> list[int]`` callable
so that the same checks can be run against a deliberately broken copy of the
oracle (tests/test_oracle_mutants.py) and shown to fail there.
"""
from __future__ import annotations

import itertools
import re


def lib_positions(text: bytes, pattern: bytes) -> list:
    """All (overlapping) occurrences via the regex engine's lookahead search."""
    return [mt.start() for mt in re.finditer(b"(?=" + re.escape(pattern) + b")", text)]


def check_closed_form_runs(search) -> None:
    """a^m in a^n has exactly the n-m+1 starts 0..n-m (all occurrences, Section 1)."""
    for byte in (b"a", b"\x00", b"\xff"):
        for n in range(0, 41):
            for m in range(1, 34):
                got = list(search(byte * n, byte * m))
                want = list(range(n - m + 1)) if m <= n else []
                assert got == want, (byte, n, m, got[:5])


def check_periodic(search) -> None:
    """(ab)^k: (ab)^j occurs at the even starts, (ba)^j at the odd ones."""
    for k in range(1, 20):
        t = b"ab" * k
        for j in range(1, k + 1):
            assert list(search(t, b"ab" * j)) == list(range(0, 2 * (k - j) + 1, 2))
            want = list(range(1, 2 * (k - j), 2)) if j < k else []
            assert list(search(t, b"ba" * j)) == want
        assert list(search(t, b"aa")) == []


def check_exhaustive_binary(search, nmax: int = 10, mmax: int = 4) -> None:
    """Every text of length <= nmax and pattern of length <= mmax over {0,1}.

    Two facts pin it: per text the positions equal the regex engine's; and for
    each fixed pattern of length m, the hit count summed over all 2^n texts is
    (n - m + 1) * 2^(n - m) (each start matches in exactly 2^(n-m) texts).
    """
    sym = (b"\x00", b"\x01")
    for n in range(0, nmax + 1):
        texts = [b"".join(c) for c in itertools.product(sym, repeat=n)]
        for m in range(1, mmax + 1):
            for pc in itertools.product(sym, repeat=m):
                p = b"".join(pc)
                total = 0
                for t in texts:
                    got = list(search(t, p))
                    assert got == lib_positions(t, p), (t, p, got)
                    total += len(got)
                want = (n - m + 1) * 2 ** (n - m) if m <= n else 0
                assert total == want, (n, p, total, want)


def check_planted(search, text: bytes, pattern: bytes, offsets) -> None:
    """A pattern over symbols absent from the text occurs exactly where planted."""
    t = bytearray(text)
    for o in offsets:
        t[o:o + len(pattern)] = pattern
    assert list(search(bytes(t), pattern)) == sorted(offsets)


def check_edges(search) -> None:
    assert list(search(b"", b"a")) == []
    assert list(search(b"abc", b"abcd")) == []
    assert list(search(b"abcd", b"abcd")) == [0]
    assert list(search(b"xabcd", b"abcd")) == [1]
    assert list(search(b"abcdx", b"abcd")) == [0]
    # unsigned bytes: 0x80..0xFF must match exactly and only themselves
    t = bytes(range(256)) * 2
    for b in (0x7F, 0x80, 0xFE, 0xFF):
        assert list(search(t, bytes([b]))) == [b, 256 + b]
        assert list(search(t, bytes([b, (b + 1) & 0xFF]))) == ([b, 256 + b] if b < 255 else [255])
