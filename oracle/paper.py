"""The paper's packed-word model and its three search procedures, restated in
plain Python for small inputs — TEST INFRASTRUCTURE (part of the oracle).

Nothing here is fast or used by the GPU library.  It exists so that the readings
taken where the paper is garbled or silent can be checked: each procedure below
follows the steps of Section 3 in the paper's order and notation, and the tests
require it to produce exactly the plain-definition result of ``oracle.search``.

Words are tuples of ``alpha`` characters (character ``i`` of a word is ``a_i``).
An alpha-bit register ``r = r_0 r_1 ... r_{alpha-1}`` is a Python int whose bit
``i`` is ``r_i`` (the little-endian order a byte-mask instruction produces).
"""
from __future__ import annotations

from typing import Sequence

# ---------------------------------------------------------------------------
# Section 3.1 — specialised word-size instructions (semantics from their
# definitions; pinned by the worked examples in tests/golden/).
# ---------------------------------------------------------------------------


def wscmp(a: Sequence[int], b: Sequence[int]) -> int:
    """Word-size compare (Section 3.1): r_i = 1 iff a_i == b_i."""
    assert len(a) == len(b)
    r = 0
    for i, (x, y) in enumerate(zip(a, b)):
        if x == y:
            r |= 1 << i
    return r


def wsmatch(a: Sequence[int], b: Sequence[int]) -> int:
    """Word-size pattern match (Section 3.1): r_i = 1 iff b occurs in a at i.

    ``b`` has length k <= alpha; r_i = 0 for alpha-k < i < alpha.
    """
    alpha, k = len(a), len(b)
    assert 0 < k <= alpha
    r = 0
    for i in range(alpha - k + 1):
        if all(a[i + j] == b[j] for j in range(k)):
            r |= 1 << i
    return r


def wsblend(a: Sequence[int], b: Sequence[int]) -> tuple:
    """Word-size blend (Section 3.1): the high half of a followed by the low half of b."""
    alpha = len(a)
    assert len(b) == alpha and alpha % 2 == 0
    h = alpha // 2
    return tuple(a[h:]) + tuple(b[:h])


CRC32C_POLY_REFLECTED = 0x82F63B78  # Castagnoli polynomial 0x1EDC6F41, bit-reflected


def crc32c_update(crc: int, data: bytes) -> int:
    """Bitwise reflected CRC-32C update (no pre/post inversion), the operation a
    hardware crc32 instruction performs on its accumulator."""
    for byte in data:
        crc ^= byte
        for _ in range(8):
            crc = (crc >> 1) ^ (CRC32C_POLY_REFLECTED if crc & 1 else 0)
    return crc & 0xFFFFFFFF


def wscrc(block8: bytes) -> int:
    """Word-size CRC (Section 3.1): 32-bit CRC of a 64-bit block.

    The accumulator's start value is not stated; it is read as 0.
    """
    assert len(block8) == 8
    return crc32c_update(0, bytes(block8))


def bits(r: int):
    """{r}: the set bits of a register, ascending (Section 3.1)."""
    i = 0
    while r:
        if r & 1:
            yield i
        r >>= 1
        i += 1


# ---------------------------------------------------------------------------
# Section 3.2-3.4 — EPSMa, EPSMb, EPSMc on SSE-width words (w=128, gamma=8,
# alpha=16).  Readings of garbled or silent points are marked "reading".
# ---------------------------------------------------------------------------

ALPHA = 16


def _naive(t: bytes, p: bytes, s: int) -> bool:
    m = len(p)
    return 0 <= s and s + m <= len(t) and t[s:s + m] == p


def epsm_a(p: bytes, t: bytes, alpha: int = ALPHA) -> list:
    """EPSMa (Section 3.2): broadcast words B_j = (p_j)^alpha, r = AND_j (s_j >> j)."""
    n, m = len(t), len(p)
    if m == 0 or m > n:
        return []
    mp = min(m, alpha // 2)
    B = [tuple([p[i]] * alpha) for i in range(mp)]
    out = []
    nblocks = n // alpha
    for i in range(nblocks):
        T = tuple(t[i * alpha:(i + 1) * alpha])
        r = (1 << alpha) - 1
        for j in range(mp):
            s_j = wscmp(T, B[j])
            # reading: the shift aligns character k+j of the block with bit k, so
            # in little-endian bit order it is a right shift (r_k needs s_j[k+j]).
            r &= s_j >> j
        for k in bits(r):
            s = i * alpha + k
            if m == mp:
                out.append(s)
            elif _naive(t, p, s):
                out.append(s)
        # reading: the starts not covered by r are the m'-1 starts whose prefix
        # crosses into the next block, (i+1)*alpha - j for j = m'-1 .. 1.
        for j in range(mp - 1, 0, -1):
            s = (i + 1) * alpha - j
            if _naive(t, p, s):
                out.append(s)
    # reading: starts in the incomplete last block are checked naively.
    for s in range(nblocks * alpha, n - m + 1):
        if _naive(t, p, s):
            out.append(s)
    return out


def epsm_b(p: bytes, t: bytes, alpha: int = ALPHA) -> list:
    """EPSMb (Section 3.3): wsmatch of the m'-prefix on T_i (first half of the
    starts) and on wsblend(T_i, T_{i+1}) (second half)."""
    n, m = len(t), len(p)
    if m == 0 or m > n:
        return []
    h = alpha // 2
    mp = min(m, h)
    pp = tuple(p[:mp])
    low = (1 << h) - 1  # the word compare yields the first alpha/2 starts only
    out = []
    nblocks = n // alpha

    def report(base, r):
        for k in bits(r):
            s = base + k
            if m == mp or _naive(t, p, s):
                if s + m <= n:
                    out.append(s)

    for i in range(nblocks):
        T = tuple(t[i * alpha:(i + 1) * alpha])
        report(i * alpha, wsmatch(T, pp) & low)
        nxt = t[(i + 1) * alpha:(i + 1) * alpha + h]
        if len(nxt) == h:
            S = wsblend(T, tuple(nxt) + tuple([0] * (alpha - h)))
            report(i * alpha + h, wsmatch(S, pp) & low)
        else:
            # reading: no next block exists at the end of the text, so the
            # second-half starts of the last block are checked naively.
            for s in range(i * alpha + h, (i + 1) * alpha):
                if _naive(t, p, s):
                    out.append(s)
    for s in range(nblocks * alpha, n - m + 1):
        if _naive(t, p, s):
            out.append(s)
    return out


def epsm_c(p: bytes, t: bytes, k: int = 11, beta: int = 8) -> list:
    """EPSMc (Section 3.4): fingerprint filter on aligned text blocks.

    reading: the fingerprint is a CRC of a 64-bit block, so blocks are beta = 8
    characters (an alpha-character block need not lie inside a short occurrence).
    reading: blocks are inspected every q = floor(m/beta) - 1 blocks, the
    paper's shift (floor(m/alpha) - 1) * alpha taken as the whole stride.
    reading: the table L keeps the pattern offsets j in [0, beta*q), so that each
    occurrence has exactly one inspected block with 8b - s in L and is reported
    once; keeping every j in [0, m-beta] would report some occurrences twice.
    reading: a candidate s = beta*b - j is valid for 0 <= s <= n - m.
    """
    n, m = len(t), len(p)
    if m == 0 or m > n:
        return []
    q = m // beta - 1
    assert q >= 1, "EPSMc needs m >= 2*beta"
    mask = (1 << k) - 1
    L = {}
    for j in range(beta * q):
        v = wscrc(p[j:j + beta]) & mask
        L.setdefault(v, []).append(j)
    out = []
    for b in range(0, n // beta, q):
        v = wscrc(t[b * beta:(b + 1) * beta]) & mask
        for j in L.get(v, ()):
            s = b * beta - j
            if 0 <= s <= n - m and _naive(t, p, s):
                out.append(s)
    return out


def epsm(p: bytes, t: bytes) -> list:
    """EPSM dispatcher (Section 3): a for 0<m<4, b for 4<=m<16, c for m>=16."""
    m = len(p)
    if m < 4:
        return epsm_a(p, t)
    if m < 16:
        return epsm_b(p, t)
    return epsm_c(p, t)
