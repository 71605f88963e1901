"""Oracle pins (CPU only): the C brute-force oracle against closed forms,
exhaustive tiny inputs, a library string routine, an independent KMP counter,
planted occurrences and the paper's worked examples."""
import os

import numpy as np
import pytest

import gen
import oracle
from oracle import paper
from tests import _pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _search(t, p):
    return [int(x) for x in oracle.search(t, p)]


def test_closed_form_runs():
    _pins.check_closed_form_runs(_search)


def test_periodic():
    _pins.check_periodic(_search)


def test_exhaustive_binary():
    _pins.check_exhaustive_binary(_search)


def test_edges():
    _pins.check_edges(_search)


def test_planted_disjoint_alphabet():
    text = bytes(gen.TextSpec("dna", 5).host(1 << 16))
    for pat in (b"x", b"xy", b"xyz" * 3, b"zyx" * 10 + b"zz"):
        offs = list(range(3, (1 << 16) - 40, 997))
        offs = [o for i, o in enumerate(offs) if i % 2 == 0 or len(pat) < 997]
        _pins.check_planted(_search, text, pat, offs)


@pytest.mark.parametrize("kind", ["dna", "protein", "nl64", "markov96", "bytes256", "binary"])
def test_library_find(kind):
    spec = gen.TextSpec(kind, 11)
    text = bytes(spec.host(200_000))
    for m in (1, 2, 3, 5, 8, 13, 16, 24, 32):
        for p in gen.mixed_patterns(spec, len(text), m, 4, stream_seed=1):
            assert _search(text, p) == _pins.lib_positions(text, p), (kind, p)


@pytest.mark.parametrize("kind", ["dna", "dna_runs", "binary", "markov96"])
def test_kmp_and_threads(kind):
    spec = gen.TextSpec(kind, 2)
    n = 1 << 21
    text = spec.host(n)
    for m in (1, 2, 4, 7, 8, 15, 16, 31, 32):
        pats = gen.mixed_patterns(spec, n, m, 2, stream_seed=3)
        if kind == "dna_runs":
            pats.append(b"A" * m)
        for p in pats:
            c = oracle.count(text, p)
            assert c == oracle.kmp_count(text, p), (kind, p)
            single = oracle.search(text, p)
            multi = oracle.search(text, p, threads=7)
            assert single.size == c
            assert np.array_equal(single, multi)


def test_capacity_truncates():
    t = b"a" * 100
    lib = oracle._load()
    out = np.zeros(10, dtype=np.uint64)
    import ctypes
    tb = np.frombuffer(t, dtype=np.uint8)
    pb = np.frombuffer(b"aa", dtype=np.uint8)
    c = lib.oracle_search(tb.ctypes.data, 100, pb.ctypes.data, 2, out.ctypes.data, 10)
    assert c == 99 and list(out) == list(range(10))


# ---- the paper's primitives and procedures --------------------------------

def _read_golden(name):
    d = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            d[k.strip()] = v.split()
    return d


def _hexes(v):
    return [int(x, 16) for x in v]


def _reg(bitlist):
    return sum(int(b) << i for i, b in enumerate(bitlist))


def test_wscmp_worked_example():
    g = _read_golden("wscmp_example.txt")
    assert paper.wscmp(_hexes(g["a"]), _hexes(g["b"])) == _reg(g["r"])
    assert set(paper.bits(_reg(g["r"]))) == {1, 6, 8, 11}


def test_wsmatch_worked_example():
    g = _read_golden("wsmatch_example.txt")
    assert paper.wsmatch(_hexes(g["a"]), _hexes(g["b"])) == _reg(g["r"])
    assert set(paper.bits(_reg(g["r"]))) == {1, 5}


def test_wsblend_worked_example():
    g = _read_golden("wsblend_example.txt")
    assert list(paper.wsblend(_hexes(g["a"]), _hexes(g["b"]))) == _hexes(g["r"])


def test_crc32c_check_value():
    g = _read_golden("crc32c_check.txt")
    data = g["input"][0].encode()
    crc = paper.crc32c_update(0xFFFFFFFF, data) ^ 0xFFFFFFFF
    assert crc == int(g["check"][0], 16)


@pytest.mark.parametrize("kind", ["dna", "binary", "nl64", "bytes256"])
def test_paper_procedures_equal_definition(kind):
    """EPSMa/b/c restated from Section 3 give exactly the plain-definition set
    (no missed and no duplicated occurrence) under the readings they state."""
    spec = gen.TextSpec(kind, 7)
    for n in (0, 1, 15, 16, 17, 31, 64, 200, 1001):
        text = bytes(spec.host(n))
        for m in range(1, 33):
            pats = gen.mixed_patterns(spec, max(n, m), m, 2, stream_seed=n)
            if n >= m:
                pats.append(text[n - m:])          # occurrence at the very end
                pats.append(text[:m])              # occurrence at 0
            for p in pats:
                want = _search(text, p)
                assert sorted(paper.epsm(p, text)) == want, ("epsm", kind, n, p)
                if m < 16:
                    assert sorted(paper.epsm_a(p, text)) == want, ("a", kind, n, p)
                    assert sorted(paper.epsm_b(p, text)) == want, ("b", kind, n, p)
                else:
                    assert sorted(paper.epsm_c(p, text)) == want, ("c", kind, n, p)


def test_paper_procedures_periodic():
    for n in range(0, 80):
        t = b"A" * n
        for m in range(1, 33):
            want = list(range(n - m + 1)) if m <= n else []
            assert sorted(paper.epsm(b"A" * m, t)) == want


def test_long_patterns_pinned():
    """Long patterns (32 < m <= 4096, single search): the closed form a^m in
    a^n, the periodic (ab)^k family, and planted occurrences over a disjoint
    alphabet pin the oracle beyond m = 32."""
    for m in (33, 100, 4096):
        n = 5000
        text = np.full(n, 0x61, dtype=np.uint8)
        assert np.array_equal(oracle.search(text, b"a" * m), np.arange(n - m + 1, dtype=np.uint64))
    text = np.frombuffer(b"ab" * 3000, dtype=np.uint8)
    for k in (17, 40):
        got = oracle.search(text, b"ab" * k)
        assert np.array_equal(got, np.arange(0, 6000 - 2 * k + 1, 2, dtype=np.uint64))
        got = oracle.search(text, b"ba" * k)  # odd starts 1 .. 6000 - 2k - 1
        assert np.array_equal(got, np.arange(1, 6000 - 2 * k, 2, dtype=np.uint64))
    rng = np.random.default_rng(7)
    text = rng.integers(0, 4, size=1 << 16).astype(np.uint8)  # bytes 0..3
    pat = bytes(range(100, 100 + 60))  # disjoint from the text's bytes
    starts = [5, 1000, 1060, 40000]
    for s in starts:
        text[s:s + len(pat)] = np.frombuffer(pat, dtype=np.uint8)
    assert list(oracle.search(text, pat)) == starts
