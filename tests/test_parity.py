"""GPU parity: every kernel variant against the CPU oracle, element by element,
on seeded inputs spanning several tiles with ragged tails and unaligned starts.
Exact equality (count and every position): the result is a set of integers."""
import numpy as np
import pytest

import gen
import oracle
from tests._texts import periodic_runs_text

pytestmark = pytest.mark.gpu

TILE = 16384  # bytes per tile of the default launch (256 threads x 4 chunks x 16 B)


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def epsm():
    import paper_1209_6449_gb300 as epsm
    return epsm


@pytest.fixture(scope="module")
def ctx(epsm):
    c = epsm.Context(0)
    yield c
    c.close()


VARIANTS = {  # variant -> covered m
    1: range(1, 5),
    2: range(4, 16),
    3: range(8, 16),
    4: range(15, 33),
    5: range(7, 17),
    6: range(2, 17),
    7: range(5, 17),
    8: range(23, 33),
}


def _check(ctx, torch, host, pattern, variant, offset=0, capacity=None):
    """Search host[offset:] on the device and compare with the oracle."""
    dev = torch.from_numpy(np.ascontiguousarray(host)).cuda()
    text = dev[offset:]
    want = oracle.search(host[offset:], pattern)
    cap = want.size + 8 if capacity is None else capacity
    cnt, pos = ctx.search(text, pattern, capacity=cap, variant=variant)
    got = pos.cpu().numpy().astype(np.uint64)
    assert cnt == want.size, (len(pattern), variant, offset, cnt, want.size)
    k = min(cap, want.size)
    assert np.array_equal(got[:k], want[:k]), (len(pattern), variant, offset)
    return want.size


@pytest.mark.parametrize("variant", sorted(VARIANTS))
@pytest.mark.parametrize("kind", ["dna", "protein", "nl64", "markov96", "bytes256", "binary"])
def test_variant_all_m(ctx, torch, variant, kind):
    spec = gen.TextSpec(kind, 3)
    n = 3 * TILE + 1234
    host = spec.host(n)
    for m in VARIANTS[variant]:
        pats = gen.mixed_patterns(spec, n, m, 4, stream_seed=variant)
        for i, p in enumerate(pats):
            _check(ctx, torch, host, p, variant, offset=(i * 5 + m) % 16)


@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_dense_runs_every_alignment(ctx, torch, variant):
    """a^m in a text of a's: n-m+1 overlapping hits; all 16 start alignments."""
    n = 2 * TILE + 77
    host = np.full(n, ord("a"), dtype=np.uint8)
    host[TILE + 5: TILE + 9] = ord("b")      # one break in the run
    for m in VARIANTS[variant]:
        for off in range(16):
            _check(ctx, torch, host, b"a" * m, variant, offset=off)


@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_periodic_patterns_in_periodic_runs(ctx, torch, variant):
    """Periodic patterns (period 1..10) in runs of the same periodic strings:
    dense candidates, each run's occurrences q apart (the block variants
    confirm those from the pattern's last 8 bytes after a full check)."""
    n = 6 * TILE + 515
    host, units = periodic_runs_text(n, 40 + variant)
    for m in VARIANTS[variant]:
        for u in units:
            p = (u * (m // len(u) + 2))[:m]
            for off in (0, 7):
                _check(ctx, torch, host, p, variant, offset=off)


@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_tile_boundary_plants(ctx, torch, variant):
    """Occurrences planted across every tile, warp-run and chunk boundary."""
    spec = gen.TextSpec("dna", 9)
    n = 4 * TILE + 999
    for m in VARIANTS[variant]:
        host = spec.host(n).copy()
        pat = bytes(gen.random_patterns(gen.TextSpec("bytes256", 1), m, 1, stream_seed=m)[0])
        pat = bytes(b | 0x80 for b in pat)      # bytes absent from the DNA text
        plants = []
        for boundary in list(range(512, n, 512)) + [0, n - m]:
            for j in (0, 1, m // 2, m - 1, m):
                o = boundary - j
                if 0 <= o <= n - m and all(abs(o - q) >= m for q in plants):
                    plants.append(o)
        for o in plants:
            host[o:o + m] = np.frombuffer(pat, dtype=np.uint8)
        for off in (0, 3):
            cnt = _check(ctx, torch, host, pat, variant, offset=off)
            assert cnt == sum(1 for o in plants if o >= off)


@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_edges(ctx, torch, epsm, variant):
    spec = gen.TextSpec("bytes256", 4)
    for m in (min(VARIANTS[variant]), max(VARIANTS[variant])):
        for n in (0, 1, m - 1, m, m + 1, 15, 16, 17, 31, 33, 511, 513, TILE - 1, TILE, TILE + 1):
            if n < 0:
                continue
            host = spec.host(n)
            if n >= m:
                for p in (bytes(host[:m]), bytes(host[n - m:])):
                    _check(ctx, torch, host, p, variant)
            else:
                dev = torch.zeros(max(n, 1), dtype=torch.uint8, device="cuda")[:n]
                cnt, _ = ctx.search(dev, b"\x00" * m, capacity=4, variant=variant)
                assert cnt == 0


def test_high_bytes_and_zero_bytes(ctx, torch):
    """Unsigned compare: 0x00 and 0x80..0xFF match exactly."""
    host = gen.TextSpec("binary", 2).host(3 * TILE + 5)
    for m in range(1, 33):
        for p in (b"\x00" * m, b"\xff" * m, (b"\x00\xff" * 16)[:m], (b"\xff\x00\xff" * 11)[:m]):
            _check(ctx, torch, host, p, 0, offset=m % 16)


@pytest.mark.parametrize("variant", [6, 8])
def test_period_one_kernels_at_text_edges(ctx, torch, variant):
    """The period-1 kernels of the code and strided block variants read the
    chunks around a lane's own (bytes outside the text read as 0): a text of
    one byte value searched with that byte repeated, 0x00 included, at ragged
    lengths and alignments, must give exactly the n - m + 1 starts (closed
    form), and a single other byte must remove exactly the starts covering
    it."""
    for byte in (0x00, 0x41, 0xFF):
        for m in (min(VARIANTS[variant]), 9, max(VARIANTS[variant])):
            if m not in VARIANTS[variant]:
                continue
            for n in (m, m + 1, 511, 2 * TILE + 7, 3 * TILE + 1):
                for offset in (0, 1, 15):
                    host = np.full(n + offset, byte, dtype=np.uint8)
                    dev = torch.from_numpy(host).cuda()[offset:]
                    cnt, pos = ctx.search(dev, bytes([byte]) * m, capacity=n + 8, variant=variant)
                    assert cnt == n - m + 1, (byte, m, n, offset, cnt)
                    assert np.array_equal(pos.cpu().numpy(), np.arange(n - m + 1))
                    if n > 2 * m:
                        host[offset + n // 2] ^= 0x5A  # one other byte in the middle
                        _check(ctx, torch, host, bytes([byte]) * m, variant, offset=offset)


def test_capacity_overflow_and_count_only(ctx, torch, epsm):
    host = np.full(50_000, ord("c"), dtype=np.uint8)
    dev = torch.from_numpy(host).cuda()
    for m in (1, 5, 12, 20):
        want = 50_000 - m + 1
        cnt, pos = ctx.search(dev, b"c" * m, capacity=1000)
        assert cnt == want and np.array_equal(pos.cpu().numpy(), np.arange(1000))
        assert ctx.count(dev, b"c" * m) == want
    # the synchronous C entry point reports EPSM_ERR_CAPACITY with the true count
    out = torch.empty(10, dtype=torch.int64, device="cuda")
    st, cnt = epsm.epsm_search(ctx.handle, dev.data_ptr(), 50_000, b"cc", 2, out.data_ptr(), 10,
                               torch.cuda.current_stream().cuda_stream)
    assert st == 2 and cnt == 49_999
    assert list(out.cpu().numpy()) == list(range(10))


def test_auto_variant_matches_oracle_every_m(ctx, torch):
    spec = gen.TextSpec("nl64", 5)
    n = 5 * TILE + 3
    host = spec.host(n)
    for m in range(1, 33):
        for p in gen.mixed_patterns(spec, n, m, 2, stream_seed=77):
            _check(ctx, torch, host, p, 0, offset=m % 7)


def test_bad_arguments(ctx, torch, epsm):
    dev = torch.zeros(100, dtype=torch.uint8, device="cuda")
    out = torch.empty(4, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    h = ctx.handle
    s = torch.cuda.current_stream().cuda_stream
    assert epsm.epsm_search_async(h, dev.data_ptr(), 100, b"", 0, out.data_ptr(), 4,
                                  cnt.data_ptr(), s) == 1
    big = epsm.MAX_M_LONG + 1  # the single search takes m up to MAX_M_LONG
    assert epsm.epsm_search_async(h, dev.data_ptr(), 100, b"a" * big, big, out.data_ptr(), 4,
                                  cnt.data_ptr(), s) == 1
    # a variant that does not cover m
    assert epsm.epsm_search_variant(h, 4, dev.data_ptr(), 100, b"abc", 3, out.data_ptr(), 4,
                                    cnt.data_ptr(), s) == 1
    assert epsm.epsm_search_variant(h, 1, dev.data_ptr(), 100, b"abcde", 5, out.data_ptr(), 4,
                                    cnt.data_ptr(), s) == 1
    # the context is still usable
    assert ctx.count(dev, b"\x00\x00") == 99


def test_generators_host_equals_device(torch):
    for kind in gen.KINDS:
        spec = gen.TextSpec(kind, 12)
        for start, n in ((0, 100_003), (65_530, 70_001)):
            host = spec.host(n, start=start)
            dev = torch.zeros(n, dtype=torch.uint8, device="cuda")
            spec.device(n, dev.data_ptr(), torch.cuda.current_stream().cuda_stream, start=start)
            assert np.array_equal(dev.cpu().numpy(), host), kind


def test_bounded_wait_gives_up_and_context_stays_usable(ctx, torch, epsm):
    """A device wait on a flag that nothing sets gives up after its limit: the
    next sync reports EPSM_ERR_TIMEOUT once, and searches work afterwards."""
    s = torch.cuda.current_stream().cuda_stream
    assert epsm.epsm_wait_probe(ctx.handle, 20_000_000, s) == 0
    assert epsm.epsm_sync(ctx.handle, s) == 5   # EPSM_ERR_TIMEOUT
    assert epsm.epsm_sync(ctx.handle, s) == 0   # reported once, then cleared
    dev = torch.zeros(1000, dtype=torch.uint8, device="cuda")
    assert ctx.count(dev, b"\x00\x00\x00") == 998
    assert epsm.epsm_wait_probe(ctx.handle, 0, s) == 1        # EPSM_ERR_ARG
    assert epsm.epsm_wait_probe(ctx.handle, 2 * 10**9, s) == 1
