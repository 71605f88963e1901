"""GPU tests of long patterns (32 < m <= 4096) in the single search: the
8-byte block filter and check on the first 32 bytes, then the rest of the
pattern at each candidate (the Section 3.4 procedure, which covers any
m >= 16).  Every position is compared with the oracle."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

LONG_MS = (33, 40, 63, 64, 65, 100, 257, 1000, 4096)


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def ctx(torch):
    import paper_1209_6449_gb300 as epsm
    c = epsm.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("kind", ["dna", "protein", "bytes256", "dna_runs"])
def test_long_patterns_match_oracle(ctx, torch, kind):
    spec = gen.TextSpec(kind, 11)
    n = (3 << 20) + 5
    host = spec.host(n)
    dev = torch.from_numpy(host).cuda()
    for m in LONG_MS:
        pats = gen.planted_patterns(spec, n, m, 2, stream_seed=m) + gen.random_patterns(spec, m, 1)
        if kind == "dna_runs":
            pats.append(b"A" * m)
        for p in pats:
            for off in (0, 3):  # text pointer at two alignments
                want = oracle.search(host[off:], p)
                cnt, pos = ctx.search(dev[off:], p, capacity=want.size + 8)
                assert cnt == want.size, (kind, m, off)
                assert np.array_equal(pos.cpu().numpy().astype(np.uint64), want), (kind, m, off)
                assert ctx.count(dev[off:], p) == want.size


def test_long_periodic_pattern(ctx, torch):
    """(ab)^k patterns in an (ab)^n text with a few mutations: overlapping
    occurrences every 2 bytes, each prefix candidate passing the first 32 bytes."""
    n = 1 << 20
    host = np.frombuffer(b"ab" * (n // 2), dtype=np.uint8).copy()
    rng = np.random.default_rng(4)
    host[rng.integers(0, n, size=40)] = ord("x")
    dev = torch.from_numpy(host).cuda()
    for k in (17, 20, 50, 300):
        p = b"ab" * k
        want = oracle.search(host, p)
        cnt, pos = ctx.search(dev, p, capacity=want.size + 8)
        assert cnt == want.size and np.array_equal(pos.cpu().numpy().astype(np.uint64), want), k


def test_long_closed_form(ctx, torch):
    """a^m in a^n: exactly the starts 0..n-m."""
    n = (1 << 20) + 3
    dev = torch.full((n,), 0x61, dtype=torch.uint8, device="cuda")
    for m in (33, 500, 4096):
        cnt, pos = ctx.search(dev, b"a" * m, capacity=n)
        assert cnt == n - m + 1
        assert np.array_equal(pos.cpu().numpy(), np.arange(n - m + 1))


def test_long_argument_errors(ctx, torch):
    import paper_1209_6449_gb300 as epsm
    dev = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(epsm.EpsmError):
        ctx.search(dev, b"a" * (epsm.MAX_M_LONG + 1))
    with pytest.raises(epsm.EpsmError):  # only the block variant takes m > 32
        ctx.search(dev, b"a" * 40, variant=epsm.VARIANT_PREFIX4)
    # m > n: count 0
    assert ctx.count(dev[:100], b"a" * 200) == 0
