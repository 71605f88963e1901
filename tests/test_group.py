"""GPU parity of the shared-text batched search: all pairs on one text are one
group (one pass over its stages, one shared fingerprint filter per length
class).  Every pattern's positions must equal the oracle's for that pattern
alone, whatever else shares the pass."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def ctx():
    import paper_1209_6449_gb300 as epsm
    c = epsm.Context(0)
    yield c
    c.close()


def _dev(torch, host, off=0):
    buf = torch.zeros(host.size + off + 1, dtype=torch.uint8, device="cuda")
    if host.size:
        buf[off:off + host.size] = torch.from_numpy(host).cuda()
    return buf, (buf.data_ptr() + off, int(host.size))


def _check(ctx, torch, views, hosts, pats, slack=8):
    """views[i] is the (ptr, n) of pair i, hosts[i] its host copy."""
    want = [oracle.search(h, p) for h, p in zip(hosts, pats)]
    total = sum(w.size for w in want)
    offs, out = ctx.search_batch(views, pats, total + slack)
    torch.cuda.synchronize()
    out = out.cpu().numpy().astype(np.uint64)
    bad = []
    for i, w in enumerate(want):
        got = out[offs[i]:offs[i + 1]]
        if not np.array_equal(got, w):
            bad.append((i, len(pats[i]), int(got.size), int(w.size),
                        sorted(set(w.tolist()) - set(got.tolist()))[:4],
                        sorted(set(got.tolist()) - set(w.tolist()))[:4]))
    assert not bad, bad[:12]
    assert offs[-1] == total
    return offs, out


@pytest.mark.parametrize("kind", ["protein", "dna", "nl64", "markov96"])
def test_many_patterns_one_text(ctx, torch, kind):
    spec = gen.TextSpec(kind, 21)
    n = (3 << 20) + 5
    host = spec.host(n)
    buf, view = _dev(torch, host, off=3)
    pats = []
    for m in range(1, 33):
        pats += gen.mixed_patterns(spec, n, m, 3, stream_seed=m)
    _check(ctx, torch, [view] * len(pats), [host] * len(pats), pats)


def test_more_patterns_than_a_class_holds(ctx, torch):
    """70 patterns of one class on one text: split over several groups."""
    spec = gen.TextSpec("protein", 5)
    n = 1 << 20
    host = spec.host(n)
    buf, view = _dev(torch, host)
    pats = []
    for m in (9, 12, 20, 31, 5):
        pats += gen.mixed_patterns(spec, n, m, 70, stream_seed=m + 100)
    _check(ctx, torch, [view] * len(pats), [host] * len(pats), pats)


def test_dense_hits_overflow_fallback(ctx, torch):
    """Runs of one symbol: every start matches for every class pattern, so the
    per-warp hit list overflows and the stage is redone pattern by pattern."""
    host = np.full(300_000, ord("A"), dtype=np.uint8)
    host[100_000:100_050] = ord("C")
    buf, view = _dev(torch, host, off=9)
    pats = [b"A" * m for m in (4, 5, 7, 8, 11, 14, 15, 16, 24, 32, 1, 2, 3)] + [b"C" * 4, b"AC" * 8]
    _check(ctx, torch, [view] * len(pats), [host] * len(pats), pats)


def test_runs_text_mixed(ctx, torch):
    spec = gen.TextSpec("dna_runs", 3)
    n = 2_000_003
    host = spec.host(n)
    buf, view = _dev(torch, host, off=1)
    pats = []
    for m in (3, 4, 6, 8, 12, 15, 16, 24, 32):
        pats += [b"A" * m] + gen.mixed_patterns(spec, n, m, 2, stream_seed=m)
    _check(ctx, torch, [view] * len(pats), [host] * len(pats), pats)


def test_alone_equals_in_the_mix(ctx, torch):
    """A pattern's result does not depend on what shares its pass: the batch
    with many texts, shared and not, equals each pattern searched alone."""
    specs = [gen.TextSpec(k, 40 + i) for i, k in enumerate(("dna", "protein", "nl64"))]
    hosts, bufs, views = [], [], []
    for i, sp in enumerate(specs):
        h = sp.host(500_000 + 77 * i)
        b, v = _dev(torch, h, off=i * 5)
        hosts.append(h)
        bufs.append(b)
        views.append(v)
    pv, ph, pp, pt = [], [], [], []
    rng = np.random.default_rng(7)
    for k in range(150):
        t = int(rng.integers(0, 3))
        m = int(rng.integers(1, 33))
        p = gen.mixed_patterns(specs[t], hosts[t].size, m, 2, stream_seed=1000 + k)[k % 2]
        pv.append(views[t])
        ph.append(hosts[t])
        pp.append(p)
        pt.append(t)
    offs, out = _check(ctx, torch, pv, ph, pp)
    for i in range(0, len(pp), 7):
        t = pt[i]
        text = bufs[t][t * 5:t * 5 + hosts[t].size]
        cnt, alone = ctx.search(text, pp[i])
        assert cnt == offs[i + 1] - offs[i], i
        assert np.array_equal(alone.cpu().numpy().astype(np.uint64), out[offs[i]:offs[i + 1]]), i


def test_group_edges(ctx, torch):
    """Texts shorter than a pattern, of one stage and of a stage plus a few
    bytes, with patterns of every class sharing them."""
    spec = gen.TextSpec("nl64", 9)
    pats = [b"e", b"th", b"the", b"the ", b"tion", b"and the", b"of the s", b"0123456789abcd",
            b"abcdefghijklmnopq", b"x" * 32]
    views, hosts, keep = [], [], []
    for n in (0, 1, 7, 16, 31, 16384, 16384 + 3, 16384 * 2 + 15, 100_000):
        h = spec.host(n)
        b, v = _dev(torch, h, off=n % 16)
        keep.append(b)
        for p in pats:
            views.append(v)
            hosts.append(h)
    _check(ctx, torch, views, hosts, pats * 9)


def test_short_patterns_share_two_byte_windows(ctx, torch):
    """Short patterns (m 2..4) of a group over a large alphabet share the
    2-byte window table; where their hits are dense the per-warp list
    overflows and each is redone alone with the masked direct compare."""
    rng = np.random.default_rng(12)
    host = gen.TextSpec("protein", 31).host(400_000).copy()
    host[50_000:90_000] = np.frombuffer(b"ab" * 20_000, dtype=np.uint8)      # dense "ab" stretch
    host[200_000:200_300] = ord("Q")
    buf, view = _dev(torch, host, off=6)
    pats = [b"ab", b"ba", b"aba", b"abab", b"QQ", b"QQQ", b"QQQQ", b"AC", b"DEF", b"KLMN"]
    for m in (2, 3, 4, 5, 9, 13, 20):
        pats += gen.mixed_patterns(gen.TextSpec("protein", 31), host.size, m, 2, stream_seed=m)
    pats += [bytes(host[o:o + int(rng.integers(2, 5))]) for o in rng.integers(0, host.size - 5, 20)]
    _check(ctx, torch, [view] * len(pats), [host] * len(pats), pats)
