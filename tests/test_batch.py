"""GPU parity of the batched persistent launch and of the host-buffer entry
point: every pair's positions equal the oracle's for that pair alone."""
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
def epsm():
    import paper_1209_6449_gb300 as epsm
    return epsm


@pytest.fixture(scope="module")
def ctx(epsm):
    c = epsm.Context(0)
    yield c
    c.close()


def _pairs(npairs, seed, hi_log2=17):
    pairs = gen.batch_pairs(npairs, seed=seed, n_lo_log2=0, n_hi_log2=hi_log2)
    hosts = [p.spec.host(p.n) for p in pairs]
    return pairs, hosts


def _run_batch(ctx, torch, hosts, patterns, offsets_in=None, capacity=None):
    devs = [torch.from_numpy(h).cuda() if h.size else torch.empty(0, dtype=torch.uint8,
                                                                   device="cuda") for h in hosts]
    # unaligned text starts: slice from a 1..15 byte offset into a padded buffer
    texts = []
    keep = []
    for i, h in enumerate(hosts):
        off = offsets_in[i] if offsets_in else (i * 7) % 16
        buf = torch.zeros(h.size + off, dtype=torch.uint8, device="cuda")
        if h.size:
            buf[off:] = devs[i]
        keep.append(buf)
        texts.append((buf.data_ptr() + off, int(h.size)))
    want = [oracle.search(h, p) for h, p in zip(hosts, patterns)]
    total = sum(w.size for w in want)
    cap = total + 8 if capacity is None else capacity
    offs, out = ctx.search_batch(texts, patterns, cap)
    torch.cuda.synchronize()
    return offs, out.cpu().numpy().astype(np.uint64), want, keep


def test_batch_matches_oracle_per_pair(ctx, torch):
    pairs, hosts = _pairs(300, seed=1)
    pats = [p.pattern for p in pairs]
    offs, out, want, _ = _run_batch(ctx, torch, hosts, pats)
    assert offs[-1] == sum(w.size for w in want)
    for i, w in enumerate(want):
        got = out[offs[i]:offs[i + 1]]
        assert np.array_equal(got, w), (i, pairs[i].n, len(pats[i]))


def test_batch_order_does_not_change_results(ctx, torch):
    pairs, hosts = _pairs(120, seed=2)
    pats = [p.pattern for p in pairs]
    offs, out, want, _ = _run_batch(ctx, torch, hosts, pats)
    perm = np.random.default_rng(5).permutation(len(pairs))
    offs2, out2, _, _ = _run_batch(ctx, torch, [hosts[i] for i in perm], [pats[i] for i in perm],
                                   offsets_in=[(int(i) * 7) % 16 for i in perm])
    for k, i in enumerate(perm):
        assert np.array_equal(out2[offs2[k]:offs2[k + 1]], out[offs[i]:offs[i + 1]])


def test_batch_dense_and_degenerate_pairs(ctx, torch):
    hosts = [np.full(n, ord("a"), dtype=np.uint8) for n in (0, 1, 5, 31, 32, 33, 40000, 70000)]
    pats = [b"a", b"a" * 2, b"a" * 6, b"a" * 32, b"a" * 32, b"a" * 15, b"a" * 16, b"a" * 3]
    offs, out, want, _ = _run_batch(ctx, torch, hosts, pats)
    for i, w in enumerate(want):
        assert np.array_equal(out[offs[i]:offs[i + 1]], w), i


def test_batch_capacity_overflow(ctx, torch, epsm):
    hosts = [np.full(10000, ord("a"), dtype=np.uint8) for _ in range(3)]
    pats = [b"aa", b"aaa", b"aaaa"]
    offs, out, want, _ = _run_batch(ctx, torch, hosts, pats, capacity=15000)
    assert list(offs) == [0, 9999, 9999 + 9998, 9999 + 9998 + 9997]
    assert np.array_equal(out[:9999], np.arange(9999))
    assert np.array_equal(out[9999:15000], np.arange(15000 - 9999))


def test_search_host_matches_oracle(ctx):
    spec = gen.TextSpec("protein", 8)
    n = 200_000 + 13
    host = spec.host(n)
    pats = []
    for m in (1, 2, 3, 4, 7, 8, 13, 15, 16, 23, 32):
        pats += gen.mixed_patterns(spec, n, m, 2, stream_seed=m)
    want = [oracle.search(host, p) for p in pats]
    total = sum(w.size for w in want)
    offs, pos = ctx.search_host(host, pats, total + 4)
    assert offs[-1] == total
    for k, w in enumerate(want):
        assert np.array_equal(pos[offs[k]:offs[k + 1]], w), k


def test_batch_graph_replay_and_reuse(ctx, torch):
    """Repeated batches of different sizes reuse the captured submission and
    stay exact."""
    for seed, npairs in ((11, 40), (12, 7), (13, 64), (14, 1)):
        pairs, hosts = _pairs(npairs, seed=seed, hi_log2=15)
        pats = [p.pattern for p in pairs]
        offs, out, want, _ = _run_batch(ctx, torch, hosts, pats)
        for i, w in enumerate(want):
            assert np.array_equal(out[offs[i]:offs[i + 1]], w), (seed, i)
    print("batch graph replay:", ctx.batch_uses_graph)


@pytest.mark.gpu
def test_autotuner_small_run():
    """The autotuner measures every candidate (variant, launch shape,
    fingerprint width) for each m and returns rows that cover their m; the
    context accepts them, and searches stay exact under every configuration
    it tried."""
    import paper_1209_6449_gb300 as epsm
    from paper_1209_6449_gb300 import autotune
    ctx = epsm.Context(0, tuning=None)
    try:
        res = autotune.autotune(ctx, ms=(2, 6, 9, 20, 27), buckets=(0,), classes=("dna", "text"),
                                bucket_n=(1 << 20,), reps=1, patterns=1)
        for cls in ("dna", "text", "mixed"):
            for m, r in res["classes"][cls]["0"].items():
                assert int(m) in autotune.COVER[r["variant"]], (cls, m, r)
                assert (r["variant"], r["shape"], r["kbits"]) in autotune.candidates(int(m))
        for m in (2, 6, 9, 20, 27):
            assert len(res["ms"]["dna"]["0"][str(m)]) == len(autotune.candidates(m))
        autotune.apply(ctx, res, "dna")
        for m, r in res["classes"]["dna"]["0"].items():
            assert ctx.get_tuning(0, int(m)) == (r["variant"], r["shape"], r["kbits"])
        # every configuration the tuner can pick gives the oracle's result
        host = gen.TextSpec("dna", 5).host((1 << 20) + 9)
        dev = __import__("torch").from_numpy(host).cuda()
        for m in (6, 27):
            p = gen.planted_patterns(gen.TextSpec("dna", 5), host.size, m, 1)[0]
            want = oracle.search(host, p)
            for v, sh, kb in autotune.candidates(m):
                ctx.set_tuning(-1, m, v, sh, kb)
                cnt, pos = ctx.search(dev, p, capacity=want.size + 8)
                assert cnt == want.size and (pos.cpu().numpy().astype("uint64") == want).all(), (v, sh, kb)
    finally:
        ctx.close()


@pytest.mark.gpu
def test_tuning_entry_points(ctx):
    import paper_1209_6449_gb300 as epsm
    h = ctx.handle
    assert epsm.epsm_set_tuning(h, 3, 5) == 1          # no such bucket
    assert epsm.epsm_set_tuning(h, 0, 3, epsm.VARIANT_BLOCK8) == 1  # does not cover m
    assert epsm.epsm_set_tuning(h, 0, 20, 0, 2) == 1   # no such shape
    assert epsm.epsm_set_tuning(h, 0, 20, 0, -1, 15) == 1  # width out of range
    assert epsm.epsm_set_tuning(h, 1, 20, epsm.VARIANT_BLOCK8, 0, 11) == 0
    assert epsm.epsm_get_tuning(h, 1, 20) == (0, epsm.VARIANT_BLOCK8, 0, 11)
    assert epsm.epsm_set_tuning(h, -1, 20, 0, -1, 12) == 0   # keep variant and shape
    assert epsm.epsm_get_tuning(h, 1, 20) == (0, epsm.VARIANT_BLOCK8, 0, 12)
