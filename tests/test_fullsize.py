"""GPU parity at the sizes the product is timed on: every position of the
CUDA path against the CPU oracle on the workloads themselves, not on small
stand-ins.

- the plain single search exactly as specified (1 MiB DNA-like text, seed 0,
  one m = 8 pattern copied from a uniform offset);
- every single-search variant on 96 MiB texts, so that every persistent
  block recycles its stage ring many times (the producer's empty-slot waits
  and the mbarrier phase flips run under the oracle check), including the
  5%-runs text searched with A^m and unaligned text starts;
- the pattern-length sweep's own 256 MiB texts and patterns (a planted and an
  i.i.d. pattern per text and m);
- a 4.5 GiB text, so that positions pass 2^32, compared start window by start
  window over the whole text;
- the large scan's 16 GiB texts in the benchmark's configuration (alphabet
  class tuning, the scan's own patterns), compared the same way;
- the full batched workload (8192 uneven pairs, about 24 GiB of text), each
  pair against the oracle on that pair alone;
- the served workload's four 1 GiB corpora, each served query against the
  oracle.

The oracle runs on all host cores.  Texts are made by the seeded generators:
on the device for the CUDA path, on the host for the oracle (the two byte
streams are identical, which test_parity checks).  Exact equality everywhere:
the result is a set of integers (Section 1: all occurrences).
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

MiB = 1 << 20
GiB = 1 << 30
CORES = os.cpu_count() or 1


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


def _device_text(torch, spec, n, lead=0):
    """The text on the device, starting `lead` bytes into its buffer."""
    buf = torch.zeros(n + lead + 16, dtype=torch.uint8, device="cuda")
    spec.device(n, buf.data_ptr() + lead, torch.cuda.current_stream().cuda_stream)
    return buf, buf[lead:lead + n]


def _gpu_positions(ctx, text, p, cap):
    cnt, pos = ctx.search(text, p, capacity=cap)
    assert cnt <= cap, (len(p), cnt, cap)
    return cnt, pos.cpu().numpy().astype(np.uint64)


def _windowed_compare(host, p, got, window=256 * MiB):
    """got (all GPU positions, ascending) against the oracle start window by
    start window: the starts in [a, b) are oracle.search(host[a:b+m-1]) + a."""
    n, m = host.size, len(p)
    starts = n - m + 1
    k = 0
    for a in range(0, starts, window):
        b = min(starts, a + window)
        want = oracle.search(host[a:b + m - 1], p, threads=CORES) + np.uint64(a)
        hi = int(np.searchsorted(got, np.uint64(b), side="left"))
        assert hi - k == want.size, (m, a, hi - k, want.size)
        assert np.array_equal(got[k:hi], want), (m, a)
        k = hi
    assert k == got.size


def test_plain_single_search_exact_config(ctx, torch, epsm):
    """1 MiB of i.i.d. ACGT (seed 0), one m = 8 pattern copied from a uniform
    random offset; count and every sorted position, through the synchronous
    C entry point and the asynchronous one."""
    n = 1 << 20
    spec = gen.TextSpec("dna", 0)
    host = spec.host(n)
    p = gen.planted_patterns(spec, n, 8, 1)[0]
    want = oracle.search(host, p)
    assert want.size >= 1 and oracle.kmp_count(host, p) == want.size
    dev = torch.from_numpy(host).cuda()
    out = torch.full((want.size + 64,), -1, dtype=torch.int64, device="cuda")
    st, cnt = epsm.epsm_search(ctx.handle, dev.data_ptr(), n, p, 8, out.data_ptr(), out.numel(),
                               torch.cuda.current_stream().cuda_stream)
    assert st == 0 and cnt == want.size
    got = out.cpu().numpy()
    assert np.array_equal(got[:cnt].astype(np.uint64), want) and (got[cnt:] == -1).all()
    cnt2, pos2 = _gpu_positions(ctx, dev, p, want.size + 8)
    assert cnt2 == want.size and np.array_equal(pos2, want)


VARIANT_MS = {  # variant -> pattern lengths: both ends of its range and one inside
    1: (1, 2, 4), 2: (4, 9, 15), 3: (8, 15), 4: (15, 24, 32), 5: (7, 16),
    6: (2, 8, 16), 7: (5, 11, 16), 8: (23, 32),
}


@pytest.mark.parametrize("kind", ["dna", "markov96", "dna_runs"])
def test_every_variant_with_ring_reuse(ctx, torch, kind):
    n = 96 * MiB + 4321
    lead = 5
    spec = gen.TextSpec(kind, 2)
    host = spec.host_parallel(n)
    buf, text = _device_text(torch, spec, n, lead=lead)
    for variant, ms in VARIANT_MS.items():
        for m in ms:
            pats = [gen.planted_patterns(spec, n, m, 1, stream_seed=variant)[0],
                    gen.random_patterns(spec, m, 1, stream_seed=variant)[0]]
            if kind == "dna_runs":
                pats.append(b"A" * m)   # every start inside a run of A is a hit
            for p in pats:
                want = oracle.search(host, p, threads=CORES)
                cnt, pos = ctx.search(text, p, capacity=want.size + 8, variant=variant)
                assert cnt == want.size, (kind, variant, m, cnt, want.size)
                assert np.array_equal(pos.cpu().numpy().astype(np.uint64), want), (kind, variant, m)
                assert ctx.count(text, p, variant=variant) == want.size


def test_pattern_length_sweep_texts(ctx, torch):
    """The sweep's 256 MiB texts (seed 0) and, per (text, m), the first planted
    and the first i.i.d. pattern of its 100."""
    n = 256 * MiB
    for kind in ("dna", "protein", "nl64"):
        spec = gen.TextSpec(kind, 0)
        host = spec.host_parallel(n)
        buf, text = _device_text(torch, spec, n)
        for m in (2, 4, 8, 16, 32):
            pats = gen.mixed_patterns(spec, n, m, 100)
            for p in (pats[0], pats[50]):
                want = oracle.search(host, p, threads=CORES)
                cnt, got = _gpu_positions(ctx, text, p, want.size + 8)
                assert cnt == want.size, (kind, m, cnt, want.size)
                assert np.array_equal(got, want), (kind, m)
        del buf, text


def test_text_past_four_gib(ctx, torch):
    """A 4.5 GiB text: 64-bit positions past 2^32, compared window by window
    over the whole text (dense, sparse and long patterns; planted ones start
    past 2^32)."""
    n = 4 * GiB + 512 * MiB + 77
    spec = gen.TextSpec("dna", 44)
    host = spec.host_parallel(n)
    buf, text = _device_text(torch, spec, n, lead=3)
    hi_start = (1 << 32) + 12345
    pats = [bytes(host[hi_start:hi_start + 8]), bytes(host[hi_start + 99:hi_start + 99 + 27]),
            bytes(host[n - 40:n]), gen.random_patterns(spec, 12, 1, stream_seed=4)[0], b"GAT"]
    for p in pats:
        cap = n // 48 if len(p) == 3 else 1 << 22
        cnt, got = _gpu_positions(ctx, text, p, cap)
        if len(p) in (8, 27, 40):
            assert got.size and int(got[-1]) >= (1 << 32)
        _windowed_compare(host, p, got)
        assert ctx.count(text, p) == cnt
    del buf, text


# the large scan's texts, their alphabet classes and a subset of its searches
# (m, pattern kind): dense and sparse outputs, every filter family, and the
# period-1 kernels on the runs text
SCAN_CASES = {"dna": ("dna", [(2, "planted"), (8, "iid"), (32, "planted")]),
              "markov96": ("text", [(4, "planted"), (16, "iid")]),
              "dna_runs": ("dna", [(3, "runs"), (8, "runs"), (24, "runs")])}


@pytest.mark.parametrize("kind", list(SCAN_CASES))
def test_large_scan_texts_in_the_timed_configuration(torch, epsm, kind):
    """The 16 GiB texts of the large scan (seed 0), searched as the benchmark
    does (a context with its alphabet class's tuning rows, the scan's own
    patterns), every position compared with the oracle start window by start
    window over the whole text."""
    n = 16 * GiB
    cls, cases = SCAN_CASES[kind]
    spec = gen.TextSpec(kind, 0)
    host = spec.host_parallel(n)
    buf, text = _device_text(torch, spec, n)
    c = epsm.Context(0, text_class=cls)
    try:
        for m, mode in cases:
            p = (b"A" * m if mode == "runs" else gen.random_patterns(spec, m, 1)[0] if mode == "iid"
                 else gen.planted_patterns(spec, n, m, 1)[0])
            cnt = c.count(text, p)
            _, got = _gpu_positions(c, text, p, cnt + 8)
            assert got.size == cnt
            _windowed_compare(host, p, got, window=1 * GiB)
    finally:
        c.close()
    del buf, text


def test_full_batched_workload(ctx, torch):
    """The 8192-pair batched workload (text lengths log-uniform 1 KiB..32 MiB,
    sigma 4/20/64, m 1..32, half planted): each pair's positions against the
    oracle on that pair alone."""
    pairs = gen.batch_pairs(8192, seed=0)
    tot = sum(p.n for p in pairs)
    buf = torch.empty(tot + 16 * len(pairs), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    views, off = [], 0
    for p in pairs:
        p.spec.device(p.n, buf.data_ptr() + off, s)
        views.append((buf.data_ptr() + off, p.n))
        off += (p.n + 15) // 16 * 16
    cap = 1 << 28
    offs, out = ctx.search_batch(views, [p.pattern for p in pairs], cap)
    torch.cuda.synchronize()
    total = int(offs[-1])
    assert total <= cap
    got = out[:total].cpu().numpy().astype(np.uint64)
    del out, buf

    def check(i):
        p = pairs[i]
        want = oracle.search(p.spec.host(p.n), p.pattern)
        g = got[int(offs[i]):int(offs[i + 1])]
        return None if np.array_equal(g, want) else (i, p.n, len(p.pattern), g.size, want.size)

    with ThreadPoolExecutor(max_workers=CORES) as ex:
        bad = [r for r in ex.map(check, range(len(pairs))) if r is not None]
    assert not bad, bad[:8]


def test_served_workload_corpora(torch):
    """The served workload's four 1 GiB corpora (seeds 900..903): a mix of
    queries served in shared batches, and a few served alone, each against the
    oracle."""
    import paper_1209_6449_gb300 as epsm
    n = GiB
    kinds = ("dna", "protein", "nl64", "markov96")
    specs = [gen.TextSpec(k, 900 + i) for i, k in enumerate(kinds)]
    devs = [_device_text(torch, sp, n)[1] for sp in specs]
    torch.cuda.synchronize()
    rng = np.random.default_rng(31)
    qs = []
    for c, sp in enumerate(specs):
        for k, m in enumerate((2, 3, 5, 8, 13, 21, 27, 32)):
            p = (gen.planted_patterns(sp, n, m, 1, stream_seed=k)[0] if k % 2
                 else gen.random_patterns(sp, m, 1, stream_seed=k)[0])
            qs.append((c, p))
    order = rng.permutation(len(qs))
    srv = epsm.Server(0, max_batch=1024, inflight=2, out_capacity=1 << 27)
    got = {}
    try:
        for d in devs:
            srv.add_corpus(d)
        req = {srv.submit(qs[i][0], qs[i][1]): int(i) for i in order}
        while len(got) < len(req):
            for r in srv.poll(64, timeout_s=30.0):
                assert r["status"] == 0, r
                got[req[r["request"]]] = (srv.read(r["request"], r["count"]) if r["count"]
                                          else np.zeros(0, np.uint64))
                srv.release(r["request"])
        assert srv.stats()["batches"] < len(qs)
    finally:
        srv.close()
    alone = {}
    solo = epsm.Server(0, max_batch=1, inflight=1, out_capacity=1 << 27)
    try:
        for d in devs:
            solo.add_corpus(d)
        for i in range(0, len(qs), 5):
            rid = solo.submit(*qs[i])
            r = solo.poll(1, timeout_s=30.0)[0]
            assert r["request"] == rid and r["status"] == 0
            alone[i] = solo.read(rid, r["count"]) if r["count"] else np.zeros(0, np.uint64)
            solo.release(rid)
    finally:
        solo.close()
    for c, sp in enumerate(specs):
        host = sp.host_parallel(n)
        for i, (cc, p) in enumerate(qs):
            if cc != c:
                continue
            want = oracle.search(host, p, threads=CORES)
            assert np.array_equal(got[i], want), (kinds[c], len(p))
            if i in alone:
                assert np.array_equal(alone[i], want), (kinds[c], len(p))
        del host
