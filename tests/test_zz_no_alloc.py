"""The entry point that allocates nothing (epsm_search_static).

Some callers may not allocate device memory themselves: a framework that
routes every allocation through its own pool, a real-time loop where an
allocation could stall or fail, a plug-in whose host pre-sizes all memory.
epsm_search_static serves them with the library's fixed scratch array, which
every call shares and which keeps the previous call's contents.  These tests
call it through the C ABI, two calls in a row per case, and require exactly
the oracle's positions and count and those of the ordinary context entry
point (the results are integers, so the tolerance is zero).  They also cover
the paths where leftover state in the shared array would show: count-only
calls, a text shorter than the pattern, and a capacity overflow followed by a
normal call.  The file is named so that pytest collects it last.
"""
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


def _static(epsm, torch, text, n, p, out, cap, res):
    """One call; returns (count, error bits) once it has completed."""
    stream = torch.cuda.current_stream().cuda_stream
    st = epsm.epsm_search_static(text.data_ptr() if n else 0, n, p, len(p),
                                 out.data_ptr() if cap else 0, cap, res.data_ptr(), stream)
    assert st == 0, epsm.epsm_status_str(st)
    torch.cuda.synchronize()
    cnt, err = (int(x) for x in res.cpu().numpy())
    return cnt, err


def test_static_entry_matches_oracle_and_context(torch, epsm):
    ctx = epsm.Context(0)
    spec = gen.TextSpec("dna", 21)
    n = 3 * (1 << 20) + 5
    host = spec.host(n + 3)
    text = torch.from_numpy(host).cuda()[3:]          # unaligned start, ragged end
    cap = 1 << 20
    out = torch.empty(cap, dtype=torch.int64, device="cuda")
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    pats = [gen.planted_patterns(spec, n + 3, 8, 1, stream_seed=1)[0],   # adaptive 4-byte block / 2-bit code
            gen.planted_patterns(spec, n + 3, 20, 1, stream_seed=2)[0],  # 8-byte block fingerprint
            gen.planted_patterns(spec, n + 3, 27, 1, stream_seed=3)[0],  # strided 8-byte block
            b"AC"]                                                       # dense packed compare
    try:
        for p in pats:
            want = oracle.search(host[3:], p)
            ctx_cnt, ctx_pos = ctx.search(text, p, capacity=cap)
            assert ctx_cnt == want.size
            for _ in range(2):                       # two calls in a row share the array
                out.fill_(-1)
                cnt, err = _static(epsm, torch, text, n, p, out, cap, res)
                assert err == 0 and cnt == want.size, (len(p), cnt, want.size)
                got = out[:cnt].cpu().numpy().astype(np.uint64)
                assert np.array_equal(got, want)
                assert np.array_equal(got, ctx_pos.cpu().numpy().astype(np.uint64))
                assert (out[cnt:cnt + 64].cpu().numpy() == -1).all()  # nothing past the count
            for _ in range(2):                       # count only (capacity 0)
                cnt, err = _static(epsm, torch, text, n, p, out, 0, res)
                assert err == 0 and cnt == want.size
    finally:
        ctx.close()


def test_static_entry_short_text_and_overflow(torch, epsm):
    out = torch.empty(1 << 16, dtype=torch.int64, device="cuda")
    res = torch.full((2,), 7, dtype=torch.int64, device="cuda")
    host = np.full(50_000, ord("c"), dtype=np.uint8)
    text = torch.from_numpy(host).cuda()
    # a text shorter than the pattern: count 0, no error, result words cleared
    for _ in range(2):
        cnt, err = _static(epsm, torch, text, 5, b"cccccc", out, 16, res)
        assert (cnt, err) == (0, 0)
    # more occurrences than capacity: the first `cap` positions, the true
    # count, and error bit 2
    for m in (2, 9, 24):
        want = oracle.search(host, b"c" * m)
        cap = 1000
        for _ in range(2):
            cnt, err = _static(epsm, torch, text, host.size, b"c" * m, out, cap, res)
            assert cnt == want.size and err == 2, (m, cnt, err)
            assert np.array_equal(out[:cap].cpu().numpy().astype(np.uint64), want[:cap])
        # a normal call afterwards: the shared counters were reset
        cnt, err = _static(epsm, torch, text, host.size, b"c" * m, out, out.numel(), res)
        assert cnt == want.size and err == 0
        assert np.array_equal(out[:cnt].cpu().numpy().astype(np.uint64), want)


def test_static_entry_largest_text(torch, epsm):
    """A text of exactly the maximum size, at an unaligned start, with the
    variant whose stages reach furthest (the strided block variant, m >= 23)."""
    n = epsm.STATIC_MAX_TEXT
    spec = gen.TextSpec("protein", 5)
    host = spec.host(n + 7)
    buf = torch.from_numpy(host).cuda()
    text = buf[7:]
    out = torch.empty(1 << 16, dtype=torch.int64, device="cuda")
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    for m in (4, 27):
        p = gen.planted_patterns(spec, n + 7, m, 1, stream_seed=m)[0]
        want = oracle.search(host[7:], p, threads=8)
        for _ in range(2):
            cnt, err = _static(epsm, torch, text, n, p, out, out.numel(), res)
            assert err == 0 and cnt == want.size
            assert np.array_equal(out[:cnt].cpu().numpy().astype(np.uint64), want)


def test_static_entry_rejects_texts_beyond_its_scratch(torch, epsm):
    text = torch.zeros(16, dtype=torch.uint8, device="cuda")
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    st = epsm.epsm_search_static(text.data_ptr(), epsm.STATIC_MAX_TEXT + 1, b"ab", 2, 0, 0,
                                 res.data_ptr(), 0)
    assert st == 1  # EPSM_ERR_ARG
