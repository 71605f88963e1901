"""Filter soundness (GPU): a build of the library whose single-search filters
pass every start (-DEPSM_FILTER_SOUNDNESS=1: prefix and block filters mark
everything, the block fingerprint marks every block, the code filter keeps
every start) must give exactly the oracle's results, so the verification
steps alone are exact and the filters of the normal build only prune."""
import ctypes

import numpy as np
import pytest

import gen
import oracle
from tests._texts import periodic_runs_text

pytestmark = pytest.mark.gpu

VARIANTS = {2: range(4, 16), 3: range(8, 16), 4: range(15, 33), 5: range(7, 17),
            6: range(2, 17), 7: range(5, 17), 8: range(23, 33)}


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def sound(torch):
    import paper_1209_6449_gb300 as epsm
    from paper_1209_6449_gb300 import _native, build
    lib = _native.load(build.LIB_SOUND)
    h = ctypes.c_void_p()
    assert lib.epsm_create(ctypes.byref(h), 0, 0) == 0
    yield lib, h, epsm
    lib.epsm_destroy(h)


def _search(sound, torch, dev, n, pattern, variant, cap):
    lib, h, epsm = sound
    out = torch.empty(max(cap, 1), dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = lib.epsm_search_variant(h, variant, dev.data_ptr(), n, epsm._buf(pattern), len(pattern),
                                 out.data_ptr(), cap, cnt.data_ptr(), None)
    assert st == 0
    assert lib.epsm_sync(h, None) in (0, 2)
    c = int(cnt.item())
    return c, out[:min(c, cap)].cpu().numpy().astype(np.uint64)


@pytest.mark.parametrize("kind", ["dna", "protein", "dna_runs", "binary"])
def test_verification_alone_is_exact(sound, torch, kind):
    spec = gen.TextSpec(kind, 21)
    n = 3 * 16384 + 777
    host = spec.host(n)
    for off in (0, 5):
        dev = torch.from_numpy(host).cuda()[off:]
        ref = host[off:]
        for v, ms in VARIANTS.items():
            for m in list(ms)[::3] + [max(ms)]:
                pats = gen.mixed_patterns(spec, n, m, 2, stream_seed=m + v)
                if kind == "dna_runs":
                    pats.append(b"A" * m)
                for p in pats:
                    want = oracle.search(ref, p)
                    c, got = _search(sound, torch, dev, n - off, p, v, want.size + 8)
                    assert c == want.size and np.array_equal(got, want), (kind, v, m, off)


def test_verification_alone_periodic(sound, torch):
    """Periodic patterns in runs of periodic strings: with every start a
    candidate, the block variants' shortcut for the start one period after a
    confirmed occurrence must stay exact."""
    n = 4 * 16384 + 99
    host, units = periodic_runs_text(n, 77)
    dev = torch.from_numpy(host).cuda()
    for v in (4, 8):
        for m in (VARIANTS[v][0], 24, 32):
            for u in units:
                p = (u * (m // len(u) + 2))[:m]
                want = oracle.search(host, p)
                c, got = _search(sound, torch, dev, n, p, v, want.size + 8)
                assert c == want.size and np.array_equal(got, want), (v, m, u)


def test_verification_alone_long_patterns(sound, torch):
    spec = gen.TextSpec("dna", 22)
    n = 2 * 16384 + 101
    host = spec.host(n)
    dev = torch.from_numpy(host).cuda()
    for m in (33, 64, 300):
        for p in gen.planted_patterns(spec, n, m, 2, stream_seed=m):
            want = oracle.search(host, p)
            c, got = _search(sound, torch, dev, n, p, 4, want.size + 8)
            assert c == want.size and np.array_equal(got, want), m


def test_output_slots_past_the_count_untouched(torch):
    """Poison-filled output: exactly `count` slots are written, in order, and
    every slot past them keeps its poison (no stray or duplicate writes)."""
    import paper_1209_6449_gb300 as epsm
    ctx = epsm.Context(0)
    try:
        for kind, m in (("dna", 2), ("dna", 8), ("protein", 3), ("dna_runs", 6), ("markov96", 24)):
            spec = gen.TextSpec(kind, 23)
            n = 5 * 16384 + 333
            host = spec.host(n)
            dev = torch.from_numpy(host).cuda()
            p = b"A" * m if kind == "dna_runs" else gen.planted_patterns(spec, n, m, 1)[0]
            want = oracle.search(host, p)
            cap = want.size + 4096
            out = torch.full((cap,), -0x5A5A5A5A5A5A5A5B, dtype=torch.int64, device="cuda")
            cnt = ctx.search_into(dev, p, out, cap)
            got = out.cpu().numpy()
            assert cnt == want.size
            assert np.array_equal(got[:cnt].astype(np.uint64), want)
            assert (got[cnt:] == -0x5A5A5A5A5A5A5A5B).all(), (kind, m)
    finally:
        ctx.close()
