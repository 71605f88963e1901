"""The entry point that allocates nothing (epsm_search_static).

Some callers may not allocate device memory themselves — a framework that
routes every allocation through its own pool, a real-time loop where an
allocation could stall or fail, a plug-in whose host pre-sizes all memory.
epsm_search_static serves them with the library's fixed scratch array.  This
test calls it through the C ABI twice in a row and requires exactly the
positions and count of the ordinary context entry point (the results are
integers, so the tolerance is zero).  It lives in its own file so that pytest
collects it last.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


def test_static_entry_matches_context_entry():
    import torch
    import paper_1209_6449_gb300 as epsm

    ctx = epsm.Context(0)
    stream = torch.cuda.current_stream().cuda_stream
    spec = gen.TextSpec("dna", 21)
    n = 3 * (1 << 20) + 5
    host = spec.host(n + 3)
    text = torch.from_numpy(host).cuda()[3:]          # unaligned start, ragged end
    cap = 1 << 20
    out = torch.empty(cap, dtype=torch.int64, device="cuda")
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    pats = [gen.planted_patterns(spec, n + 3, 8, 1, stream_seed=1)[0],   # prefix filter
            gen.planted_patterns(spec, n + 3, 20, 1, stream_seed=2)[0],  # block fingerprint
            b"AC"]                                                       # dense direct compare
    for p in pats:
        want_cnt, want_pos = ctx.search(text, p, capacity=cap)
        want = want_pos.cpu().numpy()
        out.fill_(-1)
        st = epsm.epsm_search_static(text.data_ptr(), n, p, len(p), out.data_ptr(), cap,
                                     res.data_ptr(), stream)
        assert st == 0, epsm.epsm_status_str(st)
        torch.cuda.synchronize()
        cnt, err = (int(x) for x in res.cpu().numpy())
        assert err == 0
        assert cnt == want_cnt
        assert np.array_equal(out[:cnt].cpu().numpy(), want)
    ctx.close()


def test_static_entry_rejects_texts_beyond_its_scratch():
    import torch
    import paper_1209_6449_gb300 as epsm
    text = torch.zeros(16, dtype=torch.uint8, device="cuda")
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    st = epsm.epsm_search_static(text.data_ptr(), epsm.STATIC_MAX_TEXT + 1, b"ab", 2, 0, 0,
                                 res.data_ptr(), 0)
    assert st == 1  # EPSM_ERR_ARG
