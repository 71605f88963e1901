"""GPU tests of the serving engine: every served query's count and positions
equal the oracle's and the single search's (alone), whatever shares its batch;
uploads are admitted by memory with LRU eviction; the per-query comparison
path serves the same results."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

KINDS = ("dna", "protein", "nl64", "markov96")


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def corpora(torch):
    texts = []
    for i, k in enumerate(KINDS):
        spec = gen.TextSpec(k, 70 + i)
        n = (1 << 20) + 13 * i
        host = spec.host(n)
        texts.append((spec, host, torch.from_numpy(host).cuda()))
    return texts


def _queries(corpora, count, seed):
    rng = np.random.default_rng(seed)
    qs = []
    for k in range(count):
        c = int(rng.integers(0, len(corpora)))
        m = int(rng.integers(2, 33))
        spec, host, _ = corpora[c]
        if k % 2:
            p = gen.planted_patterns(spec, host.size, m, 1, stream_seed=1000 + k)[0]
        else:
            p = gen.random_patterns(spec, m, 1, stream_seed=1000 + k)[0]
        qs.append((c, p))
    return qs


def _serve_all(srv, corpora, qs, torch):
    ids = [srv.add_corpus(t) for _, _, t in corpora]
    assert ids == list(range(len(corpora)))
    req = {}
    for c, p in qs:
        req[srv.submit(c, p)] = (c, p)
    got = {}
    while len(got) < len(req):
        for r in srv.poll(64, timeout_s=5.0):
            assert r["status"] == 0, r
            got[r["request"]] = srv.read(r["request"], r["count"]) if r["count"] else np.zeros(0, np.uint64)
            srv.release(r["request"])
    return req, got


@pytest.mark.parametrize("per_query", [False, True])
def test_served_results_match_oracle(corpora, torch, per_query):
    import paper_1209_6449_gb300 as epsm
    qs = _queries(corpora, 300 if not per_query else 60, seed=3)
    srv = epsm.Server(0, max_batch=128, inflight=2, per_query=per_query, out_capacity=1 << 16)
    try:
        req, got = _serve_all(srv, corpora, qs, torch)
        for rid, (c, p) in req.items():
            want = oracle.search(corpora[c][1], p)
            assert np.array_equal(got[rid], want), (c, p)
        st = srv.stats()
        assert st["queries"] == len(qs)
        if not per_query:
            assert st["batches"] < len(qs)  # queries were batched
    finally:
        srv.close()


def test_same_result_alone_and_in_the_mix(corpora, torch):
    """Each query served in a busy mix equals the same query searched alone
    (single search) and served alone."""
    import paper_1209_6449_gb300 as epsm
    qs = _queries(corpora, 200, seed=9)
    srv = epsm.Server(0, max_batch=64, inflight=2)
    ctx = epsm.Context(0)
    try:
        req, got = _serve_all(srv, corpora, qs, torch)
        for rid, (c, p) in list(req.items())[::5]:
            cnt, alone = ctx.search(corpora[c][2], p)
            assert np.array_equal(got[rid], alone.cpu().numpy().astype(np.uint64)), (c, p)
        solo = epsm.Server(0, max_batch=1, inflight=1)
        try:
            for _, _, t in corpora:
                solo.add_corpus(t)
            for (c, p) in [qs[i] for i in range(0, len(qs), 25)]:
                rid = solo.submit(c, p)
                r = solo.poll(1, timeout_s=10.0)[0]
                assert r["request"] == rid and r["status"] == 0
                mine = solo.read(rid, r["count"]) if r["count"] else np.zeros(0, np.uint64)
                solo.release(rid)
                assert np.array_equal(mine, oracle.search(corpora[c][1], p))
        finally:
            solo.close()
    finally:
        srv.close()
        ctx.close()


def test_dense_queries_grow_the_output(corpora, torch):
    """Short patterns on the DNA-like corpus overflow a small output buffer; the
    batch is re-run into a larger one and stays exact."""
    import paper_1209_6449_gb300 as epsm
    srv = epsm.Server(0, max_batch=32, inflight=2, out_capacity=1 << 10)
    try:
        qs = [(0, b"AC"), (0, b"G"), (0, b"TTA"), (1, b"AL"), (0, b"ACG")]
        req, got = _serve_all(srv, corpora, qs, torch)
        for rid, (c, p) in req.items():
            assert np.array_equal(got[rid], oracle.search(corpora[c][1], p))
        assert srv.stats()["reruns"] >= 1
    finally:
        srv.close()


@pytest.mark.parametrize("out_capacity", [1 << 12, 1 << 26])
def test_short_queries_on_large_corpora_follow_the_batch(torch, out_capacity):
    """On corpora of at least 16 MiB, a batch's short queries (m <= 4) run as
    single searches whose positions follow the batched part's in the same
    buffer; with a small buffer the whole mixed batch overflows and is re-run.
    Every result equals the oracle's, duplicates included."""
    import paper_1209_6449_gb300 as epsm
    big = []
    for i, k in enumerate(("dna", "protein")):
        spec = gen.TextSpec(k, 90 + i)
        host = spec.host((20 << 20) + 7 * i)
        big.append((spec, host, torch.from_numpy(host).cuda()))
    rng = np.random.default_rng(21)
    qs = []
    for k in range(60):
        c = k % 2
        m = int(rng.integers(1, 5)) if k % 3 else int(rng.integers(5, 33))
        spec, host, _ = big[c]
        p = (gen.planted_patterns(spec, host.size, m, 1, stream_seed=k)[0] if k % 2
             else gen.random_patterns(spec, m, 1, stream_seed=k)[0])
        qs.append((c, p))
    qs += qs[:6]  # the same queries again in the batch
    srv = epsm.Server(0, max_batch=128, inflight=1, out_capacity=out_capacity)
    try:
        req, got = _serve_all(srv, big, qs, torch)
        for rid, (c, p) in req.items():
            assert np.array_equal(got[rid], oracle.search(big[c][1], p, threads=8)), (c, p)
        if out_capacity < 1 << 20:
            assert srv.stats()["reruns"] >= 1
    finally:
        srv.close()


def test_upload_admission_and_eviction(corpora, torch):
    import paper_1209_6449_gb300 as epsm
    n = 1 << 20
    srv = epsm.Server(0, max_batch=16, upload_budget=3 * (n + 16))
    try:
        hosts = [gen.TextSpec("protein", 200 + i).host(n) for i in range(5)]
        cids = []
        for h in hosts:
            srv.upload(h)
            r = srv.poll(1, timeout_s=30.0)
            assert len(r) == 1 and r[0]["status"] == 0 and r[0]["count"] == n
            cids.append(r[0]["corpus"])
        st = srv.stats()
        assert st["uploads"] == 5 and st["evictions"] == 2
        # the two oldest uploads were evicted: queries on them are refused
        with pytest.raises(epsm.serve.ServerError):
            srv.submit(cids[0], b"ACDEFG")
        # the newest is resident and searchable
        p = bytes(hosts[4][1000:1012])
        rid = srv.submit(cids[4], p)
        r = srv.poll(1, timeout_s=10.0)[0]
        assert r["request"] == rid and r["status"] == 0
        assert np.array_equal(srv.read(rid, r["count"]), oracle.search(hosts[4], p))
        srv.release(rid)
    finally:
        srv.close()


def test_replay_counts_and_latencies(corpora, torch):
    import paper_1209_6449_gb300 as epsm
    qs = _queries(corpora, 400, seed=17)
    srv = epsm.Server(0, max_batch=256, inflight=2)
    try:
        for _, _, t in corpora:
            srv.add_corpus(t)
        rng = np.random.default_rng(1)
        at = np.cumsum(rng.exponential(1e9 / 20000.0, size=len(qs) + 1)).astype(np.int64)
        kinds = np.zeros(len(qs) + 1, dtype=np.uint32)
        kinds[200] = 1  # one upload in the stream
        corp = np.array([c for c, _ in qs[:200]] + [0] + [c for c, _ in qs[200:]], dtype=np.uint32)
        payload = [p for _, p in qs[:200]] + [gen.TextSpec("dna", 5).host(1 << 22)] + [p for _, p in qs[200:]]
        res = srv.replay(at, kinds, corp, payload)
        assert (res["status"] == 0).all()
        assert (res["latency_ns"] > 0).all()
        allq = qs[:200] + [None] + qs[200:]
        for i, q in enumerate(allq):
            if q is None:
                assert res["counts"][i] == 1 << 22
                continue
            c, p = q
            assert res["counts"][i] == oracle.count(corpora[c][1], p), i
        assert srv.stats()["uploads"] == 1
    finally:
        srv.close()


def _one(srv, timeout=30.0):
    r = srv.poll(1, timeout_s=timeout)
    assert len(r) == 1
    return r[0]


def test_injected_buffer_failure_fails_the_batch_and_serving_continues(corpora, torch):
    """A failure to obtain an output buffer (injected on the host) fails the
    queries of that batch with EPSM_ERR_NOMEM; the next queries are served
    exactly."""
    import paper_1209_6449_gb300 as epsm
    srv = epsm.Server(0, max_batch=16, inflight=1)
    try:
        for _, _, t in corpora:
            srv.add_corpus(t)
        srv.inject_fault(srv.FAULT_ALLOC, 1)
        p = bytes(corpora[1][1][5000:5009])
        rid = srv.submit(1, p)
        r = _one(srv)
        assert r["request"] == rid and r["status"] == 4 and r["count"] == 0  # EPSM_ERR_NOMEM
        for c in range(len(corpora)):
            q = bytes(corpora[c][1][777:777 + 6 + c])
            rid = srv.submit(c, q)
            r = _one(srv)
            assert r["request"] == rid and r["status"] == 0
            assert np.array_equal(srv.read(rid, r["count"]), oracle.search(corpora[c][1], q))
            srv.release(rid)
    finally:
        srv.close()


def test_injected_admission_and_upload_failures(corpora, torch):
    """Admission refused, then an upload copy failed (both injected on the
    host): those uploads complete with EPSM_ERR_NOMEM and EPSM_ERR_CUDA, hold no
    memory, and the next upload is admitted and searchable."""
    import paper_1209_6449_gb300 as epsm
    n = 1 << 20
    srv = epsm.Server(0, max_batch=16, upload_budget=2 * (n + 16))
    try:
        host = gen.TextSpec("protein", 301).host(n)
        srv.inject_fault(srv.FAULT_ADMIT, 1)
        srv.upload(host)
        assert _one(srv)["status"] == 4      # EPSM_ERR_NOMEM
        srv.inject_fault(srv.FAULT_UPLOAD, 1)
        srv.upload(host)
        assert _one(srv)["status"] == 3      # EPSM_ERR_CUDA
        assert srv.stats()["uploads"] == 0
        srv.upload(host)
        r = _one(srv)
        assert r["status"] == 0 and r["count"] == n
        cid = r["corpus"]
        p = bytes(host[4242:4254])
        rid = srv.submit(cid, p)
        q = _one(srv)
        assert q["request"] == rid and q["status"] == 0
        assert np.array_equal(srv.read(rid, q["count"]), oracle.search(host, p))
        srv.release(rid)
        # the two failed uploads left the budget free: a second text fits
        srv.upload(host)
        assert _one(srv)["status"] == 0
        assert srv.stats()["evictions"] == 0
    finally:
        srv.close()


def test_faults_armed_from_the_environment(corpora, torch, monkeypatch):
    import paper_1209_6449_gb300 as epsm
    monkeypatch.setenv("EPSM_FAULT", "alloc:2,bogus:3")
    srv = epsm.Server(0, max_batch=1, inflight=1)
    monkeypatch.delenv("EPSM_FAULT")
    try:
        srv.add_corpus(corpora[0][2])
        st = []
        for k in range(3):
            srv.submit(0, b"ACGTA"[:2 + k])
            st.append(_one(srv)["status"])
        assert st == [4, 4, 0]
    finally:
        srv.close()
