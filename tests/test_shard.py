"""Multi-rank path on the CPU (gloo, world size 2 and 3): the text's starts are
split over ranks and the merged result equals the single-rank oracle result.
The per-shard search here is the oracle (a CPU stand-in); on GPUs it is the
library search of the shard's bytes."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import gen
import oracle


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, cases, results):
    import torch
    import torch.distributed as dist
    from paper_1209_6449_gb300.shard import sharded_search
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for kind, n, pat in cases:
            text = gen.TextSpec(kind, 3).host(n)

            def search_shard(s0, b1, p):
                return torch.from_numpy(oracle.search(text[s0:b1], p).astype(np.int64))

            merged, total = sharded_search(search_shard, n, pat)
            if rank == 0:
                results.append((kind, n, pat, merged.numpy().tolist(), total))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_search_equals_single_rank(world):
    cases = [("dna", 100_003, b"ACGTA"), ("dna", 5000, b"A"), ("binary", 70_001, b"\x00\xff\x00"),
             ("dna", 10, b"ACGTACGTACGTAC"), ("protein", 50_000, b"PQRS")]
    spec = gen.TextSpec("dna", 3)
    t = spec.host(100_003)
    cases.append(("dna", 100_003, bytes(t[50_000:50_020])))  # occurrence across a shard boundary
    mgr = mp.get_context("spawn").Manager()
    results = mgr.list()
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, cases, results), nprocs=world, join=True,
                       start_method="spawn")
    assert len(results) == len(cases)
    for kind, n, pat, merged, total in results:
        want = oracle.search(gen.TextSpec(kind, 3).host(n), pat)
        assert total == want.size
        assert merged == [int(x) for x in want], (kind, n, pat)


def test_shard_bounds_cover_every_start_once():
    from paper_1209_6449_gb300.shard import shard_bounds
    for n in (0, 1, 5, 31, 1000):
        for m in (1, 2, 7, 32):
            for world in (1, 2, 3, 8):
                starts = []
                for r in range(world):
                    s0, s1, b1 = shard_bounds(n, m, world, r)
                    starts += list(range(s0, s1))
                    if s1 > s0:
                        assert b1 == s1 + m - 1 and b1 <= n
                assert starts == list(range(max(n - m + 1, 0)))
