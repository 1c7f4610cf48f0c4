"""The multi-rank path on CPU: a vote split across world_size-2 gloo ranks
(each rank votes its 4 KiB-aligned shard; here with the oracle standing in for
the rank's GPU) and merged with one SUM and one MIN all-reduce equals the
oracle's vote of the whole problem, digests included.  Also the bench's
max-over-ranks timing reduction."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1405_2912_b300 import shard, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = {}
        for name, p in (("cfg3_f64", synth.cfg3(n=50_001, block=2000, ties=40)[0]),
                        ("cfg1", synth.cfg1(n=70_003, flips=60))):
            s0, s1 = shard.shard_range(p.n, p.itemsize, rank, world)
            part = oracle.vote([r[s0:s1] for r in p.replicas], p.dtype, p.abs_tol, p.rel_tol)
            local = {"mismatch": [int(x) for x in part["mismatch"]],
                     "first_mismatch": [int(x) for x in part["first_mismatch"]],
                     "no_majority": part["no_majority"], "first_no_majority": part["first_no_majority"]}
            merged = shard.all_reduce_stats(shard.local_to_global(local, s0))
            res[name] = (merged, s0, s1, part["out"].tobytes(), part["block_crc"].tobytes())
        import bench
        t = bench.max_over_ranks(float(rank + 1), world)
        q.put((rank, res, t))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_vote_merge():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort(key=lambda x: x[0])
    for name, p in (("cfg3_f64", synth.cfg3(n=50_001, block=2000, ties=40)[0]),
                    ("cfg1", synth.cfg1(n=70_003, flips=60))):
        whole = oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol)
        ranks = [g[1][name] for g in got]
        for merged, *_ in ranks:
            assert merged["mismatch"] == [int(x) for x in whole["mismatch"]]
            assert merged["first_mismatch"] == [int(x) for x in whole["first_mismatch"]]
            assert merged["no_majority"] == whole["no_majority"]
            assert merged["first_no_majority"] == whole["first_no_majority"]
        assert ranks[0][1] == 0 and ranks[0][2] == ranks[1][1] and ranks[1][2] == p.n
        assert b"".join(r[3] for r in ranks) == whole["out"].tobytes()
        crc = np.concatenate([np.frombuffer(r[4], dtype=np.uint32) for r in ranks])
        assert np.array_equal(crc, whole["block_crc"])
    assert all(g[2] == 2.0 for g in got)


@pytest.mark.parametrize("n,itemsize,world", [(0, 4, 3), (1, 4, 2), (1024, 4, 2), (1025, 4, 2),
                                             (10_000_001, 8, 8), (4096 * 7 + 5, 1, 4)])
def test_shard_ranges_cover_and_align(n, itemsize, world):
    rs = [shard.shard_range(n, itemsize, r, world) for r in range(world)]
    assert rs[0][0] == 0 and rs[-1][1] == n
    for (a0, a1), (b0, b1) in zip(rs, rs[1:]):
        assert a1 == b0
    for a0, a1 in rs:
        if a0 == a1:
            continue                      # an empty shard
        assert (a0 * itemsize) % 4096 == 0
        assert a1 == n or (a1 * itemsize) % 4096 == 0


def test_merge_host_side():
    a = {"mismatch": [0, 2], "first_mismatch": [-1, 10], "no_majority": 1, "first_no_majority": 10}
    b = {"mismatch": [3, 0], "first_mismatch": [200, -1], "no_majority": 0, "first_no_majority": -1}
    m = shard.merge([a, b])
    assert m == {"mismatch": [3, 2], "first_mismatch": [200, 10], "no_majority": 1, "first_no_majority": 10}
