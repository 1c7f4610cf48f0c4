"""The multi-GPU split exercised on the real kernel with one GPU: a vote cut
into W 4 KiB-aligned shards (shard.shard_range), each shard voted by its own
ft_vote on views of the same device buffers (shards on different streams, so
that they also run at the same time), the per-shard statistics merged on the
host (shard.merge) and compared with the oracle's vote of the whole problem:
voted bytes, block digests, counts and first indices.  No peer memory and no
collective is involved: this is the data path each rank would run."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1405_2912_b300 import shard, synth

from _gpu import to_dev

pytestmark = pytest.mark.gpu


def _problems():
    f64, i32 = synth.cfg3(n=300_007, block=20_000, ties=200)
    return {"cfg1_f32": synth.cfg1(n=250_003, flips=80), "cfg3_f64": f64, "cfg3_i32": i32}


@pytest.mark.parametrize("world", [2, 3, 7])
@pytest.mark.parametrize("name", ["cfg1_f32", "cfg3_f64", "cfg3_i32"])
def test_sharded_ft_vote_equals_whole_oracle(name, world):
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    p = _problems()[name]
    n, isz = p.n, p.itemsize
    nbytes = n * isz
    reps = [to_dev(r) for r in p.replicas]
    out = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    nb = fv.n_blocks(nbytes)
    crc = torch.full((nb,), -1, dtype=torch.int32, device="cuda")
    stats = torch.full((world, 18), 99, dtype=torch.int64, device="cuda")
    streams = [torch.cuda.Stream() for _ in range(2)]
    ranges = [shard.shard_range(n, isz, r, world) for r in range(world)]
    descs = []
    for r, (s0, s1) in enumerate(ranges):
        off = s0 * isz
        d = fv.make_desc([x.data_ptr() + off for x in reps], out.data_ptr() + off,
                         crc.data_ptr() + 4 * (off // 4096), stats[r], p.abs_tol, p.rel_tol,
                         dtype=p.dtype, n=s1 - s0)
        descs.append(d)
    torch.cuda.synchronize()
    for r, d in enumerate(descs):
        fv.check(fv.ft_vote(ctypes.byref(d), fv.stream_handle(streams[r % 2])), "ft_vote")
    torch.cuda.synchronize()
    parts = [shard.local_to_global(fv.parse_stats(stats[r], p.R), s0) for r, (s0, _) in enumerate(ranges)]
    merged = shard.merge(parts)
    whole = oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol)
    assert out.cpu().numpy().tobytes() == whole["out"].tobytes()
    assert np.array_equal(crc.cpu().numpy().view(np.uint32), whole["block_crc"])
    assert merged["mismatch"] == [int(x) for x in whole["mismatch"]]
    assert merged["first_mismatch"] == [int(x) for x in whole["first_mismatch"]]
    assert merged["no_majority"] == whole["no_majority"]
    assert merged["first_no_majority"] == whole["first_no_majority"]
