"""Splitting one vote across ranks (one process per GPU) and merging the
per-rank statistics.

Elements are voted independently and each 4 KiB block of the voted buffer has
its own CRC32C, so a vote shards at 4096-byte-aligned element boundaries with
no exchange of data; the only exchange is the reduction of the per-replica
statistics: counts add up, first indices take the minimum of the shard-local
first index plus the shard's offset (-1 meaning none).  The block digests of
the shards concatenate in rank order.
"""
from __future__ import annotations

BLOCK = 4096


def shard_range(n: int, itemsize: int, rank: int, world: int) -> tuple:
    """[start, stop) element range of `rank`: whole 4 KiB blocks split as evenly
    as possible, the partial last block going to the last rank that has work."""
    per_block = BLOCK // itemsize
    nblocks = (n + per_block - 1) // per_block
    q, r = divmod(nblocks, world)
    b0 = rank * q + min(rank, r)
    b1 = b0 + q + (1 if rank < r else 0)
    return min(n, b0 * per_block), min(n, b1 * per_block)


NONE = (1 << 63) - 1


def local_to_global(stats: dict, start: int) -> dict:
    """Shard-local statistics with first indices moved to global indices."""
    g = dict(stats)
    g["first_mismatch"] = [f + start if f >= 0 else -1 for f in stats["first_mismatch"]]
    g["first_no_majority"] = stats["first_no_majority"] + start if stats["first_no_majority"] >= 0 else -1
    return g


def merge(parts: list) -> dict:
    """Merge global-index statistics of several shards (host-side)."""
    R = len(parts[0]["mismatch"])
    out = {"mismatch": [sum(int(p["mismatch"][r]) for p in parts) for r in range(R)],
           "no_majority": sum(int(p["no_majority"]) for p in parts)}
    firsts = []
    for r in range(R):
        c = [int(p["first_mismatch"][r]) for p in parts if int(p["first_mismatch"][r]) >= 0]
        firsts.append(min(c) if c else -1)
    out["first_mismatch"] = firsts
    c = [int(p["first_no_majority"]) for p in parts if int(p["first_no_majority"]) >= 0]
    out["first_no_majority"] = min(c) if c else -1
    return out


def all_reduce_stats(stats: dict, group=None) -> dict:
    """The same merge across the ranks of a torch.distributed group (any
    backend): one SUM and one MIN all-reduce of R+1 int64 values each."""
    import torch
    import torch.distributed as dist
    R = len(stats["mismatch"])
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else "cpu"
    cnt = torch.tensor([int(x) for x in stats["mismatch"]] + [int(stats["no_majority"])], dtype=torch.int64, device=dev)
    fst = torch.tensor([int(x) if int(x) >= 0 else NONE for x in stats["first_mismatch"]] +
                       [int(stats["first_no_majority"]) if int(stats["first_no_majority"]) >= 0 else NONE],
                       dtype=torch.int64, device=dev)
    dist.all_reduce(cnt, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(fst, op=dist.ReduceOp.MIN, group=group)
    c, f = cnt.tolist(), fst.tolist()
    return {"mismatch": c[:R], "no_majority": c[R],
            "first_mismatch": [x if x != NONE else -1 for x in f[:R]],
            "first_no_majority": f[R] if f[R] != NONE else -1}
