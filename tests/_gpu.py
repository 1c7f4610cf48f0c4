"""Helpers for the GPU parity tests: run the CUDA path through the C ABI on
numpy inputs and compare with the oracle on the same inputs."""
import numpy as np

import oracle


def to_dev(a):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).copy())
    return t.to("cuda")


def gpu_vote(replicas, dtype, abs_tol=0.0, rel_tol=0.0):
    """ft_vote on byte copies of the numpy replicas; returns a dict like the oracle's."""
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    import ctypes
    n = replicas[0].size
    itemsize = np.dtype(oracle.NP_OF[dtype]).itemsize
    nbytes = n * itemsize
    devs = [to_dev(r) if n else torch.empty(16, dtype=torch.uint8, device="cuda") for r in replicas]
    out = torch.empty(max(nbytes, 16), dtype=torch.uint8, device="cuda")
    nb = fv.n_blocks(nbytes)
    crc = torch.full((max(nb, 1),), -1, dtype=torch.int32, device="cuda")
    stats = torch.full((18,), 12345, dtype=torch.int64, device="cuda")
    d = fv.make_desc(devs, out, crc, stats, abs_tol, rel_tol, dtype=dtype, n=n)
    fv.check(fv.ft_vote(ctypes.byref(d), fv.stream_handle()), "ft_vote")
    torch.cuda.synchronize()
    s = fv.parse_stats(stats, len(replicas))
    return {"out": out[:nbytes].cpu().numpy().view(oracle.NP_OF[dtype]),
            "block_crc": crc[:nb].cpu().numpy().view(np.uint32),
            "mismatch": np.array(s["mismatch"], dtype=np.uint64),
            "first_mismatch": np.array(s["first_mismatch"], dtype=np.int64),
            "no_majority": s["no_majority"], "first_no_majority": s["first_no_majority"],
            "raw_stats": stats.cpu().numpy()}


def assert_same(gpu, ref, R):
    assert gpu["out"].tobytes() == ref["out"].tobytes(), _first_diff(gpu["out"], ref["out"])
    assert np.array_equal(gpu["block_crc"], ref["block_crc"]), \
        f"crc differs at blocks {np.flatnonzero(gpu['block_crc'] != ref['block_crc'])[:8]}"
    assert list(gpu["mismatch"]) == list(ref["mismatch"])
    assert list(gpu["first_mismatch"]) == list(ref["first_mismatch"])
    assert gpu["no_majority"] == ref["no_majority"]
    assert gpu["first_no_majority"] == ref["first_no_majority"]
    raw = gpu["raw_stats"]
    # entries beyond R are reset to (0, -1)
    assert all(raw[r] == 0 for r in range(R, 8)) and all(raw[8 + r] == -1 for r in range(R, 8))


def _first_diff(a, b):
    ab, bb = a.view(np.uint8), b.view(np.uint8)
    if ab.size != bb.size:
        return f"size {ab.size} vs {bb.size}"
    d = np.flatnonzero(ab != bb)
    return f"{d.size} bytes differ, first at byte {d[0] if d.size else None}"


class DevTask:
    """One vote task's device buffers, built from host replicas."""

    def __init__(self, prob):
        import torch
        from paper_1405_2912_b300 import ftvote as fv
        self.prob = prob
        n = prob.n
        nbytes = n * prob.itemsize
        self.nbytes = nbytes
        self.reps = [to_dev(r) if n else torch.empty(16, dtype=torch.uint8, device="cuda") for r in prob.replicas]
        self.out = torch.empty(max(nbytes, 16), dtype=torch.uint8, device="cuda")
        self.nb = fv.n_blocks(nbytes)
        self.crc = torch.full((max(self.nb, 1),), -1, dtype=torch.int32, device="cuda")
        self.stats = torch.full((18,), 777, dtype=torch.int64, device="cuda")
        self.desc = fv.make_desc(self.reps, self.out, self.crc, self.stats, prob.abs_tol, prob.rel_tol,
                                 dtype=prob.dtype, n=n)

    def result(self):
        from paper_1405_2912_b300 import ftvote as fv
        s = fv.parse_stats(self.stats, self.prob.R)
        t = oracle.NP_OF[self.prob.dtype]
        return {"out": self.out[:self.nbytes].cpu().numpy().view(t),
                "block_crc": self.crc[:self.nb].cpu().numpy().view(np.uint32),
                "mismatch": np.array(s["mismatch"], dtype=np.uint64),
                "first_mismatch": np.array(s["first_mismatch"], dtype=np.int64),
                "no_majority": s["no_majority"], "first_no_majority": s["first_no_majority"],
                "raw_stats": self.stats.cpu().numpy()}


def desc_array(tasks):
    from paper_1405_2912_b300 import ftvote as fv
    arr = (fv.ft_vote_desc * max(1, len(tasks)))()
    for i, t in enumerate(tasks):
        arr[i] = t.desc
    return arr
