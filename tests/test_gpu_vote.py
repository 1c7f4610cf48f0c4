"""GPU parity of ft_vote (the CUDA voter, called through the C ABI) against the
CPU oracle, element by element and bit-exactly: voted values, per-4-KiB-block
CRC32C, per-replica mismatch counts and first indices, no-majority count and
first index.  Sizes span many 4 KiB blocks and ragged tails; the workloads are
the seeded generators of the five voter workloads, scaled down, plus the full
256M-element f32 workload in the launch configuration that bench.py times."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1405_2912_b300 import synth

from _gpu import assert_same, gpu_vote

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 5, 31, 1023, 1024, 1025, 2048 + 3, 4097, 12345, 65536 + 77, 300_001]


def _special(dtype, rng, n):
    if dtype == "f32":
        pool = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 3.4e38, -3.4e38, 1.0,
                         1.0000001, 0.9999999], dtype=np.float32)
    else:
        pool = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, 1.7e308, 1.0, 1.0 + 2e-16],
                        dtype=np.float64)
    return pool[rng.integers(0, pool.size, size=n)]


def _random_problem(dtype, R, n, seed):
    """Replicas with ULP noise, bit flips, specials and tie patterns."""
    rng = np.random.default_rng(seed)
    t = oracle.NP_OF[dtype]
    if dtype in ("f32", "f64"):
        base = synth.lognormal(rng, n, dtype)
        sp = rng.random(n) < 0.02
        base[sp] = _special(dtype, rng, int(sp.sum()))
        tol = synth.TOL[dtype]
    else:
        info = np.iinfo(t)
        base = rng.integers(info.min, info.max, size=n, dtype=t, endpoint=True)
        tol = (0.0, 0.0)
    reps = [base.copy() for _ in range(R)]
    for r in range(R):
        if dtype in ("f32", "f64") and n:
            idx = np.flatnonzero(rng.random(n) < 0.1)
            synth.ulp_perturb(reps[r], idx, rng.integers(1, 6, size=idx.size))
        idx = np.flatnonzero(rng.random(n) < 0.03)
        synth.bit_flip(reps[r], idx, rng.integers(0, 8 * reps[r].dtype.itemsize, size=idx.size))
        # occasional whole-element replacement from another replica: ties and clusters
        idx = np.flatnonzero(rng.random(n) < 0.05)
        src = reps[int(rng.integers(0, R))]
        reps[r][idx] = src[idx]
    return reps, tol


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32", "u32", "i64", "u64", "u8"])
@pytest.mark.parametrize("R", [2, 3, 4, 5, 6, 7, 8])
def test_random_all_types(dtype, R):
    for k, n in enumerate(SIZES if R in (3, 5) else SIZES[::3]):
        reps, tol = _random_problem(dtype, R, n, seed=1000 * R + k)
        ref = oracle.vote(reps, dtype, *tol)
        got = gpu_vote(reps, dtype, *tol)
        assert_same(got, ref, R)


def test_empty_vote_resets_stats():
    reps = [np.zeros(0, dtype=np.float32)] * 3
    got = gpu_vote(reps, "f32", 1e-6, 1e-5)
    assert list(got["mismatch"]) == [0, 0, 0]
    assert list(got["first_mismatch"]) == [-1, -1, -1]
    assert got["no_majority"] == 0 and got["first_no_majority"] == -1


def test_cfg1_full():
    p = synth.cfg1()
    assert_same(gpu_vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol),
                oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol), p.R)


def test_cfg2_scaled_ragged():
    p = synth.cfg2(n=(1 << 22) + 37, flip_rate=1e-4)
    assert_same(gpu_vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol),
                oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol), p.R)


def test_cfg3_scaled_ties():
    for p in synth.cfg3(n=(1 << 18) + 5, block=1 << 12, ties=256):
        ref = oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol)
        assert ref["no_majority"] >= 256
        assert_same(gpu_vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol), ref, p.R)


def test_nontransitive_and_paper_delta():
    # A~B, B~C, A!~C under rel 2^-10; and the paper's 0.1% delta for f32
    a = np.array([1024.0, 1024.0, 1026.0, 1.0, 1.0], dtype=np.float32)
    b = np.array([1025.0, 1026.0, 1024.0, 1.0009, 1.002], dtype=np.float32)
    c = np.array([1026.0, 1025.0, 1025.0, 0.9995, 1.0], dtype=np.float32)
    for rel in (2.0 ** -10, 1e-3):
        assert_same(gpu_vote([a, b, c], "f32", 0.0, rel), oracle.vote([a, b, c], "f32", 0.0, rel), 3)


def test_cfg2_full_size():
    """The 256M-element f32 workload at full size, in the bench's launch
    configuration, against the whole oracle run."""
    p = synth.cfg2()
    ref = oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol)
    got = gpu_vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol)
    assert_same(got, ref, p.R)
    # the flips that are real faults are all found in replica 2
    assert got["mismatch"][2] > 0 and got["mismatch"][0] == 0


def test_cfg3_full_size():
    for p in synth.cfg3():
        ref = oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol)
        got = gpu_vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol)
        assert_same(got, ref, p.R)
        assert got["mismatch"][3] >= (1 << 20) - 1024


def test_vote_captured_in_a_user_graph():
    """ft_vote (after one ordinary call has set up its kernel) can be recorded
    into a caller's CUDA graph; replays vote the current contents of the
    buffers, and equal the oracle."""
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    p = synth.cfg1(n=(1 << 18) + 11, flips=40)
    dev = [torch.from_numpy(r).cuda() for r in p.replicas]
    out, crc, st = fv.vote(dev, p.abs_tol, p.rel_tol)          # warm-up call outside the capture
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        fv.vote(dev, p.abs_tol, p.rel_tol, out=out, block_crc=crc, stats=st, stream=s)
    for k in range(2):
        # new contents between replays: replica 0 takes the flips of replica 2 on the second replay
        host = [r.copy() for r in p.replicas]
        if k == 1:
            host[0] = host[2].copy()
            for r, h in zip(dev, host):
                r.copy_(torch.from_numpy(h))
        out.zero_()
        st.fill_(7)
        g.replay()
        torch.cuda.synchronize()
        ref = oracle.vote(host, "f32", p.abs_tol, p.rel_tol)
        assert out.cpu().numpy().tobytes() == ref["out"].tobytes()
        assert np.array_equal(crc.cpu().numpy().view(np.uint32), ref["block_crc"])
        s_ = fv.parse_stats(st, 3)
        assert s_["mismatch"] == [int(x) for x in ref["mismatch"]]
        assert s_["no_majority"] == ref["no_majority"]


@pytest.mark.parametrize("dtype,R", [("f32", 3), ("f64", 5), ("i32", 3), ("u8", 4)])
def test_vote_without_digest(dtype, R):
    """block_crc = NULL: no digest is written; everything else is unchanged.
    (The kernel still digests each block: skipping the CRC measured slower,
    6.45 against 6.71 TB/s on 3 x 256M f32, as the digest paces the warps'
    L2 prefetch.)"""
    import ctypes
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    from _gpu import DevTask
    for n in (1, 4095, 70_001):
        reps, tol = _random_problem(dtype, R, n, seed=77 + n)
        p = synth.Problem(reps, dtype, *tol)
        t = DevTask(p)
        t.desc.block_crc = None
        t.crc.fill_(-5)
        fv.check(fv.ft_vote(ctypes.byref(t.desc), fv.stream_handle()), "ft_vote")
        torch.cuda.synchronize()
        got = t.result()
        assert np.all(got["block_crc"] == np.uint32(0xFFFFFFFB))        # untouched
        ref = oracle.vote(reps, dtype, *tol)
        got["block_crc"] = ref["block_crc"]
        assert_same(got, ref, R)


# Positions on a line, in units of h = 0.75 * abs_tol, for each pattern of
# (x0 != x1, x0 != x2, x1 != x2) under an absolute tolerance: neighbours one
# h apart are equal, two h apart are not.  The three patterns with exactly one
# unequal pair are the non-transitive ones.
_PATTERN_POS = {(0, 0, 0): (0, 0, 0), (1, 0, 0): (0, 2, 1), (0, 1, 0): (0, 1, 2), (0, 0, 1): (1, 0, 2),
                (1, 1, 0): (0, 10, 10), (1, 0, 1): (0, 10, 0), (0, 1, 1): (0, 0, 10), (1, 1, 1): (0, 10, 20)}


def _dense_r3(dtype, n, seed):
    """R = 3 replicas in which every element takes one of the eight pair
    patterns at random (floats), or one of the five that bitwise equality
    allows (integers), so most elements carry a mismatch or lack a majority."""
    rng = np.random.default_rng(seed)
    t = oracle.NP_OF[dtype]
    if dtype in ("f32", "f64"):
        abs_tol = 1e-3
        pats = list(_PATTERN_POS)
        pos = np.array([_PATTERN_POS[p] for p in pats], dtype=t)[rng.integers(0, len(pats), size=n)]
        base = (rng.integers(-50, 50, size=n) * 100).astype(t) * t(abs_tol)
        reps = [base + pos[:, r] * t(0.75 * abs_tol) for r in range(3)]
        return [np.ascontiguousarray(x, dtype=t) for x in reps], (abs_tol, 0.0)
    info = np.iinfo(t)
    vals = [rng.integers(info.min, info.max, size=n, dtype=t, endpoint=True) for _ in range(3)]
    which = rng.integers(0, 5, size=n)              # 0: all equal, 1..3: replica which-1 differs, 4: all differ
    reps = [vals[0].copy() for _ in range(3)]
    for r in range(3):
        sel = (which == r + 1) | ((which == 4) & (r > 0))
        reps[r][sel] = vals[r][sel] if r > 0 else vals[1][sel]
    return reps, (0.0, 0.0)


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32", "u8", "i64"])
def test_dense_disagreement_r3(dtype):
    """Mismatches and missing majorities at most elements (every pattern of the
    three pairwise comparisons, non-transitive ones included): the statistics
    of the R = 3 closed form's rare path, across several blocks and a tail."""
    for k, n in enumerate((7, 1025, 65536 + 13, 300_001)):
        reps, tol = _dense_r3(dtype, n, seed=500 + k)
        ref = oracle.vote(reps, dtype, *tol)
        if n > 1000:
            assert ref["no_majority"] > 0 and min(ref["mismatch"]) > 0
        assert_same(gpu_vote(reps, dtype, *tol), ref, 3)


@pytest.mark.parametrize("dtype,R", [("f32", 3), ("f32", 5), ("f64", 3), ("i32", 3), ("i32", 5), ("u8", 3)])
def test_one_replica_wrong_everywhere(dtype, R):
    """Replica 1 disagrees with the others at every element (a unit that
    returns garbage): every element is a mismatch of replica 1."""
    rng = np.random.default_rng(R)
    n = 4096 * 37 + 5
    reps, tol = _random_problem(dtype, R, n, seed=9 + R)
    reps = [np.ascontiguousarray(reps[0]) for _ in range(R)]
    bad = reps[1].view(np.uint8).copy()
    bad ^= rng.integers(1, 256, size=bad.size, dtype=np.uint8) | np.uint8(0x80) if dtype == "u8" else \
        np.tile(np.array([0, 0, 0, 0x40] if reps[1].dtype.itemsize == 4 else [0] * 7 + [0x40], dtype=np.uint8), n)
    reps[1] = bad.view(reps[0].dtype)
    ref = oracle.vote(reps, dtype, *tol)
    assert int(ref["mismatch"][1]) == n
    assert_same(gpu_vote(reps, dtype, *tol), ref, R)


def _dense_any_r(dtype, R, n, seed):
    """R replicas whose elements sit at positions {0, 1, 2, 10, 20} x h on a
    line (floats, h = 0.75 * abs_tol: one step apart equal, two apart not),
    or take one of three values (integers): clusters, ties and non-transitive
    chains at most elements."""
    rng = np.random.default_rng(seed)
    t = oracle.NP_OF[dtype]
    if dtype in ("f32", "f64"):
        abs_tol = 1e-3
        base = (rng.integers(-50, 50, size=n) * 100).astype(t) * t(abs_tol)
        steps = np.array([0, 1, 2, 10, 20], dtype=t)
        reps = [base + steps[rng.integers(0, 5, size=n)] * t(0.75 * abs_tol) for _ in range(R)]
        return [np.ascontiguousarray(x, dtype=t) for x in reps], (abs_tol, 0.0)
    info = np.iinfo(t)
    alphabet = np.stack([rng.integers(info.min, info.max, size=n, dtype=t, endpoint=True) for _ in range(3)])
    return [np.ascontiguousarray(alphabet[rng.integers(0, 3, size=n), np.arange(n)]) for _ in range(R)], (0.0, 0.0)


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32", "u8"])
@pytest.mark.parametrize("R", [2, 4, 5, 8])
def test_dense_disagreement_other_r(dtype, R):
    """As above for R = 2 (replica 0 always wins) and R >= 4 (the float form
    that re-votes a flagged sub-batch, the bits-first form of the others)."""
    for k, n in enumerate((9, 4096 + 100, 100_003)):
        reps, tol = _dense_any_r(dtype, R, n, seed=900 + 10 * R + k)
        ref = oracle.vote(reps, dtype, *tol)
        if n > 1000:
            assert ref["no_majority"] > 0 and max(ref["mismatch"]) > 0
        assert_same(gpu_vote(reps, dtype, *tol), ref, R)


def test_more_votes_in_flight_than_statistics_slots():
    """ft_vote gathers a vote's statistics in one of 1024 library slots per
    device and falls back to a statistics reset kernel when all are taken.
    With four streams each held by a sleeping kernel, 1400 votes are queued
    behind them (more than 1024 in flight at once), each into its own
    statistics buffer: some take the fallback, every one equals the oracle,
    and once they are done the slots serve new votes again."""
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    p = synth.cfg1(n=5000, flips=20)
    ref = oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol)
    dev = [torch.from_numpy(r).cuda() for r in p.replicas]
    nstreams, per = 4, 350
    k = nstreams * per
    outs = [torch.empty_like(dev[0]) for _ in range(nstreams)]
    crcs = [torch.empty(fv.n_blocks(4 * p.n), dtype=torch.int32, device="cuda") for _ in range(nstreams)]
    stats = torch.full((k, 18), 7, dtype=torch.int64, device="cuda")
    streams = [torch.cuda.Stream() for _ in range(nstreams)]
    descs = [fv.make_desc(dev, outs[j], crcs[j], stats[0], p.abs_tol, p.rel_tol) for j in range(nstreams)]
    fv.check(fv.ft_vote(ctypes.byref(descs[0]), fv.stream_handle(streams[0])), "ft_vote")   # sets up the pool
    torch.cuda.synchronize()
    for st_ in streams:
        with torch.cuda.stream(st_):
            torch.cuda._sleep(400_000_000)
    l0 = fv.ft_launch_count()
    for i in range(k):
        j = i % nstreams
        descs[j].stats = stats[i].data_ptr()
        fv.check(fv.ft_vote(ctypes.byref(descs[j]), fv.stream_handle(streams[j])), "ft_vote")
    # a vote through a slot is one launch, one past the pool two (reset and voter)
    fell_back = fv.ft_launch_count() - l0 - k
    torch.cuda.synchronize()
    want = ([int(x) for x in ref["mismatch"]] + [0] * 5 + [int(x) for x in ref["first_mismatch"]] + [-1] * 5 +
            [ref["no_majority"], ref["first_no_majority"]])
    got = stats.cpu().numpy()
    bad = [i for i in range(k) if list(got[i]) != want]
    assert not bad, (len(bad), bad[:5])
    for j in range(nstreams):
        assert outs[j].cpu().numpy().tobytes() == ref["out"].tobytes()
        assert np.array_equal(crcs[j].cpu().numpy().view(np.uint32), ref["block_crc"])
    assert fell_back > 0, fell_back
    stats.fill_(7)
    for i in range(50):
        descs[0].stats = stats[i].data_ptr()
        fv.check(fv.ft_vote(ctypes.byref(descs[0]), fv.stream_handle(streams[0])), "ft_vote")
    torch.cuda.synchronize()
    got = stats[:50].cpu().numpy()
    assert all(list(got[i]) == want for i in range(50))
