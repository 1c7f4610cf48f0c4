"""ft_vote_host: the vote on host buffers, streamed through the device in
chunks.  Voted bytes, digests and statistics equal the oracle's on the same
replicas, for votes spanning many chunks with a ragged last chunk and block,
with pageable and with pinned host memory; n = 0 resets the statistics."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1405_2912_b300 import synth

pytestmark = pytest.mark.gpu


def _host_vote(reps, dtype, tol, chunk, pinned):
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    n = reps[0].size
    np_t = oracle.NP_OF[dtype]
    nb = n * np.dtype(np_t).itemsize
    if pinned:
        hreps = [torch.from_numpy(np.ascontiguousarray(r).view(np.uint8).copy()).pin_memory() for r in reps]
        out = torch.empty(max(nb, 16), dtype=torch.uint8).pin_memory()
        crc = torch.empty(max(fv.n_blocks(nb), 1), dtype=torch.int32).pin_memory()
        rp, op, cp = [t.data_ptr() for t in hreps], out.data_ptr(), crc.data_ptr()
        keep = (hreps, out, crc)
    else:
        hreps = [np.ascontiguousarray(r).copy() for r in reps]
        out = np.empty(max(nb, 16), dtype=np.uint8)
        crc = np.empty(max(fv.n_blocks(nb), 1), dtype=np.uint32)
        rp, op, cp = [a.ctypes.data for a in hreps], out.ctypes.data, crc.ctypes.data
        keep = (hreps, out, crc)
    st = fv.ft_stats()
    d = fv.ft_vote_desc()
    for r, p in enumerate(rp):
        d.replicas[r] = p
    d.R, d.dtype, d.n = len(reps), fv.DTYPE[dtype], n
    d.abs_tol, d.rel_tol = tol
    d.out, d.block_crc, d.stats = op, cp, ctypes.addressof(st)
    fv.check(fv.ft_vote_host(ctypes.byref(d), chunk), "ft_vote_host")
    o = (out.numpy() if pinned else out)[:nb].view(np_t)
    c = (crc.numpy().view(np.uint32) if pinned else crc)[:fv.n_blocks(nb)]
    R = len(reps)
    return {"out": o.copy(), "block_crc": c.copy(), "mismatch": list(st.mismatch)[:R],
            "first_mismatch": list(st.first_mismatch)[:R], "no_majority": st.no_majority,
            "first_no_majority": st.first_no_majority, "keep": keep}


def _check(got, ref):
    assert got["out"].tobytes() == ref["out"].tobytes()
    assert np.array_equal(got["block_crc"], ref["block_crc"])
    assert [int(x) for x in got["mismatch"]] == [int(x) for x in ref["mismatch"]]
    assert [int(x) for x in got["first_mismatch"]] == [int(x) for x in ref["first_mismatch"]]
    assert int(got["no_majority"]) == int(ref["no_majority"])
    assert int(got["first_no_majority"]) == int(ref["first_no_majority"])


@pytest.mark.parametrize("dtype,R,pinned", [("f32", 3, True), ("f64", 5, False), ("i32", 2, True), ("u8", 4, False)])
def test_many_chunks_ragged(dtype, R, pinned):
    rng = np.random.default_rng(R)
    t = oracle.NP_OF[dtype]
    n = (3 * 8192) // np.dtype(t).itemsize * 7 + 1029          # 7 chunks of 3 blocks, a ragged eighth
    if dtype in ("f32", "f64"):
        base = synth.lognormal(rng, n, dtype)
        tol = synth.TOL[dtype]
    else:
        info = np.iinfo(t)
        base = rng.integers(info.min, info.max, size=n, dtype=t, endpoint=True)
        tol = (0.0, 0.0)
    reps = [base.copy() for _ in range(R)]
    for r in range(R):
        idx = np.flatnonzero(rng.random(n) < 0.01)
        synth.bit_flip(reps[r], idx, rng.integers(0, 8 * reps[r].dtype.itemsize, size=idx.size))
    # faults only in later chunks for one replica: its first index comes from a later chunk
    late = n - 5000
    reps[R - 1][:late] = reps[0][:late]
    ref = oracle.vote(reps, dtype, *tol)
    _check(_host_vote(reps, dtype, tol, 3 * 8192, pinned), ref)


def test_default_chunk_large_pinned():
    p = synth.cfg1(n=40_000_000)                      # 160 MB per replica: three 64 MiB chunks
    ref = oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol)
    _check(_host_vote(p.replicas, p.dtype, (p.abs_tol, p.rel_tol), 0, True), ref)


def test_empty_and_bad_chunk():
    from paper_1405_2912_b300 import ftvote as fv
    reps = [np.zeros(0, dtype=np.float32) for _ in range(3)]
    got = _host_vote(reps, "f32", (1e-6, 1e-5), 0, False)
    assert [int(x) for x in got["mismatch"]] == [0, 0, 0] and int(got["first_no_majority"]) == -1
    a = np.zeros(1024, dtype=np.float32)
    st = fv.ft_stats()
    d = fv.ft_vote_desc()
    for r in range(3):
        d.replicas[r] = a.ctypes.data
    d.R, d.dtype, d.n = 3, fv.DTYPE["f32"], a.size
    o = np.empty_like(a)
    d.out, d.stats = o.ctypes.data, ctypes.addressof(st)
    assert fv.ft_vote_host(ctypes.byref(d), 1000) == fv.FT_EINVAL        # not a multiple of 4096


def _mixed_vote(reps, dtype, tol, chunk, where):
    """ft_vote_host with each buffer placed as `where` says: a dict of
    'rep0'..'repR-1', 'out', 'crc', 'stats' -> 'dev' | 'pinned' | 'pageable'
    ('crc' may also be None: no digests)."""
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    n = reps[0].size
    np_t = oracle.NP_OF[dtype]
    nb = n * np.dtype(np_t).itemsize
    nblk = max(fv.n_blocks(nb), 1)

    def place(arr_u8, kind):
        t = torch.from_numpy(arr_u8.copy())
        if kind == "dev":
            t = t.cuda()
        elif kind == "pinned":
            t = t.pin_memory()
        return t

    keep = []
    rp = []
    for r, a in enumerate(reps):
        t = place(np.ascontiguousarray(a).view(np.uint8), where[f"rep{r}"])
        keep.append(t)
        rp.append(t.data_ptr())
    out = place(np.zeros(max(nb, 16), dtype=np.uint8), where["out"])
    crc = place(np.zeros(4 * nblk, dtype=np.uint8), where["crc"]) if where["crc"] else None
    st = place(np.zeros(ctypes.sizeof(fv.ft_stats), dtype=np.uint8), where["stats"])
    keep += [out, st] + ([crc] if crc is not None else [])
    torch.cuda.synchronize()                        # device inputs complete before the call
    d = fv.ft_vote_desc()
    for r, p in enumerate(rp):
        d.replicas[r] = p
    d.R, d.dtype, d.n = len(reps), fv.DTYPE[dtype], n
    d.abs_tol, d.rel_tol = tol
    d.out, d.block_crc, d.stats = out.data_ptr(), (crc.data_ptr() if crc is not None else None), st.data_ptr()
    fv.check(fv.ft_vote_host(ctypes.byref(d), chunk), "ft_vote_host")
    s = fv.ft_stats.from_buffer_copy(st.cpu().numpy().tobytes())
    R = len(reps)
    return {"out": out.cpu().numpy()[:nb].view(np_t).copy(),
            "block_crc": (crc.cpu().numpy().view(np.uint32)[:fv.n_blocks(nb)].copy() if crc is not None else None),
            "mismatch": list(s.mismatch)[:R], "first_mismatch": list(s.first_mismatch)[:R],
            "no_majority": s.no_majority, "first_no_majority": s.first_no_majority}


@pytest.mark.parametrize("where", [
    # a device-resident replica beside host ones, the voted bytes left on the device
    {"rep0": "dev", "rep1": "pinned", "rep2": "pageable", "out": "dev", "crc": "pinned", "stats": "dev"},
    # every replica on the device, the result brought to the host
    {"rep0": "dev", "rep1": "dev", "rep2": "dev", "out": "pinned", "crc": "dev", "stats": "pageable"},
    # host replicas, device outputs
    {"rep0": "pinned", "rep1": "pinned", "rep2": "pinned", "out": "dev", "crc": "dev", "stats": "pinned"},
    # no digests, the output on the host
    {"rep0": "dev", "rep1": "pageable", "rep2": "dev", "out": "pageable", "crc": None, "stats": "dev"},
])
def test_mixed_residency(where):
    rng = np.random.default_rng(11)
    n = (2 * 8192) // 4 * 5 + 777                  # five chunks of two blocks and a ragged sixth
    base = synth.lognormal(rng, n, "f32")
    reps = [base.copy() for _ in range(3)]
    for r in range(3):
        idx = np.flatnonzero(rng.random(n) < 0.02)
        synth.bit_flip(reps[r], idx, rng.integers(0, 32, size=idx.size))
    tol = synth.TOL["f32"]
    ref = oracle.vote(reps, "f32", *tol)
    got = _mixed_vote(reps, "f32", tol, 2 * 8192, where)
    if where["crc"] is None:
        got["block_crc"] = ref["block_crc"]       # none asked for
    _check(got, ref)


def test_mixed_residency_empty_device_stats():
    where = {"rep0": "dev", "rep1": "pinned", "rep2": "dev", "out": "dev", "crc": "dev", "stats": "dev"}
    reps = [np.zeros(0, dtype=np.float32) for _ in range(3)]
    got = _mixed_vote(reps, "f32", (1e-6, 1e-5), 0, where)
    assert [int(x) for x in got["mismatch"]] == [0, 0, 0]
    assert [int(x) for x in got["first_mismatch"]] == [-1, -1, -1] and int(got["first_no_majority"]) == -1
