"""ft_vote_batched_noalloc: the batched vote for callers that cannot allocate
device memory (its scratch is a fixed device array inside the library).  Its
results must equal those of ft_vote, task by task and bit for bit, and those
of the oracle, on two calls in a row (the second call reuses the scratch left
by the first).  Empty batches and batches of empty tasks return FT_OK and
leave each task's statistics at their initial values; a stream that is being
captured into a graph is refused.  This file is collected last so that a
failure here comes after every other test."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1405_2912_b300 import synth

from _gpu import DevTask, assert_same, desc_array

pytestmark = pytest.mark.gpu


def _batch(seed, k):
    rng = np.random.default_rng(seed)
    dts = ["f32", "f64", "i32", "u8", "i64"]
    sizes = [0, 1, 5, 1023, 4096, 4099, 20_000, 65_537, 150_000]
    specs = [synth.TaskSpec(int(sizes[int(rng.integers(0, len(sizes)))]), dts[i % len(dts)],
                            int(rng.integers(2, 9)), bool(i % 2), seed * 1000 + i) for i in range(k)]
    return [synth.task_problem(s, config_id=6, ulp_frac=0.1, flip_rate=1e-3) for s in specs]


def test_noalloc_matches_ft_vote_and_oracle_twice():
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    for call, (seed, k, tile) in enumerate([(1, 40, 0), (2, 29, 3), (3, 33, 0)]):
        probs = _batch(seed, k)
        ref_tasks = [DevTask(p) for p in probs]
        for t in ref_tasks:
            fv.check(fv.ft_vote(ctypes.byref(t.desc), fv.stream_handle()), "ft_vote")
        tasks = [DevTask(p) for p in probs]
        rc = fv.ft_vote_batched_noalloc(desc_array(tasks), len(tasks), tile, fv.stream_handle())
        assert rc == fv.FT_OK, (call, rc)
        torch.cuda.synchronize()
        for p, a, b in zip(probs, tasks, ref_tasks):
            got = a.result()
            assert_same(got, b.result(), p.R)
            assert_same(got, oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol), p.R)


def test_noalloc_empty_batches():
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    # no task at all: nothing to do
    assert fv.ft_vote_batched_noalloc(None, 0, 0, fv.stream_handle()) == fv.FT_OK
    # only empty tasks (several groups): FT_OK and initial statistics
    specs = [synth.TaskSpec(0, dt, R, False, 900 + i) for i, (dt, R) in
             enumerate([("f32", 3), ("f64", 5), ("i32", 2), ("u8", 8), ("f32", 3)])]
    tasks = [DevTask(synth.task_problem(s, config_id=6)) for s in specs]
    for tile in (0, 4):
        for t in tasks:
            t.stats.fill_(555)
        rc = fv.ft_vote_batched_noalloc(desc_array(tasks), len(tasks), tile, fv.stream_handle())
        assert rc == fv.FT_OK
        torch.cuda.synchronize()
        for t in tasks:
            raw = t.stats.cpu().numpy()
            assert (raw[:8] == 0).all() and (raw[8:16] == -1).all() and raw[16] == 0 and raw[17] == -1


def test_noalloc_refuses_a_capturing_stream():
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    p = synth.task_problem(synth.TaskSpec(5000, "f32", 3, True, 7), config_id=6)
    t = DevTask(p)
    s = torch.cuda.Stream()
    # an ordinary call first (on a fresh process this one looks up the array)
    fv.check(fv.ft_vote_batched_noalloc(desc_array([t]), 1, 0, fv.stream_handle(s)), "noalloc")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        rc = fv.ft_vote_batched_noalloc(desc_array([t]), 1, 0, fv.stream_handle(s))
    assert rc == fv.FT_EINVAL
    # the refusal leaves nothing behind: a later ordinary call still votes
    t.stats.fill_(3)
    fv.check(fv.ft_vote_batched_noalloc(desc_array([t]), 1, 0, fv.stream_handle(s)), "noalloc")
    torch.cuda.synchronize()
    assert_same(t.result(), oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol), p.R)


def test_noalloc_rejects_too_many_tasks():
    from paper_1405_2912_b300 import ftvote as fv
    p = synth.task_problem(synth.TaskSpec(100, "f32", 3, False, 5))
    t = DevTask(p)
    n = fv.FT_NOALLOC_MAX_TASKS + 1
    arr = (fv.ft_vote_desc * n)()
    for i in range(n):
        arr[i] = t.desc
    assert fv.ft_vote_batched_noalloc(arr, n, 0, fv.stream_handle()) == fv.FT_EINVAL
    assert fv.ft_vote_batched_noalloc(arr, 1, 65, fv.stream_handle()) == fv.FT_EINVAL
