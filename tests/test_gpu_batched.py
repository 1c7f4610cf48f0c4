"""GPU parity of the batched form (ft_plan_create / ft_vote_batched): every task
of a mixed batch (element types, R, sizes including empty and ragged) gets the
same bit-exact results as the oracle and as ft_vote alone, with the autotuned
and with fixed tile sizes and launch shapes (8, 12 and 16 warps per CTA, with
and without the L2 prefetch), through the captured graph and without it, and
again on a second replay."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1405_2912_b300 import synth

from _gpu import DevTask, assert_same, desc_array

pytestmark = pytest.mark.gpu


def _mixed_specs(k=48, seed=9):
    rng = np.random.default_rng(seed)
    specs = []
    dts = ["f32", "f64", "i32", "u8", "i64", "u32"]
    sizes = [0, 1, 7, 1024, 1025, 4096, 5000, 40_000, 70_001]
    for i in range(k):
        specs.append(synth.TaskSpec(int(sizes[i % len(sizes)] + rng.integers(0, 3) * (i % 2)),
                                    dts[i % len(dts)], int(2 + (i % 7)), bool(i % 3 == 0), 500 + i))
    return specs


def _run(tasks, tune=None, graph=True, reps=1):
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    arr = desc_array(tasks)
    plan = ctypes.c_void_p()
    t = None
    if tune is not None:
        t = fv.ft_tune(*tune)
    fv.check(fv.ft_plan_create(ctypes.byref(plan), arr, len(tasks), ctypes.byref(t) if t else None),
             "ft_plan_create")
    try:
        for _ in range(reps):
            for tk in tasks:     # scribble the outputs so that a stale result cannot pass
                tk.out.fill_(0x5A)
                tk.crc.fill_(-1)
                tk.stats.fill_(999)
            f = fv.ft_vote_batched if graph else fv.ft_vote_batched_nograph
            fv.check(f(plan, fv.stream_handle()), "batched")
            torch.cuda.synchronize()
        chosen = fv.ft_tune()
        fv.ft_plan_tune(plan, ctypes.byref(chosen))
        n = ctypes.c_int32()
        fv.check(fv.ft_plan_groups(plan, None, 0, ctypes.byref(n)), "ft_plan_groups")
        groups = (fv.ft_plan_group * max(1, n.value))()
        fv.check(fv.ft_plan_groups(plan, groups, n.value, ctypes.byref(n)), "ft_plan_groups")
        return (chosen.tile_blocks, chosen.ctas_per_sm, chosen.warps, chosen.l2_prefetch, chosen.kernels), \
            list(groups)[:n.value]
    finally:
        fv.ft_plan_destroy(plan)


@pytest.mark.parametrize("tune,graph", [(None, True), ((1, 1), True), ((3, 0), False), ((64, 1), True),
                                        ((4, 0, 8, 2), True), ((2, 0, 12, 1), True), ((0, 0, 16, 2), False),
                                        ((5, 0, 8, 1), False), ((7, 0, 12, 2), True), ((1, 0, 16, 1), True),
                                        ((4, 0, 0, 0, 1), True), ((0, 0, 0, 0, 1), False), ((1, 0, 16, 1, 1), True),
                                        ((8, 0, 0, 0, 2), True), ((3, 0, 0, 0, 1), False)])
def test_mixed_batch_matches_oracle(tune, graph):
    from paper_1405_2912_b300 import ftvote as fv
    specs = _mixed_specs()
    probs = [synth.task_problem(s, ulp_frac=0.1, flip_rate=1e-3) for s in specs]
    tasks = [DevTask(p) for p in probs]
    chosen, groups = _run(tasks, tune, graph, reps=2)
    assert 1 <= chosen[0] <= 64
    if tune is not None and tune[0]:
        assert chosen[0] == tune[0]
    # the groups: sorted by element kind and R, every task in one, a built shape each
    assert sum(g.tasks for g in groups) == len(tasks)
    kinds = [(g.dtype, g.R) for g in groups]
    assert len(set(kinds)) == len(kinds)
    assert chosen[4] in (1, 2)
    if tune is not None and len(tune) > 4:
        assert chosen[4] == tune[4]
    for g in groups:
        assert g.warps in (8, 12, 16) and g.l2_prefetch in (0, 1) and g.tile_blocks == chosen[0]
        if tune is not None and len(tune) > 2 and (tune[2] or tune[3]):
            assert g.warps == (tune[2] or 16) and g.l2_prefetch == (1 if tune[3] == 2 else 0)
    if tune is not None and len(tune) > 2 and (tune[2] or tune[3]):
        assert chosen[2] == (tune[2] or 16) and chosen[3] == (2 if tune[3] == 2 else 1)
    for p, tk in zip(probs, tasks):
        assert_same(tk.result(), oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol), p.R)


def test_plan_rejects_bad_tune():
    from paper_1405_2912_b300 import ftvote as fv
    p = synth.task_problem(synth.TaskSpec(100, "f32", 3, False, 1))
    tk = DevTask(p)
    plan = ctypes.c_void_p()
    for bad in ((65, 0, 0, 0), (1, 9, 0, 0), (1, 0, 10, 0), (1, 0, 0, 3), (1, 0, -1, 0), (1, 0, 0, 0, 3),
                (1, 0, 8, 0, 1), (1, 0, 0, 2, 1)):
        t = fv.ft_tune(*bad)
        assert fv.ft_plan_create(ctypes.byref(plan), desc_array([tk]), 1, ctypes.byref(t)) == fv.FT_EINVAL, bad


def test_batched_equals_single_votes_cfg4_scaled():
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    specs = synth.cfg4_specs(ntasks=256, hi=1 << 18)
    probs = [synth.task_problem(s) for s in specs]
    tasks = [DevTask(p) for p in probs]
    _run(tasks)
    got = [tk.result() for tk in tasks]
    for tk in tasks:
        fv.check(fv.ft_vote(ctypes.byref(tk.desc), fv.stream_handle()), "ft_vote")
    torch.cuda.synchronize()
    for p, g, tk in zip(probs, got, tasks):
        assert_same(g, tk.result(), p.R)
    for i in range(0, len(probs), 17):
        p = probs[i]
        assert_same(got[i], oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol), p.R)


def test_vote_many_matches():
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    specs = _mixed_specs(k=20, seed=3)
    probs = [synth.task_problem(s, flip_rate=1e-3) for s in specs]
    tasks = [DevTask(p) for p in probs]
    fv.check(fv.ft_vote_many(desc_array(tasks), len(tasks), fv.stream_handle()), "ft_vote_many")
    torch.cuda.synchronize()
    for p, tk in zip(probs, tasks):
        assert_same(tk.result(), oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol), p.R)


def test_plan_rejects_bad_task():
    from paper_1405_2912_b300 import ftvote as fv
    p = synth.task_problem(synth.TaskSpec(100, "f32", 3, False, 1))
    tk = DevTask(p)
    tk.desc.R = 9
    plan = ctypes.c_void_p()
    assert fv.ft_plan_create(ctypes.byref(plan), desc_array([tk]), 1, None) == fv.FT_EINVAL
