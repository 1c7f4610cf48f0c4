"""The server's resident mode (ft_server_config.resident = 1): one persistent
voter kernel takes every request from a host-mapped mailbox, with no launch
per request.  Each result is bit-identical to the same vote alone through
ft_vote and to the oracle, for every element type and R = 2..8, ragged and
empty requests included; requests beyond the 32 device slots wait on the
host; a caller's statistics buffer is filled; a small request submitted
behind a large one completes first; the kernel leaves when idle and the next
request launches it again; destroying the server while a request is on the
device waits for it."""
import ctypes
import time

import numpy as np
import pytest

import oracle
from paper_1405_2912_b300 import synth

from _gpu import DevTask, assert_same

pytestmark = pytest.mark.gpu


def _resident(budget=1 << 34, idle_us=0, mode=1):
    from paper_1405_2912_b300 import ftvote as fv
    cfg = fv.ft_server_config(budget, 16, 1 if mode == 1 else 4, 0, 0)
    cfg.resident = mode
    cfg.idle_spin_us = idle_us
    srv = ctypes.c_void_p()
    fv.check(fv.ft_server_create(ctypes.byref(srv), ctypes.byref(cfg)), "ft_server_create")
    return srv


def _problems(seed=11):
    """Requests of every element type and R = 2..8: ragged sizes from one
    element to several tiles per warp, faults in some, one empty request."""
    rng = np.random.default_rng(seed)
    probs = []
    sizes = [1, 1023, 1024, 4096 + 3, 65_537, 300_001, 1 << 20]
    for i in range(54):
        dt = ["f32", "f64", "i32", "u8", "i64", "u32", "u64"][i % 7]
        R = 2 + (i % 7 + i // 7) % 7
        n = sizes[(i * 3) % len(sizes)] + int(rng.integers(0, 3))
        if dt in ("f32", "f64", "i32"):
            probs.append(synth.task_problem(synth.TaskSpec(n, dt, R, i % 3 == 0, 7000 + i), config_id=5,
                                            ulp_frac=0.05 if dt != "i32" else 0.0, flip_rate=1e-3))
        else:
            base = synth.uniform_int(rng, n, dt)
            reps = [base.copy() for _ in range(R)]
            if i % 3 == 0:
                idx = rng.choice(n, size=max(1, n // 500), replace=False)
                reps[int(rng.integers(0, R))][idx] ^= 1
            probs.append(synth.Problem(reps, dt))
    probs.append(synth.Problem([np.zeros(0, dtype=np.float32)] * 3, "f32", 1e-6, 1e-5))
    return probs


def _stats_dict(st, R):
    return {"mismatch": np.array(list(st.mismatch)[:R], dtype=np.uint64),
            "first_mismatch": np.array(list(st.first_mismatch)[:R], dtype=np.int64),
            "no_majority": int(st.no_majority), "first_no_majority": int(st.first_no_majority)}


def _submit(fv, srv, desc):
    tk = ctypes.c_uint64()
    fv.check(fv.ft_submit(srv, ctypes.byref(desc), ctypes.byref(tk)), "ft_submit")
    return tk.value


def _poll(fv, srv, tk):
    r = fv.ft_result()
    fv.check(fv.ft_poll(srv, tk, 30_000_000, ctypes.byref(r)), "ft_poll")
    assert r.status == fv.FT_OK
    return r


@pytest.mark.parametrize("mode", [1, 2])     # 2: small requests resident, the others batched
def test_resident_same_as_alone_and_oracle(mode):
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    probs = _problems()
    alone = [DevTask(p) for p in probs]
    for t in alone:
        fv.check(fv.ft_vote(ctypes.byref(t.desc), fv.stream_handle()), "ft_vote")
    torch.cuda.synchronize()
    alone_res = [t.result() for t in alone]
    mixed = [DevTask(p) for p in probs]
    srv = _resident(mode=mode)
    try:
        # all at once: more requests than device slots, so some wait on the host
        descs = []
        for i, t in enumerate(mixed):
            d = fv.ft_vote_desc.from_buffer_copy(t.desc)
            if i % 2 == 0:
                d.stats = None          # statistics only through ft_result
            descs.append(d)
        ptrs = (ctypes.c_void_p * len(descs))(*[ctypes.addressof(d) for d in descs])
        tickets = (ctypes.c_uint64 * len(descs))()
        acc = ctypes.c_int32()
        fv.check(fv.ft_submit_many(srv, ptrs, len(descs), tickets, ctypes.byref(acc)), "ft_submit_many")
        assert acc.value == len(descs)
        results = [_poll(fv, srv, tickets[i]) for i in range(len(descs))]
        info = fv.ft_server_stats()
        fv.ft_server_info(srv, ctypes.byref(info))
        assert info.requests == len(descs) and info.completed == len(descs)
    finally:
        fv.ft_server_destroy(srv)
    torch.cuda.synchronize()
    for i, (p, t, a, r) in enumerate(zip(probs, mixed, alone_res, results)):
        got = t.result()
        sd = _stats_dict(r.stats, p.R)
        if i % 2 == 0:
            got.update(sd)
            got["raw_stats"] = a["raw_stats"]
        else:
            # the caller's statistics buffer holds what the result reports
            for k, v in sd.items():
                assert np.array_equal(np.asarray(got[k]), np.asarray(v)), (i, k)
        assert_same(got, a, p.R)
        assert_same(got, oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol), p.R)


@pytest.mark.parametrize("mode", [1, 2])
def test_resident_small_request_overtakes_a_large_one(mode):
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    big = DevTask(synth.task_problem(synth.TaskSpec(64 << 20, "f32", 3, True, 41), config_id=5, flip_rate=1e-6))
    small = [DevTask(synth.task_problem(synth.TaskSpec(4096 * (1 + k), "f64", 5, k % 2 == 0, 50 + k),
                                        config_id=5, flip_rate=1e-3)) for k in range(8)]
    srv = _resident(mode=mode)
    try:
        # warm: the kernel is running when the large request arrives
        _poll(fv, srv, _submit(fv, srv, small[0].desc))
        tb = _submit(fv, srv, big.desc)
        ts = [_submit(fv, srv, t.desc) for t in small]
        rs = [_poll(fv, srv, tk) for tk in ts]
        rb = _poll(fv, srv, tb)
    finally:
        fv.ft_server_destroy(srv)
    torch.cuda.synchronize()
    # the small requests were admitted after the large one and still
    # completed before it: their tiles were claimed first (mode 2: they ran
    # on the resident kernel's SMs beside the large one's batch)
    assert max(r.done_us for r in rs) < rb.done_us
    for t in [big] + small:
        p = t.prob
        if p.n <= 1 << 20:
            assert_same(t.result(), oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol), p.R)
    a = DevTask(big.prob)
    fv.check(fv.ft_vote(ctypes.byref(a.desc), fv.stream_handle()), "ft_vote")
    torch.cuda.synchronize()
    assert_same(big.result(), a.result(), 3)


def test_resident_kernel_leaves_when_idle_and_comes_back():
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    probs = [synth.task_problem(synth.TaskSpec(100_003 + k, "f32", 3, True, 60 + k), config_id=5, flip_rate=1e-3)
             for k in range(3)]
    tasks = [DevTask(p) for p in probs]
    srv = _resident(idle_us=500)
    try:
        l0 = fv.ft_launch_count()
        for t in tasks:
            _poll(fv, srv, _submit(fv, srv, t.desc))
            time.sleep(0.05)        # far beyond the 0.5 ms idle limit: the kernel leaves
        launches = fv.ft_launch_count() - l0
    finally:
        fv.ft_server_destroy(srv)
    torch.cuda.synchronize()
    assert launches == 3            # one launch per request after an idle gap, none per request otherwise
    for t, p in zip(tasks, probs):
        assert_same(t.result(), oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol), p.R)


def test_resident_stream_of_requests_one_launch():
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    probs = [synth.task_problem(synth.TaskSpec(8192 + 17 * k, ["f32", "f64"][k % 2], [3, 5][k % 2], k % 4 == 0,
                                               80 + k), config_id=5, flip_rate=1e-3) for k in range(16)]
    tasks = [DevTask(p) for p in probs]
    srv = _resident(idle_us=200_000)
    try:
        l0 = fv.ft_launch_count()
        for rnd in range(5):
            tks = [_submit(fv, srv, t.desc) for t in tasks]
            for tk in tks:
                _poll(fv, srv, tk)
        launches = fv.ft_launch_count() - l0
    finally:
        fv.ft_server_destroy(srv)
    torch.cuda.synchronize()
    assert launches == 1            # 80 requests, one kernel launch
    for t, p in zip(tasks, probs):
        assert_same(t.result(), oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol), p.R)


@pytest.mark.parametrize("mode", [1, 2])
def test_resident_destroy_waits_for_the_request_on_the_device(mode):
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    n = (16 << 20) if mode == 1 else 100_000     # mode 2: a small request, on the resident kernel
    t = DevTask(synth.task_problem(synth.TaskSpec(n, "f64", 5, True, 90), config_id=5, flip_rate=1e-6))
    srv = _resident(mode=mode)
    _submit(fv, srv, t.desc)
    # destroy as soon as the request is on the device
    info = fv.ft_server_stats()
    t_end = time.monotonic() + 10.0
    while time.monotonic() < t_end:
        fv.ft_server_info(srv, ctypes.byref(info))
        if info.requests == 1:
            break
    assert info.requests == 1
    assert fv.ft_server_destroy(srv) == fv.FT_OK
    torch.cuda.synchronize()
    a = DevTask(t.prob)
    fv.check(fv.ft_vote(ctypes.byref(a.desc), fv.stream_handle()), "ft_vote")
    torch.cuda.synchronize()
    # the request was on the device when the server was destroyed: it was voted whole
    assert_same(t.result(), a.result(), 5)
