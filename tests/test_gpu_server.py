"""The serving form (ft_server_create / ft_submit / ft_poll): continuous
batching gives every request the same bit-exact result alone and in the mix;
admission follows the device-memory budget; waits are bounded (a request held
back on the host times out and completes once released); unknown tickets are
reported.  Failures are made on the host only."""
import collections
import ctypes
import time

import numpy as np
import pytest

import oracle
from paper_1405_2912_b300 import synth

from _gpu import DevTask, assert_same

pytestmark = pytest.mark.gpu


def _server(budget, max_slots=16, streams=2, tile=8, max_inflight=0, size_ratio=0):
    from paper_1405_2912_b300 import ftvote as fv
    cfg = fv.ft_server_config(budget, max_slots, streams, tile, max_inflight)
    cfg.size_ratio = size_ratio
    srv = ctypes.c_void_p()
    fv.check(fv.ft_server_create(ctypes.byref(srv), ctypes.byref(cfg)), "ft_server_create")
    return srv


def _requests(k=40, seed=2):
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(k):
        n = int(np.exp(rng.uniform(np.log(4096), np.log(300_000))))
        specs.append(synth.TaskSpec(n + int(rng.integers(0, 5)), ["f32", "f64"][i % 2], [3, 5][(i // 2) % 2],
                                    bool(i % 4 == 0), 9000 + i))
    return [synth.task_problem(s, config_id=5, ulp_frac=0.05, flip_rate=1e-3) for s in specs]


def _stats_dict(st, R):
    return {"mismatch": np.array(list(st.mismatch)[:R], dtype=np.uint64),
            "first_mismatch": np.array(list(st.first_mismatch)[:R], dtype=np.int64),
            "no_majority": int(st.no_majority), "first_no_majority": int(st.first_no_majority)}


@pytest.mark.parametrize("tile", [8, 0])          # 0: tile size chosen per batch
def test_same_alone_and_in_the_mix(tile):
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    probs = _requests()
    alone = [DevTask(p) for p in probs]
    for t in alone:
        fv.check(fv.ft_vote(ctypes.byref(t.desc), fv.stream_handle()), "ft_vote")
    torch.cuda.synchronize()
    alone_res = [t.result() for t in alone]
    mixed = [DevTask(p) for p in probs]
    srv = _server(budget=1 << 34, tile=tile)
    try:
        tickets = []
        for i, t in enumerate(mixed):
            d = fv.ft_vote_desc.from_buffer_copy(t.desc)
            if i % 3 == 0:
                d.stats = None          # statistics only through ft_result
            tk = ctypes.c_uint64()
            fv.check(fv.ft_submit(srv, ctypes.byref(d), ctypes.byref(tk)), "ft_submit")
            tickets.append(tk.value)
        results = []
        for tk in tickets:
            r = fv.ft_result()
            fv.check(fv.ft_poll(srv, tk, 30_000_000, ctypes.byref(r)), "ft_poll")
            assert r.status == fv.FT_OK and r.done_us >= r.submit_us
            results.append(r)
    finally:
        fv.ft_server_destroy(srv)
    torch.cuda.synchronize()
    for i, (p, t, a, r) in enumerate(zip(probs, mixed, alone_res, results)):
        got = t.result()
        sd = _stats_dict(r.stats, p.R)
        if i % 3 == 0:
            got.update(sd)
            got["raw_stats"] = a["raw_stats"]
        else:
            for k, v in sd.items():
                assert np.array_equal(np.asarray(got[k]), np.asarray(v)), (i, k)
        assert_same(got, a, p.R)
        if i % 7 == 0:
            assert_same(got, oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol), p.R)


def test_admission_by_budget_and_slots():
    from paper_1405_2912_b300 import ftvote as fv
    probs = _requests(k=3, seed=5)
    tasks = [DevTask(p) for p in probs]
    need = [(p.R + 1) * p.n * p.itemsize for p in probs]
    srv = _server(budget=need[0] + need[1])
    try:
        fv.ft_server_pause(srv, 1)
        t = [ctypes.c_uint64() for _ in range(3)]
        assert fv.ft_submit(srv, ctypes.byref(tasks[0].desc), ctypes.byref(t[0])) == fv.FT_OK
        assert fv.ft_submit(srv, ctypes.byref(tasks[1].desc), ctypes.byref(t[1])) == fv.FT_OK
        # over budget: refused, nothing kept
        assert fv.ft_submit(srv, ctypes.byref(tasks[2].desc), ctypes.byref(t[2])) == fv.FT_EAGAIN
        fv.ft_server_pause(srv, 0)
        r = fv.ft_result()
        assert fv.ft_poll(srv, t[0].value, 30_000_000, ctypes.byref(r)) == fv.FT_OK
        # budget released by collecting the result
        assert fv.ft_submit(srv, ctypes.byref(tasks[2].desc), ctypes.byref(t[2])) == fv.FT_OK
        for k in (1, 2):
            assert fv.ft_poll(srv, t[k].value, 30_000_000, ctypes.byref(r)) == fv.FT_OK
        # a request larger than the whole budget can never be admitted
        big = fv.ft_vote_desc.from_buffer_copy(tasks[0].desc)
        big.n = 1 << 40
        assert fv.ft_submit(srv, ctypes.byref(big), ctypes.byref(t[0])) == fv.FT_EINVAL
    finally:
        fv.ft_server_destroy(srv)
    srv = _server(budget=1 << 34, max_inflight=1)
    try:
        fv.ft_server_pause(srv, 1)
        assert fv.ft_submit(srv, ctypes.byref(tasks[0].desc), ctypes.byref(t[0])) == fv.FT_OK
        assert fv.ft_submit(srv, ctypes.byref(tasks[1].desc), ctypes.byref(t[1])) == fv.FT_EAGAIN
        fv.ft_server_pause(srv, 0)
        assert fv.ft_poll(srv, t[0].value, -1, ctypes.byref(r)) == fv.FT_OK
    finally:
        fv.ft_server_destroy(srv)


def test_bounded_wait_and_unknown_tickets():
    from paper_1405_2912_b300 import ftvote as fv
    p = _requests(k=1, seed=7)[0]
    t = DevTask(p)
    srv = _server(budget=1 << 32)
    try:
        fv.ft_server_pause(srv, 1)
        tk = ctypes.c_uint64()
        assert fv.ft_submit(srv, ctypes.byref(t.desc), ctypes.byref(tk)) == fv.FT_OK
        r = fv.ft_result()
        t0 = time.monotonic()
        assert fv.ft_poll(srv, tk.value, 20_000, ctypes.byref(r)) == fv.FT_ETIMEDOUT
        assert time.monotonic() - t0 >= 0.015
        assert fv.ft_poll(srv, tk.value, 0, ctypes.byref(r)) == fv.FT_ETIMEDOUT
        fv.ft_server_pause(srv, 0)
        assert fv.ft_poll(srv, tk.value, 30_000_000, ctypes.byref(r)) == fv.FT_OK
        assert fv.ft_poll(srv, tk.value, 0, ctypes.byref(r)) == fv.FT_ENOTFOUND
        assert fv.ft_poll(srv, 123456789, 0, ctypes.byref(r)) == fv.FT_ENOTFOUND
        ref = oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol)
        assert list(r.stats.mismatch)[:p.R] == [int(x) for x in ref["mismatch"]]
    finally:
        fv.ft_server_destroy(srv)


def test_server_counters():
    from paper_1405_2912_b300 import ftvote as fv
    probs = _requests(k=12, seed=8)
    tasks = [DevTask(p) for p in probs]
    # no size rule: the 12 requests are packed up to four per batch whatever
    # their sizes (spread over the free slots: how many batches depends on
    # when a slot frees up)
    srv = _server(budget=1 << 34, max_slots=4, streams=2, size_ratio=-1)
    try:
        fv.ft_server_pause(srv, 1)
        tks = []
        for t in tasks:
            tk = ctypes.c_uint64()
            assert fv.ft_submit(srv, ctypes.byref(t.desc), ctypes.byref(tk)) == fv.FT_OK
            tks.append(tk.value)
        info = fv.ft_server_stats()
        fv.ft_server_info(srv, ctypes.byref(info))
        assert info.batches == 0 and info.inflight_requests == 12
        fv.ft_server_pause(srv, 0)
        r = fv.ft_result()
        launch = []
        for tk in tks:
            assert fv.ft_poll(srv, tk, 30_000_000, ctypes.byref(r)) == fv.FT_OK
            launch.append(r.launch_us)
        fv.ft_server_info(srv, ctypes.byref(info))
        # 12 queued requests, at most 4 per batch, on up to 2 streams at once
        per_batch = list(collections.Counter(launch).values())
        assert info.batches == len(per_batch) and max(per_batch) <= 4 and info.batches >= 3
        assert info.requests == 12 and info.completed == 12
        assert 1 <= info.max_batches_in_flight <= 2
        assert info.inflight_requests == 0 and info.inflight_bytes == 0
    finally:
        fv.ft_server_destroy(srv)


def test_batch_byte_cap():
    from paper_1405_2912_b300 import ftvote as fv
    p = _requests(k=1, seed=12)[0]
    tasks = [DevTask(p) for _ in range(6)]
    need = (p.R + 1) * p.n * p.itemsize
    cfg = fv.ft_server_config(1 << 34, 4096, 1, 8, 0, 2 * need)
    srv = ctypes.c_void_p()
    fv.check(fv.ft_server_create(ctypes.byref(srv), ctypes.byref(cfg)), "ft_server_create")
    try:
        fv.ft_server_pause(srv, 1)
        tks = []
        for t in tasks:
            tk = ctypes.c_uint64()
            assert fv.ft_submit(srv, ctypes.byref(t.desc), ctypes.byref(tk)) == fv.FT_OK
            tks.append(tk.value)
        fv.ft_server_pause(srv, 0)
        r = fv.ft_result()
        for tk in tks:
            assert fv.ft_poll(srv, tk, 30_000_000, ctypes.byref(r)) == fv.FT_OK
        info = fv.ft_server_stats()
        fv.ft_server_info(srv, ctypes.byref(info))
        # two requests' bytes per batch: 6 requests in 3 batches on the single stream
        assert info.batches == 3 and info.requests == 6 and info.max_batches_in_flight == 1
    finally:
        fv.ft_server_destroy(srv)


def test_concurrent_clients():
    """Four host threads submit and poll at once (the ctypes calls release the
    GIL, so the server's locking is exercised for real); every result equals
    the payload voted alone."""
    import threading
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    probs = _requests(k=16, seed=21)
    tasks = [DevTask(p) for p in probs]
    for t in tasks:
        fv.check(fv.ft_vote(ctypes.byref(t.desc), fv.stream_handle()), "ft_vote")
    torch.cuda.synchronize()
    alone = [fv.parse_stats(t.stats, p.R) for t, p in zip(tasks, probs)]
    descs = []
    for t in tasks:
        d = fv.ft_vote_desc.from_buffer_copy(t.desc)
        d.stats = None
        descs.append(d)
    srv = _server(budget=1 << 33, max_slots=8, streams=3, tile=0)
    errors = []

    def client(cid):
        rng = np.random.default_rng(cid)
        res = fv.ft_result()
        tk = ctypes.c_uint64()
        try:
            for _ in range(150):
                k = int(rng.integers(0, len(descs)))
                while True:
                    rc = fv.ft_submit(srv, ctypes.byref(descs[k]), ctypes.byref(tk))
                    if rc == fv.FT_OK:
                        break
                    assert rc == fv.FT_EAGAIN
                    time.sleep(0.0005)
                assert fv.ft_poll(srv, tk.value, 30_000_000, ctypes.byref(res)) == fv.FT_OK
                R = probs[k].R
                got = {"mismatch": list(res.stats.mismatch)[:R], "first_mismatch": list(res.stats.first_mismatch)[:R],
                       "no_majority": res.stats.no_majority, "first_no_majority": res.stats.first_no_majority}
                assert got == alone[k], (cid, k)
        except Exception as e:          # reported by the main thread
            errors.append(repr(e))

    try:
        threads = [threading.Thread(target=client, args=(i,)) for i in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join(timeout=120)
        assert not any(th.is_alive() for th in threads)
        info = fv.ft_server_stats()
        fv.ft_server_info(srv, ctypes.byref(info))
        assert info.completed == 600 and info.inflight_requests == 0
    finally:
        fv.ft_server_destroy(srv)
    assert not errors, errors[:3]


def test_bulk_submit_and_poll():
    """ft_submit_many admits the prefix that fits the budget and stops at an
    invalid request; ft_poll_many retires the finished prefix of a ticket
    run; results are those of single votes."""
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    probs = _requests(k=6, seed=11)
    tasks = [DevTask(p) for p in probs]
    need = [(p.R + 1) * p.n * p.itemsize for p in probs]
    assert need[4] + need[5] <= sum(need[:4])       # the last two fit once the first four are retired
    ptrs = (ctypes.c_void_p * 6)(*[ctypes.addressof(t.desc) for t in tasks])
    tickets = (ctypes.c_uint64 * 6)()
    results = (fv.ft_result * 6)()
    acc, nd = ctypes.c_int32(), ctypes.c_int32()
    A = ctypes.addressof
    srv = _server(budget=sum(need[:4]))
    try:
        fv.ft_server_pause(srv, 1)
        # the first four fit, the fifth is refused for now
        assert fv.ft_submit_many(srv, A(ptrs), 6, A(tickets), ctypes.byref(acc)) == fv.FT_OK
        assert acc.value == 4
        assert len({tickets[k] for k in range(4)}) == 4
        # nothing has run: the first ticket times out, nothing is retired
        assert fv.ft_poll_many(srv, A(tickets), 4, 0, A(results), ctypes.byref(nd)) == fv.FT_ETIMEDOUT
        assert nd.value == 0
        fv.ft_server_pause(srv, 0)
        head = 0
        deadline = time.time() + 30
        while head < 4 and time.time() < deadline:
            rc = fv.ft_poll_many(srv, A(tickets) + 8 * head, 4 - head, 1_000_000,
                                 A(results) + ctypes.sizeof(fv.ft_result) * head, ctypes.byref(nd))
            assert rc in (fv.FT_OK, fv.FT_ETIMEDOUT)
            head += nd.value
        assert head == 4
        # retired tickets are unknown now; the count stops before them
        assert fv.ft_poll_many(srv, A(tickets), 2, 0, None, ctypes.byref(nd)) == fv.FT_ENOTFOUND
        assert nd.value == 0
        # the rest fit now; an invalid request stops the run at its index
        bad = fv.ft_vote_desc.from_buffer_copy(tasks[0].desc)
        bad.R = 1
        ptrs2 = (ctypes.c_void_p * 3)(A(tasks[4].desc), A(bad), A(tasks[5].desc))
        tk2 = (ctypes.c_uint64 * 3)()
        assert fv.ft_submit_many(srv, A(ptrs2), 3, A(tk2), ctypes.byref(acc)) == fv.FT_EINVAL
        assert acc.value == 1
        tickets[4] = tk2[0]
        ptrs3 = (ctypes.c_void_p * 1)(A(tasks[5].desc))
        assert fv.ft_submit_many(srv, A(ptrs3), 1, A(tickets) + 8 * 5, ctypes.byref(acc)) == fv.FT_OK
        assert acc.value == 1
        for k in (4, 5):
            assert fv.ft_poll_many(srv, A(tickets) + 8 * k, 1, -1, A(results) + ctypes.sizeof(fv.ft_result) * k,
                                   ctypes.byref(nd)) == fv.FT_OK and nd.value == 1
        # a run of zero is accepted and does nothing
        assert fv.ft_submit_many(srv, A(ptrs), 0, A(tickets), ctypes.byref(acc)) == fv.FT_OK and acc.value == 0
        assert fv.ft_poll_many(srv, A(tickets), 0, 0, None, ctypes.byref(nd)) == fv.FT_OK and nd.value == 0
    finally:
        fv.ft_server_destroy(srv)
    torch.cuda.synchronize()
    for k, (p, t) in enumerate(zip(probs, tasks)):
        assert results[k].status == fv.FT_OK and results[k].done_us >= results[k].submit_us
        got = t.result()
        ref = oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol)
        assert_same(got, ref, p.R)
        sd = _stats_dict(results[k].stats, p.R)
        for key, v in sd.items():
            assert np.array_equal(np.asarray(got[key]), np.asarray(v)), (k, key)


@pytest.mark.parametrize("user_stats", [False, True])
def test_empty_requests_and_groups_in_a_batch(user_stats):
    """One batch holding empty requests: inside a (kind, R) group that has
    tiles and as the whole of a group (no kernel runs for it); the server
    completes them at launch, or with the group kernel's copy-out where the
    caller gave statistics pointers.  Every
    empty request reads (0, -1) for all replicas; the others match the
    oracle.  Without caller statistics pointers the batch travels in the
    kernel parameters; one caller pointer sends it through the upload path
    (and that request's device statistics must match too).  The same server
    then takes a second batch, on counters and statistics left reset."""
    from paper_1405_2912_b300 import ftvote as fv
    specs = [synth.TaskSpec(0, "f64", 5, False, 41), synth.TaskSpec(5000, "f32", 3, True, 42),
             synth.TaskSpec(0, "f64", 5, False, 43), synth.TaskSpec(0, "i32", 4, False, 44),
             synth.TaskSpec(3001, "f64", 5, True, 45)]
    probs = [synth.task_problem(s, config_id=5, ulp_frac=0.05, flip_rate=1e-3) for s in specs]
    tasks = [DevTask(p) for p in probs]
    srv = _server(budget=1 << 32, streams=1, tile=0)    # one stream: all five in one batch
    try:
        for rnd in range(2):
            fv.ft_server_pause(srv, 1)
            tickets = []
            for i, t in enumerate(tasks):
                d = fv.ft_vote_desc.from_buffer_copy(t.desc)
                if not (user_stats and i == 1):
                    d.stats = None
                tk = ctypes.c_uint64()
                assert fv.ft_submit(srv, ctypes.byref(d), ctypes.byref(tk)) == fv.FT_OK
                tickets.append(tk.value)
            fv.ft_server_pause(srv, 0)
            for i, (p, tk) in enumerate(zip(probs, tickets)):
                r = fv.ft_result()
                assert fv.ft_poll(srv, tk, 30_000_000, ctypes.byref(r)) == fv.FT_OK
                assert r.status == fv.FT_OK
                if p.n == 0:
                    assert list(r.stats.mismatch) == [0] * 8 and list(r.stats.first_mismatch) == [-1] * 8
                    assert r.stats.no_majority == 0 and r.stats.first_no_majority == -1
                    continue
                ref = oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol)
                views = [_stats_dict(r.stats, p.R)]
                if user_stats and i == 1:
                    views.append(tasks[i].result())
                for got in views:
                    assert [int(x) for x in got["mismatch"]] == [int(x) for x in ref["mismatch"]]
                    assert [int(x) for x in got["first_mismatch"]] == [int(x) for x in ref["first_mismatch"]]
                    assert int(got["no_majority"]) == int(ref["no_majority"])
                    assert int(got["first_no_majority"]) == int(ref["first_no_majority"])
            info = fv.ft_server_stats()
            fv.ft_server_info(srv, ctypes.byref(info))
            assert info.batches == rnd + 1
    finally:
        fv.ft_server_destroy(srv)


@pytest.mark.parametrize("user_stats", [False, True])
def test_every_kind_and_r_through_the_server(user_stats):
    """Every element type with every R from 2 to 8 (49 requests with specials,
    ties and flips, sizes from 1 element to ragged multi-block), voted by a
    server that packs up to 16 requests per batch, so that batches hold
    several (kind, R) groups on the auxiliary streams.  Without caller
    statistics pointers the batches take the small-batch path (each group in
    a kernel parameter); with them, the upload path.  Voted values, digests
    and statistics equal the oracle's bit for bit."""
    from paper_1405_2912_b300 import ftvote as fv
    from test_gpu_vote import _random_problem
    dts = ["f32", "f64", "i32", "u32", "i64", "u64", "u8"]
    sizes = [1, 1023, 4097, 12345, 65536 + 77]
    probs = []
    for i, (dt, R) in enumerate((d, r) for d in dts for r in range(2, 9)):
        reps, tol = _random_problem(dt, R, sizes[i % len(sizes)], seed=7000 + i)
        probs.append(synth.Problem(reps, dt, *tol))
    tasks = [DevTask(p) for p in probs]
    srv = _server(budget=1 << 34, max_slots=16, streams=3, tile=0)
    try:
        fv.ft_server_pause(srv, 1)
        tickets = []
        for t in tasks:
            d = fv.ft_vote_desc.from_buffer_copy(t.desc)
            if not user_stats:
                d.stats = None
            tk = ctypes.c_uint64()
            assert fv.ft_submit(srv, ctypes.byref(d), ctypes.byref(tk)) == fv.FT_OK
            tickets.append(tk.value)
        fv.ft_server_pause(srv, 0)
        for p, t, tk in zip(probs, tasks, tickets):
            r = fv.ft_result()
            assert fv.ft_poll(srv, tk, 30_000_000, ctypes.byref(r)) == fv.FT_OK
            assert r.status == fv.FT_OK
            ref = oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol)
            got = t.result()
            assert got["out"].tobytes() == ref["out"].tobytes(), (p.dtype, p.R, p.n)
            assert np.array_equal(got["block_crc"], ref["block_crc"]), (p.dtype, p.R, p.n)
            views = [_stats_dict(r.stats, p.R)] + ([got] if user_stats else [])
            for v in views:
                assert [int(x) for x in v["mismatch"]] == [int(x) for x in ref["mismatch"]], (p.dtype, p.R)
                assert [int(x) for x in v["first_mismatch"]] == [int(x) for x in ref["first_mismatch"]]
                assert int(v["no_majority"]) == int(ref["no_majority"])
                assert int(v["first_no_majority"]) == int(ref["first_no_majority"])
        info = fv.ft_server_stats()
        fv.ft_server_info(srv, ctypes.byref(info))
        assert info.batches >= 4      # 49 requests, at most 16 per batch
    finally:
        fv.ft_server_destroy(srv)


def test_size_rule_keeps_small_requests_out_of_a_large_ones_batch():
    """With a slot to spare, a batch takes waiting requests only within the
    size factor of its first one: a large request and small ones queued behind
    it go into separate batches, and every result equals the oracle."""
    from paper_1405_2912_b300 import ftvote as fv
    big = synth.task_problem(synth.TaskSpec(1 << 20, "f32", 3, True, 31), config_id=5)
    small = [synth.task_problem(synth.TaskSpec(3000 + 17 * i, "f32", 3, i % 2 == 0, 40 + i), config_id=5)
             for i in range(5)]
    probs = [big] + small
    tasks = [DevTask(p) for p in probs]
    srv = _server(budget=1 << 34, max_slots=16, streams=3)
    try:
        fv.ft_server_pause(srv, 1)
        tks = []
        for t in tasks:
            tk = ctypes.c_uint64()
            assert fv.ft_submit(srv, ctypes.byref(t.desc), ctypes.byref(tk)) == fv.FT_OK
            tks.append(tk.value)
        fv.ft_server_pause(srv, 0)
        r = fv.ft_result()
        launch = []
        for tk in tks:
            assert fv.ft_poll(srv, tk, 30_000_000, ctypes.byref(r)) == fv.FT_OK
            launch.append(r.launch_us)
        # the large request alone in its batch, the small ones in others
        assert launch[0] not in launch[1:]
        info = fv.ft_server_stats()
        fv.ft_server_info(srv, ctypes.byref(info))
        assert info.batches == len(set(launch)) >= 2
    finally:
        fv.ft_server_destroy(srv)
    for p, t in zip(probs, tasks):
        assert_same(t.result(), oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol), p.R)


@pytest.mark.parametrize("nsmall", [5, 20])
def test_requests_complete_on_their_own_inside_a_batch(nsmall):
    """Small requests packed into one batch with a large one complete as soon
    as their own tiles are voted, before the large one: the batch runs its
    requests smallest first, and the warp that votes a request's last tile
    flags it to the host.  Five small requests travel in the kernel
    parameters, twenty through the upload path.  Every result equals the
    oracle's."""
    from paper_1405_2912_b300 import ftvote as fv
    big = synth.task_problem(synth.TaskSpec(1 << 26, "f32", 3, True, 61), config_id=5)
    small = [synth.task_problem(synth.TaskSpec(4096 * (1 + i % 3) + 7 * i, "f32", 3, i % 3 == 0, 70 + i),
                                config_id=5)
             for i in range(nsmall)]
    probs = [big] + small                 # the large one is the oldest
    tasks = [DevTask(p) for p in probs]
    # one stream: every waiting request goes into the one free slot's batch
    srv = _server(budget=1 << 36, max_slots=64, streams=1, tile=0, size_ratio=-1)
    try:
        fv.ft_server_pause(srv, 1)
        tks = []
        for t in tasks:
            d = fv.ft_vote_desc.from_buffer_copy(t.desc)
            d.stats = None
            tk = ctypes.c_uint64()
            assert fv.ft_submit(srv, ctypes.byref(d), ctypes.byref(tk)) == fv.FT_OK
            tks.append(tk.value)
        fv.ft_server_pause(srv, 0)
        res = []
        for tk in tks:
            r = fv.ft_result()
            assert fv.ft_poll(srv, tk, 30_000_000, ctypes.byref(r)) == fv.FT_OK
            assert r.status == fv.FT_OK
            res.append(r)
        info = fv.ft_server_stats()
        fv.ft_server_info(srv, ctypes.byref(info))
        assert info.batches == 1
        assert len({r.launch_us for r in res}) == 1
        # 1 GiB of replicas takes well over 100 us; the small ones finish first
        assert max(r.done_us for r in res[1:]) < res[0].done_us
    finally:
        fv.ft_server_destroy(srv)
    for p, t, r in zip(probs, tasks, res):
        ref = oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol)
        got = t.result()
        assert got["out"].tobytes() == ref["out"].tobytes()
        assert np.array_equal(got["block_crc"], ref["block_crc"])
        sd = _stats_dict(r.stats, p.R)
        assert [int(x) for x in sd["mismatch"]] == [int(x) for x in ref["mismatch"]]
        assert [int(x) for x in sd["first_mismatch"]] == [int(x) for x in ref["first_mismatch"]]
        assert sd["no_majority"] == int(ref["no_majority"])
        assert sd["first_no_majority"] == int(ref["first_no_majority"])


def test_large_requests_of_a_small_batch_vote_on_their_own():
    """In a batch of at most 16 requests, each request of 64 MiB or more of
    replicas and output votes on its own through the single-task voter, on a
    stream beside the batch's small-batch kernels; the small requests share
    one kernel per (kind, R) group.  Two large requests of different kinds,
    three small ones in two groups and an empty one: four launches, and every
    result equals the oracle's, statistics included."""
    from paper_1405_2912_b300 import ftvote as fv
    specs = [synth.TaskSpec(5000, "f32", 3, True, 81), synth.TaskSpec(0, "f32", 3, False, 82),
             synth.TaskSpec(1 << 23, "f32", 3, True, 83), synth.TaskSpec(7000, "f64", 5, True, 84),
             synth.TaskSpec(3 << 20, "f64", 5, True, 85), synth.TaskSpec(9000, "f32", 3, False, 86)]
    probs = [synth.task_problem(sp, config_id=5, ulp_frac=0.05, flip_rate=1e-3) for sp in specs]
    big = [(p.R + 1) * p.n * p.itemsize >= 64 << 20 for p in probs]
    assert big == [False, False, True, False, True, False]
    tasks = [DevTask(p) for p in probs]
    srv = _server(budget=1 << 36, max_slots=16, streams=1, tile=0, size_ratio=-1)
    try:
        fv.ft_server_pause(srv, 1)
        tks = []
        for t in tasks:
            d = fv.ft_vote_desc.from_buffer_copy(t.desc)
            d.stats = None
            tk = ctypes.c_uint64()
            assert fv.ft_submit(srv, ctypes.byref(d), ctypes.byref(tk)) == fv.FT_OK
            tks.append(tk.value)
        l0 = fv.ft_launch_count()
        fv.ft_server_pause(srv, 0)
        res = []
        for tk in tks:
            r = fv.ft_result()
            assert fv.ft_poll(srv, tk, 30_000_000, ctypes.byref(r)) == fv.FT_OK
            assert r.status == fv.FT_OK
            res.append(r)
        launches = fv.ft_launch_count() - l0
        info = fv.ft_server_stats()
        fv.ft_server_info(srv, ctypes.byref(info))
        assert info.batches == 1
    finally:
        fv.ft_server_destroy(srv)
    # f32 R=3 and f64 R=5 small-batch kernels, and the two single votes
    assert launches == 4
    for p, t, r in zip(probs, tasks, res):
        ref = oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol)
        sd = _stats_dict(r.stats, p.R)
        assert [int(x) for x in sd["mismatch"]] == [int(x) for x in ref["mismatch"]]
        assert [int(x) for x in sd["first_mismatch"]] == [int(x) for x in ref["first_mismatch"]]
        assert sd["no_majority"] == int(ref["no_majority"])
        assert sd["first_no_majority"] == int(ref["first_no_majority"])
        if p.n:
            got = t.result()
            assert got["out"].tobytes() == ref["out"].tobytes()
            assert np.array_equal(got["block_crc"], ref["block_crc"])
