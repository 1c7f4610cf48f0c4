"""Replay of a vote-request arrival stream against an ft_server.

A load generator for the serving form: it submits each request at its
scheduled arrival time (host monotonic clock of the library, ft_clock_us),
retries requests that the budget refuses, collects results in arrival order,
and reports latency = completion time (when the server's worker saw the
request complete) minus the scheduled arrival time, so that queueing behind
the budget and in the server both count.  Each pass of its loop submits every
request that has arrived with one ft_submit_many, and retires the finished
ones with one ft_poll_many every so often, so the generator's own cost does
not grow with the request rate.  It only calls the C ABI; all voting runs on the GPU.
"""
from __future__ import annotations

import collections
import ctypes
import gc

import numpy as np

from . import ftvote as fv


def replay(srv, descs, arrivals_s, payload_of, start_delay_us=2000.0, poll_every_us=50.0):
    """Submit descs[payload_of[i]] at arrivals_s[i] seconds after the start.

    Returns a dict with per-request latencies (us), the number of budget
    refusals, and the wall span from the first arrival to the last completion.
    Python's cyclic garbage collector is paused for the replay: one of its
    full collections stalls the submitting loop for milliseconds, which would
    show as server latency.  Finished requests are collected at most every
    poll_every_us: a request's completion time is the server's, so collecting
    it later changes no latency, and fewer polls leave the loop free to submit
    on time and the server's lock to its worker.
    """
    was_enabled = gc.isenabled()
    gc.collect()
    gc.disable()
    try:
        return _replay(srv, descs, arrivals_s, payload_of, start_delay_us, poll_every_us)
    finally:
        if was_enabled:
            gc.enable()


def _replay(srv, descs, arrivals_s, payload_of, start_delay_us, poll_every_us):
    n = len(arrivals_s)
    m = max(n, 1)
    # one descriptor pointer, ticket and result slot per request, laid out
    # before the clock starts; the loop passes offsets into them
    dptr = (ctypes.c_void_p * m)(*[ctypes.addressof(descs[k]) for k in payload_of])
    tickets = (ctypes.c_uint64 * m)()
    results = (fv.ft_result * m)()
    a_d, a_t, a_r = ctypes.addressof(dptr), ctypes.addressof(tickets), ctypes.addressof(results)
    rsz = ctypes.sizeof(fv.ft_result)
    acc, nd = ctypes.c_int32(), ctypes.c_int32()
    pacc, pnd = ctypes.byref(acc), ctypes.byref(nd)
    submit_many, poll_many, clock = fv.ft_submit_many, fv.ft_poll_many, fv.ft_clock_us
    t0 = clock() + start_delay_us
    arr = t0 + np.asarray(arrivals_s, dtype=np.float64) * 1e6
    arr_l = arr.tolist()                  # scalar reads of a list are cheaper than of an array
    i = head = 0
    refused = 0
    last_poll = 0.0
    while head < n:
        now = clock()
        due = i
        while due < n and arr_l[due] <= now:   # arrivals that have passed
            due += 1
        blocked = False
        if due > i:
            fv.check(submit_many(srv, a_d + 8 * i, due - i, a_t + 8 * i, pacc), "ft_submit_many")
            blocked = acc.value < due - i
            if blocked:
                refused += 1              # the budget is full: collect, then retry on the next pass
            i += acc.value
        if head < i and (blocked or i == n or now - last_poll >= poll_every_us):
            last_poll = now
            rc = poll_many(srv, a_t + 8 * head, i - head, 0, a_r + rsz * head, pnd)
            if rc != fv.FT_ETIMEDOUT:
                fv.check(rc, "ft_poll_many")
            head += nd.value
    done_at = np.array([results[k].done_us for k in range(n)], dtype=np.float64)
    submit_at = np.array([results[k].submit_us for k in range(n)], dtype=np.float64)
    launch_at = np.array([results[k].launch_us for k in range(n)], dtype=np.float64)
    launched_at = np.array([results[k].launched_us for k in range(n)], dtype=np.float64)
    errors = sum(1 for k in range(n) if results[k].status != fv.FT_OK)
    lat = done_at - arr
    span_s = (done_at.max() - arr.min()) / 1e6 if n else 0.0
    return {"latency_us": lat, "submit_lag_us": submit_at - arr, "server_us": done_at - submit_at,
            "queue_us": launch_at - submit_at, "launch_us": launched_at - launch_at, "launch_stamp": launch_at,
            "device_us": done_at - launched_at, "refused": refused, "span_s": span_s, "errors": errors}


def summarize(r, bytes_per_req):
    lat = r["latency_us"]
    n = lat.size
    return {"requests": int(n),
            "p50_us": round(float(np.percentile(lat, 50)), 1) if n else None,
            "p99_us": round(float(np.percentile(lat, 99)), 1) if n else None,
            "mean_us": round(float(lat.mean()), 1) if n else None,
            "max_us": round(float(lat.max()), 1) if n else None,
            # the latency split at the server's submit timestamp: the load
            # generator's lag behind the schedule, and submit -> completion
            "submit_lag_p50_us": round(float(np.percentile(r["submit_lag_us"], 50)), 1) if n else None,
            "server_p50_us": round(float(np.percentile(r["server_us"], 50)), 1) if n else None,
            "server_p99_us": round(float(np.percentile(r["server_us"], 99)), 1) if n else None,
            "req_per_s": round(n / r["span_s"], 1) if r["span_s"] > 0 else None,
            "gb_per_s": round(float(np.sum(bytes_per_req)) / r["span_s"] / 1e9, 2) if r["span_s"] > 0 else None,
            "budget_refusals": int(r["refused"]), "errors": int(r["errors"])}


def replay_plain(descs, arrivals_s, payload_of, nstreams=3, start_delay_us=2000.0):
    """The same arrival stream without a server: each request is one ft_vote
    call, issued at its arrival on the next of `nstreams` streams in turn,
    followed by an event on that stream.  The loop that issues the calls also
    polls the oldest outstanding event of each stream and takes the time at
    which it sees it complete, as the server's worker does for a batch, so
    that latency = seen complete - scheduled arrival has the same meaning in
    both.  descs[s][p] is payload p's descriptor for stream s (each stream
    with its own statistics buffers, so that two requests in flight on
    different streams never share one)."""
    was_enabled = gc.isenabled()
    gc.collect()
    gc.disable()
    try:
        return _replay_plain(descs, arrivals_s, payload_of, nstreams, start_delay_us)
    finally:
        if was_enabled:
            gc.enable()


def _replay_plain(descs, arrivals_s, payload_of, nstreams, start_delay_us):
    import torch
    n = len(arrivals_s)
    streams = [torch.cuda.Stream() for _ in range(nstreams)]
    handles = [int(s.cuda_stream) for s in streams]
    events = [torch.cuda.Event() for _ in range(max(n, 1))]
    # a torch event creates its CUDA event at its first record: record each
    # once before the clock starts, so that the loop creates none
    for k, e in enumerate(events):
        e.record(streams[k % nstreams])
    torch.cuda.synchronize()
    refs = [[ctypes.byref(d) for d in per_stream] for per_stream in descs]
    vote, clock = fv.ft_vote, fv.ft_clock_us
    queues = [collections.deque() for _ in range(nstreams)]
    done_at = np.zeros(n, dtype=np.float64)
    issued_at = np.zeros(n, dtype=np.float64)
    errors = 0
    torch.cuda.synchronize()
    t0 = clock() + start_delay_us
    arr = t0 + np.asarray(arrivals_s, dtype=np.float64) * 1e6
    i = head = 0
    while head < n:
        now = clock()
        while i < n and arr[i] <= now:
            s = i % nstreams
            issued_at[i] = clock()
            if vote(refs[s][payload_of[i]], handles[s]) != fv.FT_OK:
                errors += 1
            events[i].record(streams[s])
            queues[s].append(i)
            i += 1
        for q in queues:
            while q and events[q[0]].query():
                done_at[q.popleft()] = clock()
                head += 1
    torch.cuda.synchronize()
    lat = done_at - arr
    span_s = (done_at.max() - arr.min()) / 1e6 if n else 0.0
    return {"latency_us": lat, "submit_lag_us": issued_at - arr, "server_us": done_at - issued_at,
            "refused": 0, "span_s": span_s, "errors": errors}
