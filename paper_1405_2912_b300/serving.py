"""Replay of a vote-request arrival stream against an ft_server.

A load generator for the serving form: it submits each request at its
scheduled arrival time (host monotonic clock of the library, ft_clock_us),
retries requests that the budget refuses, collects results in arrival order,
and reports latency = completion time (the batch's completion callback) minus
the scheduled arrival time, so that queueing behind the budget and in the
server both count.  It only calls the C ABI; all voting runs on the GPU.
"""
from __future__ import annotations

import collections
import ctypes

import numpy as np

from . import ftvote as fv


def replay(srv, descs, arrivals_s, payload_of, start_delay_us=2000.0):
    """Submit descs[payload_of[i]] at arrivals_s[i] seconds after the start.

    Returns a dict with per-request latencies (us), the number of budget
    refusals, and the wall span from the first arrival to the last completion.
    """
    n = len(arrivals_s)
    t0 = fv.ft_clock_us() + start_delay_us
    arr = t0 + np.asarray(arrivals_s, dtype=np.float64) * 1e6
    lat = np.zeros(n)
    done_at = np.zeros(n)
    outstanding = collections.deque()
    res = fv.ft_result()
    tk = ctypes.c_uint64()
    i = 0
    refused = 0
    submit = fv.ft_submit
    poll = fv.ft_poll
    clock = fv.ft_clock_us
    pres = ctypes.byref(res)
    ptk = ctypes.byref(tk)
    dptr = [ctypes.byref(d) for d in descs]
    errors = 0
    while i < n or outstanding:
        now = clock()
        while i < n and arr[i] <= now:
            rc = submit(srv, dptr[payload_of[i]], ptk)
            if rc == fv.FT_EAGAIN:
                refused += 1
                break
            fv.check(rc, "ft_submit")
            outstanding.append((tk.value, i))
            i += 1
        while outstanding:
            t, k = outstanding[0]
            rc = poll(srv, t, 0, pres)
            if rc == fv.FT_ETIMEDOUT:
                break
            fv.check(rc, "ft_poll")
            if res.status != fv.FT_OK:
                errors += 1
            lat[k] = res.done_us - arr[k]
            done_at[k] = res.done_us
            outstanding.popleft()
    span_s = (done_at.max() - arr.min()) / 1e6 if n else 0.0
    return {"latency_us": lat, "refused": refused, "span_s": span_s, "errors": errors}


def summarize(r, bytes_per_req):
    lat = r["latency_us"]
    n = lat.size
    return {"requests": int(n),
            "p50_us": round(float(np.percentile(lat, 50)), 1) if n else None,
            "p99_us": round(float(np.percentile(lat, 99)), 1) if n else None,
            "mean_us": round(float(lat.mean()), 1) if n else None,
            "req_per_s": round(n / r["span_s"], 1) if r["span_s"] > 0 else None,
            "gb_per_s": round(float(np.sum(bytes_per_req)) / r["span_s"] / 1e9, 2) if r["span_s"] > 0 else None,
            "budget_refusals": int(r["refused"]), "errors": int(r["errors"])}
