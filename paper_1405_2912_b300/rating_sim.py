"""A seeded simulation of the paper's fault-injection experiment (Sec. V.C)
on the fault-aware rating of Sec. IV.B.

A CPU kernel three times faster than the GPU kernel faults with probability q;
a faulty run is redone on the next unit until a run is valid.  Two scheduling
strategies choose the unit that runs first:
  - fault-aware: the order of ft_rating_rank over the units' fault-free
    runtimes and observed valid / total runs (a unit that always failed is
    retried only in check rounds);
  - avoid: the CPU until its first fault, the GPU from then on.
The result is the mean time until a valid result, in units of the CPU
kernel's fault-free runtime.  Only the scheduling decision calls the library
(ft_rating_rank); the faults are drawn here."""
from __future__ import annotations

import ctypes

import numpy as np

from . import ftvote as fv


def rank(units, round_=1, check_interval=0):
    """ft_rating_rank over (runtime, valid_runs, total_runs) tuples."""
    arr = (fv.ft_unit_rating * len(units))(*[fv.ft_unit_rating(*u) for u in units])
    order = (ctypes.c_int32 * len(units))()
    count = ctypes.c_int32()
    fv.check(fv.ft_rating_rank(arr, len(units), round_, check_interval, order, ctypes.byref(count)),
             "ft_rating_rank")
    return list(order[:count.value])


def simulate(q, rounds, strategy, seed, speedup=3.0, check_interval=50):
    """Mean time per valid result over `rounds` results."""
    rng = np.random.default_rng(seed)
    runtime = [1.0, speedup]         # fault-free runtimes: CPU, GPU
    p_fault = [q, 0.0]
    counts = [[0, 0], [0, 0]]        # valid, total
    avoided = False
    total = 0.0
    for k in range(1, rounds + 1):
        if strategy == "fault-aware":
            order = rank([(runtime[u], counts[u][0], counts[u][1]) for u in (0, 1)], k, check_interval) or [1]
        elif strategy == "avoid":
            order = [1] if avoided else [0, 1]
        else:
            raise ValueError(strategy)
        for u in order + [1]:
            total += runtime[u]
            ok = rng.random() >= p_fault[u]
            counts[u][1] += 1
            counts[u][0] += ok
            if not ok and u == 0:
                avoided = True
            if ok:
                break
    return total / rounds


def sweep(qs, rounds=4000, seed=1, speedup=3.0):
    """Mean time per result of both strategies for each fault probability."""
    return [{"q": float(q), "fault_aware": round(simulate(q, rounds, "fault-aware", seed, speedup), 3),
             "avoid_after_first_fault": round(simulate(q, rounds, "avoid", seed, speedup), 3)} for q in qs]
