"""Seeded synthetic replica buffers with injected faults.

This module is the one source of inputs for both the CUDA path and the CPU
oracle.  It holds no voting or digest arithmetic: it only draws values (numpy
PCG64, seeded) and injects the kinds of disagreement the voter must handle:

* ``ulp_perturb``  -- move a float by a few units in the last place (what a
  different operation order or rounding mode on another processing unit does,
  Sec. IV.D of the paper); usually inside the stated tolerance.
* ``bit_flip``     -- flip one bit of an element (a transient hardware fault).
* a contiguous block of systematically wrong values (a software bug in one
  kernel, the case the paper's HetDMR mode targets, Sec. IV.D).
* deliberate tie sites, where two groups of replicas of equal size disagree.

The paper's own workloads (Rodinia and CUDA SDK outputs, Sec. V) are not
available; these generators stand in for them with the shapes of the five
workloads of the voter (3 x 1M f32; 3 x 256M f32; 5 x 64M f64 + 5 x 64M i32;
4096 batched tasks; a Poisson request stream).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NP_OF = {"i32": np.int32, "u32": np.uint32, "i64": np.int64, "u64": np.uint64,
         "u8": np.uint8, "f32": np.float32, "f64": np.float64}
SEED_BASE = 20140512

# Tolerances of the five workloads.
TOL = {"f32": (1e-6, 1e-5), "f64": (0.0, 1e-12)}


def rng_for(config_id: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([SEED_BASE + config_id, salt]))


@dataclass
class Problem:
    """R replica buffers of one dtype plus the tolerances to vote them with."""
    replicas: list
    dtype: str
    abs_tol: float = 0.0
    rel_tol: float = 0.0
    truth: dict = field(default_factory=dict)   # injected positions, for invariant tests

    @property
    def n(self) -> int:
        return int(self.replicas[0].size)

    @property
    def R(self) -> int:
        return len(self.replicas)

    @property
    def itemsize(self) -> int:
        return np.dtype(NP_OF[self.dtype]).itemsize

    @property
    def bytes_moved(self) -> int:
        """Algorithmic traffic of one vote: R reads plus one write."""
        return (self.R + 1) * self.n * self.itemsize


# ---------------------------------------------------------------------------
# value distributions
# ---------------------------------------------------------------------------

def uniform_f32(rng, n, lo=-1.0, hi=1.0):
    return rng.uniform(lo, hi, size=n).astype(np.float32)


def lognormal(rng, n, dtype, sigma=2.0):
    """Magnitudes exp(N(0, sigma)), random sign."""
    mag = rng.lognormal(0.0, sigma, size=n)
    sign = rng.integers(0, 2, size=n, dtype=np.int8) * 2 - 1
    return (mag * sign).astype(NP_OF[dtype])


def uniform_int(rng, n, dtype):
    info = np.iinfo(NP_OF[dtype])
    return rng.integers(info.min, info.max, size=n, dtype=NP_OF[dtype], endpoint=True)


# ---------------------------------------------------------------------------
# fault injection (all in place, all return the touched indices)
# ---------------------------------------------------------------------------

def _bits_view(a):
    return a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)


def ulp_perturb(a: np.ndarray, idx: np.ndarray, delta: np.ndarray) -> None:
    """Add delta units in the last place to |a[idx]| (integer add on the bit
    pattern of the magnitude, sign kept).  A step that would cross zero or
    reach the exponent of Inf/NaN is taken in the other direction instead."""
    bits = _bits_view(a)
    wide = np.int64
    if a.dtype.itemsize == 4:
        sign_mask, inf_bits = np.uint32(0x80000000), 0x7F800000
    else:
        sign_mask, inf_bits = np.uint64(0x8000000000000000), 0x7FF0000000000000
    b = bits[idx]
    sign = b & sign_mask
    mag = (b & ~sign_mask).astype(wide)
    d = delta.astype(wide)
    m2 = mag + d
    bad = (m2 < 0) | (m2 >= inf_bits)
    m2 = np.where(bad, mag - d, m2)
    bits[idx] = sign | m2.astype(bits.dtype)


def bit_flip(a: np.ndarray, idx: np.ndarray, bit: np.ndarray) -> None:
    """Flip bit number bit[k] (0 = least significant) of element idx[k]."""
    raw = a.view({1: np.uint8, 4: np.uint32, 8: np.uint64}[a.dtype.itemsize])
    one = raw.dtype.type(1)
    raw[idx] ^= (one << bit.astype(raw.dtype))


def distinct_indices(rng, n, k):
    k = int(min(k, n))
    if k == 0:
        return np.zeros(0, dtype=np.int64)
    if k * 4 > n:
        return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)
    idx = np.unique(rng.integers(0, n, size=k + k // 8 + 16))
    while idx.size < k:
        idx = np.unique(np.concatenate([idx, rng.integers(0, n, size=k)]))
    return np.sort(rng.permutation(idx)[:k]).astype(np.int64)


def bernoulli_indices(rng, n, p):
    return distinct_indices(rng, n, rng.binomial(n, p))


# ---------------------------------------------------------------------------
# the five workloads (sizes default to the full workloads; tests shrink n)
# ---------------------------------------------------------------------------

def cfg1(n: int = 1 << 20, flips: int = 100, ulp_frac: float = 0.10) -> Problem:
    """3 x n f32 ~ U[-1,1]; B = A with +-1..2 ULP on 10% of elements;
    C = A with `flips` single-bit flips at uniform (index, bit)."""
    rng = rng_for(1)
    a = uniform_f32(rng, n)
    b = a.copy()
    c = a.copy()
    ulp_idx = np.flatnonzero(rng.random(n) < ulp_frac)
    mag = rng.integers(1, 3, size=ulp_idx.size)
    ulp_perturb(b, ulp_idx, mag * (rng.integers(0, 2, size=ulp_idx.size) * 2 - 1))
    fidx = distinct_indices(rng, n, flips)
    fbit = rng.integers(0, 32, size=fidx.size)
    bit_flip(c, fidx, fbit)
    return Problem([a, b, c], "f32", *TOL["f32"],
                   truth={"clean": a, "ulp_idx": ulp_idx, "flip_idx": fidx, "flip_bit": fbit})


def cfg2(n: int = 1 << 28, ulp_frac: float = 0.20, flip_rate: float = 1e-6) -> Problem:
    """3 x n f32, lognormal magnitudes (sigma 2), random sign; replica 1 with
    +-1..4 ULP on 20% of elements; replica 2 with bit flips at 1e-6/element."""
    rng = rng_for(2)
    a = lognormal(rng, n, "f32")
    b = a.copy()
    c = a.copy()
    ulp_idx = np.flatnonzero(rng.random(n, dtype=np.float32) < ulp_frac)
    mag = rng.integers(1, 5, size=ulp_idx.size, dtype=np.int32)
    sgn = rng.integers(0, 2, size=ulp_idx.size, dtype=np.int32) * 2 - 1
    ulp_perturb(b, ulp_idx, mag * sgn)
    fidx = bernoulli_indices(rng, n, flip_rate)
    fbit = rng.integers(0, 32, size=fidx.size)
    bit_flip(c, fidx, fbit)
    return Problem([a, b, c], "f32", *TOL["f32"],
                   truth={"clean": a, "ulp_idx": ulp_idx, "flip_idx": fidx, "flip_bit": fbit})


def cfg3(n: int = 1 << 26, block: int = 1 << 20, flip_rate: float = 1e-5,
         ties: int = 1024) -> tuple:
    """5 x n f64 (lognormal, rel_tol 1e-12) and 5 x n i32 (uniform full range).
    Replica 3 is wrong on one contiguous `block` of elements (f64 scaled by
    1+1e-6, i32 + 1); replicas 1 and 4 carry sparse bit flips; at `ties` sites
    replicas {1,2} hold one value, {0,3} another and 4 a third, so that the
    lowest-index tie rule decides.  Returns (f64 Problem, i32 Problem)."""
    rng = rng_for(3)
    start = int(rng.integers(0, max(1, n - block + 1)))
    tie_idx = distinct_indices(rng, n, ties)
    out = []
    for dt in ("f64", "i32"):
        base = lognormal(rng, n, "f64") if dt == "f64" else uniform_int(rng, n, "i32")
        reps = [base.copy() for _ in range(5)]
        sl = slice(start, min(n, start + block))
        if dt == "f64":
            reps[3][sl] = reps[3][sl] * (1.0 + 1e-6)
        else:
            reps[3][sl] = reps[3][sl] + np.int32(1)
        flips = {}
        for r in (1, 4):
            fidx = bernoulli_indices(rng, n, flip_rate)
            fbit = rng.integers(0, 64 if dt == "f64" else 32, size=fidx.size)
            bit_flip(reps[r], fidx, fbit)
            flips[r] = (fidx, fbit)
        if tie_idx.size:
            x = base[tie_idx]
            if dt == "f64":
                xp = x * (1.0 + 1e-3)
                z = x * (1.0 - 1e-3) + 1.0
            else:
                xp = x + np.int32(7)
                z = uniform_int(rng, tie_idx.size, "i32")
            for r, v in ((0, x), (3, x), (1, xp), (2, xp), (4, z)):
                reps[r][tie_idx] = v
        tol = TOL["f64"] if dt == "f64" else (0.0, 0.0)
        out.append(Problem(reps, dt, *tol, truth={"clean": base, "block": (sl.start, sl.stop),
                                                  "flips": flips, "tie_idx": tie_idx}))
    return tuple(out)


@dataclass
class TaskSpec:
    n: int
    dtype: str
    R: int
    faulty: bool
    seed: int


def cfg4_specs(ntasks: int = 4096, lo: int = 1 << 10, hi: int = 1 << 22,
               fault_frac: float = 0.05, R: int = 3) -> list:
    """Task list of the batched workload: n log-uniform in [lo, hi], dtypes
    f32/f64/i32 at 40/30/30 %, one fault-injected replica in 5% of tasks."""
    rng = rng_for(4)
    ns = np.exp(rng.uniform(math.log(lo), math.log(hi), size=ntasks)).astype(np.int64)
    dts = rng.choice(np.array(["f32", "f64", "i32"]), size=ntasks, p=[0.4, 0.3, 0.3])
    faulty = rng.random(ntasks) < fault_frac
    return [TaskSpec(int(ns[i]), str(dts[i]), R, bool(faulty[i]), i) for i in range(ntasks)]


def task_problem(spec: TaskSpec, config_id: int = 4, flip_rate: float = 1e-4,
                 ulp_frac: float = 0.0) -> Problem:
    """Replicas of one batched / served task."""
    rng = rng_for(config_id, 1 + spec.seed)
    if spec.dtype == "i32":
        base = uniform_int(rng, spec.n, "i32")
    else:
        base = lognormal(rng, spec.n, spec.dtype)
    reps = [base.copy() for _ in range(spec.R)]
    truth = {"clean": base}
    if ulp_frac > 0 and spec.dtype in ("f32", "f64"):
        idx = np.flatnonzero(rng.random(spec.n) < ulp_frac)
        ulp_perturb(reps[1], idx, rng.integers(1, 3, size=idx.size))
    if spec.faulty:
        r = int(rng.integers(0, spec.R))
        fidx = bernoulli_indices(rng, spec.n, flip_rate)
        fbit = rng.integers(0, 8 * reps[r].dtype.itemsize, size=fidx.size)
        bit_flip(reps[r], fidx, fbit)
        truth.update(faulty_replica=r, flip_idx=fidx, flip_bit=fbit)
    tol = TOL.get(spec.dtype, (0.0, 0.0))
    return Problem(reps, spec.dtype, *tol, truth=truth)


@dataclass
class Request:
    t_arrival: float      # seconds from the start of the run
    n: int
    dtype: str
    R: int
    payload: int          # index into the resident payload pool


def cfg5_requests(duration_s: float = 1.0, rate: float = 20000.0, lo: int = 1 << 12,
                  hi: int = 1 << 24, pool: int = 64) -> tuple:
    """Poisson arrivals of vote requests: n log-uniform in [lo, hi], R uniform
    in {3, 5}, dtype f32/f64 50/50.  Returns (requests, payload specs); each
    request votes one of `pool` resident payloads with matching (n, dtype, R)."""
    rng = rng_for(5)
    specs = []
    for p in range(pool):
        n = int(math.exp(rng.uniform(math.log(lo), math.log(hi))))
        specs.append(TaskSpec(n, str(rng.choice(["f32", "f64"])), int(rng.choice([3, 5])),
                              bool(rng.random() < 0.05), 10_000 + p))
    t = 0.0
    reqs = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration_s:
            break
        p = int(rng.integers(0, pool))
        s = specs[p]
        reqs.append(Request(t, s.n, s.dtype, s.R, p))
    return reqs, specs
