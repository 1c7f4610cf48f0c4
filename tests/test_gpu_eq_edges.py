"""The GPU's float comparison at the edges of its accepted domain.

The kernels do not evaluate the comparison rule (Sec. IV.D: floats are equal
when they differ by at most a programmer-set maximum) literally: for f32 they
compare |a - b| with max(u_a, u_b), u_x = min(max(abs_tol, rel_tol * |x|),
FLT_MAX), which equals the rule only inside the domain the host accepts
(0 <= rel_tol <= 1, abs_tol finite once rounded to the element type).  These
tests pin that reformulation where random data never goes:

- every in-domain row of tests/golden/eq_special.txt (hand-derived outcomes:
  +-0, NaN payloads, +-Inf, overflowing differences, inclusive boundaries,
  subnormals, the rounding of the tolerances) voted as R = 2, 3 and 5
  replicas, in a full 4 KiB block (the fast forms) and in the partial last
  block (the exact form), each result checked against the row and against the
  oracle;
- the largest tolerances the host accepts (rel_tol = 1, abs_tol = FLT_MAX or
  1e308) on operands near +-FLT_MAX / +-DBL_MAX whose differences overflow,
  mixed with infinities, NaNs, zeros and subnormals, against the oracle."""
import os

import numpy as np
import pytest

import oracle

from _gpu import assert_same, gpu_vote

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
FLT_MAX = float(np.finfo(np.float32).max)


def _rows():
    rows = []
    with open(os.path.join(HERE, "golden", "eq_special.txt")) as f:
        for line in f:
            body, _, why = line.partition("#")
            body = body.strip()
            if not body:
                continue
            dt, a, b, at, rt, exp = body.split()
            at, rt = float(at), float(rt)
            # the domain ft_vote accepts
            tol_t = np.float32 if dt == "f32" else np.float64
            with np.errstate(over="ignore"):
                in_domain = 0.0 <= rt <= 1.0 and at >= 0.0 and np.isfinite(tol_t(at))
            if in_domain:
                rows.append((dt, int(a, 16), int(b, 16), at, rt, int(exp), why.strip()))
    return rows


ROWS = _rows()


def _bits_to(dt, bits):
    u = np.uint32 if dt == "f32" else np.uint64
    return np.array(bits, dtype=u).view(np.float32 if dt == "f32" else np.float64)


@pytest.mark.parametrize("row", ROWS, ids=[r[6][:40] for r in ROWS])
@pytest.mark.parametrize("R", [2, 3, 5])
def test_golden_rows_through_ft_vote(row, R):
    dt, a_bits, b_bits, at, rt, exp, why = row
    itemsize = 4 if dt == "f32" else 8
    per_block = 4096 // itemsize
    n = 2 * per_block + 37                       # two full blocks and a partial one
    pos = [3, per_block - 1, per_block + 17, 2 * per_block + 5, n - 1]
    a = np.zeros(n, dtype=np.uint32 if dt == "f32" else np.uint64)
    a[:] = a_bits
    b = a.copy()
    b[pos] = b_bits
    x, y = _bits_to(dt, a), _bits_to(dt, b)
    # replica 1 differs at `pos`; for R > 2 the others follow replica 0 or 1
    # so that replica 0's support decides the outcome the row states
    reps = [x, y] + [x if k % 2 == 0 else y for k in range(R - 2)]
    g = gpu_vote(reps, dt, at, rt)
    ref = oracle.vote(reps, dt, at, rt)
    assert_same(g, ref, R)
    if R == 2:
        # DMR: replica 0 always wins; replica 1 mismatches where not equal
        assert int(g["mismatch"][1]) == (0 if exp else len(pos)), why
        assert g["no_majority"] == (0 if exp else len(pos)), why


def _extreme_pool(dt):
    if dt == "f32":
        f = np.float32
        big = f(FLT_MAX)
        vals = [big, -big, np.nextafter(big, f(0)), -np.nextafter(big, f(0)), f(1e38), f(-1e38),
                f(3e38), f(-3e38), f(np.inf), f(-np.inf), f(np.nan), f(0.0), f(-0.0),
                np.frombuffer(np.uint32(1).tobytes(), dtype=f)[0], f(1.0), f(-1.0), f(1.5e38)]
        return np.array(vals, dtype=f)
    d = np.float64
    big = d(np.finfo(d).max)
    vals = [big, -big, np.nextafter(big, d(0)), -np.nextafter(big, d(0)), d(1e308), d(-1e308),
            d(1.7e308), d(-1.7e308), d(np.inf), d(-np.inf), d(np.nan), d(0.0), d(-0.0),
            np.frombuffer(np.uint64(1).tobytes(), dtype=d)[0], d(1.0), d(-1.0), d(9e307)]
    return np.array(vals, dtype=d)


@pytest.mark.parametrize("dt,abs_tol", [("f32", FLT_MAX), ("f32", 0.0), ("f64", 1e308), ("f64", 0.0)])
@pytest.mark.parametrize("R", [2, 3, 5])
def test_largest_tolerances_on_overflowing_differences(dt, abs_tol, R):
    rng = np.random.default_rng(100 + R + (0 if dt == "f32" else 50) + (1 if abs_tol else 0))
    pool = _extreme_pool(dt)
    itemsize = pool.itemsize
    n = 3 * (4096 // itemsize) + 101
    base = pool[rng.integers(0, pool.size, size=n)]
    reps = []
    for r in range(R):
        x = base.copy()
        # each replica replaces a third of the elements with another pool value
        idx = rng.random(n) < 0.33
        x[idx] = pool[rng.integers(0, pool.size, size=int(idx.sum()))]
        reps.append(x)
    g = gpu_vote(reps, dt, abs_tol, 1.0)
    assert_same(g, oracle.vote(reps, dt, abs_tol, 1.0), R)
