"""Pins for the oracle's typed comparison (Sec. IV.D: bit-wise for integers, a
programmer-set maximum difference for floating point).

tests/golden/eq_special.txt lists hand-derived outcomes for +-0, NaN payloads,
+-Inf, overflow of |a-b|, inclusive tolerance boundaries, subnormals (which a
flush-to-zero implementation would get wrong) and the f32 rounding of the
tolerances.  Integer types must reduce to byte equality.
"""
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _cases():
    rows = []
    with open(os.path.join(HERE, "golden", "eq_special.txt")) as f:
        for line in f:
            body, _, why = line.partition("#")
            body = body.strip()
            if not body:
                continue
            dt, a, b, at, rt, exp = body.split()
            rows.append((dt, int(a, 16), int(b, 16), float(at), float(rt), int(exp), why.strip()))
    return rows


CASES = _cases()


def _val(dt, bits):
    if dt == "f32":
        return np.array([bits], dtype=np.uint32).view(np.float32)
    return np.array([bits], dtype=np.uint64).view(np.float64)


@pytest.mark.parametrize("case", CASES, ids=[c[6][:40] for c in CASES])
def test_special_values(case):
    dt, a, b, at, rt, exp, why = case
    assert oracle.eq(dt, _val(dt, a), _val(dt, b), at, rt) == bool(exp), why
    # the comparison is symmetric
    assert oracle.eq(dt, _val(dt, b), _val(dt, a), at, rt) == bool(exp), why


@pytest.mark.parametrize("dt", ["i32", "u32", "i64", "u64", "u8"])
def test_integers_are_bitwise(dt):
    rng = np.random.default_rng(3)
    t = oracle.NP_OF[dt]
    info = np.iinfo(t)
    a = rng.integers(info.min, info.max, size=200, dtype=t, endpoint=True)
    b = a.copy()
    b[::3] ^= t(1)
    for x, y in zip(a, b):
        # tolerances are ignored for integer types
        assert oracle.eq(dt, x, y, 1e30, 1.0) == (x.tobytes() == y.tobytes())


def test_float_identity_and_tolerance_monotone():
    rng = np.random.default_rng(4)
    xs = rng.standard_normal(300).astype(np.float32)
    for x in xs:
        assert oracle.eq("f32", x, x)
        # a relative step of 1e-3 is outside rel 1e-5 but inside rel 1e-2
        y = np.float32(x * np.float32(1.001))
        if abs(x) > 1e-3:
            assert not oracle.eq("f32", x, y, 1e-6, 1e-5)
            assert oracle.eq("f32", x, y, 0.0, 1e-2)
