"""The fault-aware runtime estimate of Sec. IV.B (ft_fault_aware_runtime,
ft_rating_record, ft_rating_rank), pinned by the paper's own numbers:
  - a fault probability of 0.75 makes a unit's fault-aware runtime four times
    its fault-free runtime (the Fig. 2 example);
  - a unit twice as fast as any other stays the better choice while its fault
    probability is below 50 %;
  - for a unit three times as fast, the expected crossover is p = 1 - 1/3;
  - in the paper's experiment with injected faults, choosing by the estimate is
    more than twice as fast as abandoning the faster unit after its first
    fault, at a 10 % fault probability (Sec. V.C); reproduced here by a seeded
    simulation of that experiment.
and checked against the plain formula in oracle/rating.py."""
import ctypes
import math

import numpy as np
import pytest

from oracle import rating as ref


@pytest.fixture(scope="module")
def fv():
    from paper_1405_2912_b300 import build
    build.build()
    from paper_1405_2912_b300 import ftvote
    return ftvote


def test_paper_example_p075_four_times(fv):
    # 3 faulty runs out of 4: p = 0.75 -> F = 4 R
    assert fv.ft_fault_probability(1, 4) == 0.75
    assert fv.ft_fault_aware_runtime(2.5, 1, 4) == pytest.approx(10.0, rel=0, abs=1e-12)
    assert ref.fault_aware_runtime(2.5, 1, 4) == 10.0


def test_special_cases(fv):
    assert fv.ft_fault_aware_runtime(3.0, 0, 0) == 3.0          # no runs yet: p = 0
    assert math.isinf(fv.ft_fault_aware_runtime(3.0, 0, 7))     # always faulty: p = 1
    assert math.isnan(fv.ft_fault_aware_runtime(3.0, 8, 7))     # inconsistent counts
    assert fv.ft_fault_probability(5, 5) == 0.0


def test_matches_plain_formula(fv):
    rng = np.random.default_rng(0)
    for _ in range(2000):
        t = int(rng.integers(0, 1000))
        v = int(rng.integers(0, t + 1))
        r = float(rng.uniform(0.001, 1000))
        a, b = fv.ft_fault_aware_runtime(r, v, t), ref.fault_aware_runtime(r, v, t)
        assert (math.isinf(a) and math.isinf(b)) or a == pytest.approx(b, rel=1e-15)


def _rank(fv, units, round_=1, interval=0):
    arr = (fv.ft_unit_rating * len(units))(*[fv.ft_unit_rating(*u) for u in units])
    order = (ctypes.c_int32 * len(units))()
    count = ctypes.c_int32()
    assert fv.ft_rating_rank(arr, len(units), round_, interval, order, ctypes.byref(count)) == fv.FT_OK
    return list(order[:count.value])


@pytest.mark.parametrize("speedup,cross", [(2.0, 0.5), (3.0, 1 - 1 / 3)])
def test_crossover(fv, speedup, cross):
    # unit 0 is `speedup` times faster than unit 1, which never faults
    t = 3000
    for p in np.linspace(0.02, 0.98, 49):
        v = round((1 - p) * t)
        pe = (t - v) / t
        order = _rank(fv, [(1.0, v, t), (speedup, 10, 10)])
        if abs(pe - cross) < 1e-9:
            continue
        assert order[0] == (0 if pe < cross else 1), (speedup, pe)


def test_record_from_vote_stats(fv):
    units = (fv.ft_unit_rating * 3)(fv.ft_unit_rating(1.0, 0, 0), fv.ft_unit_rating(2.0, 0, 0),
                                      fv.ft_unit_rating(3.0, 0, 0))
    st = fv.ft_stats()
    st.mismatch[0], st.mismatch[1], st.mismatch[2] = 0, 5, 0
    who = (ctypes.c_int32 * 3)(2, 0, 0)          # replica 0 from unit 2, replicas 1-2 from unit 0
    assert fv.ft_rating_record(units, 3, who, 3, ctypes.byref(st)) == fv.FT_OK
    assert (units[0].valid_runs, units[0].total_runs) == (1, 2)
    assert (units[2].valid_runs, units[2].total_runs) == (1, 1)
    assert (units[1].valid_runs, units[1].total_runs) == (0, 0)
    bad = (ctypes.c_int32 * 3)(0, 3, 0)
    assert fv.ft_rating_record(units, 3, bad, 3, ctypes.byref(st)) == fv.FT_EINVAL


def test_failed_unit_only_in_check_rounds(fv):
    units = [(1.0, 0, 5), (4.0, 9, 10)]                  # unit 0 always failed
    assert _rank(fv, units, round_=7, interval=10) == [1]
    assert _rank(fv, units, round_=20, interval=10) == [0, 1]     # tried first in a check round
    assert _rank(fv, units, round_=20, interval=0) == [1]


def _simulate(fv, q, rounds, strategy, seed):
    from paper_1405_2912_b300 import rating_sim
    return rating_sim.simulate(q, rounds, strategy, seed)


def test_simulated_injection_experiment(fv):
    # a faulty CPU run costs 1 and is redone on the GPU (3): 1 + 3 q per result
    fa = _simulate(fv, 0.10, 4000, "fault-aware", 1)
    av = _simulate(fv, 0.10, 4000, "avoid", 1)
    assert fa == pytest.approx(1.3, abs=0.06)
    assert av / fa > 2.0                        # "more than 2 times faster" at 10 %
    # below the crossover the estimate keeps the faster, faulty unit ...
    assert _simulate(fv, 0.30, 4000, "fault-aware", 2) == pytest.approx(1.9, abs=0.1)
    # ... and well above it settles on the slower reliable one (3 per result,
    # plus the check rounds that retry the failing unit)
    assert _simulate(fv, 0.90, 4000, "fault-aware", 3) == pytest.approx(3.0, abs=0.15)
