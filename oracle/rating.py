"""Plain fault-aware runtime estimate of Sec. IV.B (test infrastructure).

Only the tests may import this module; the product's implementation is the C
library's ft_fault_aware_runtime / ft_rating_rank.

  p_i = (t_i - v_i) / t_i          share of the unit's past runs that were faulty
                                   (0 for a unit that has not run)
  F_i = R_i / (1 - p_i)            fault-free runtime times the expected number
                                   of attempts until a run is correct
  p_i = 1  ->  F_i = infinity
"""
import math


def fault_probability(valid, total):
    return 0.0 if total == 0 else (total - valid) / total


def fault_aware_runtime(runtime, valid, total):
    p = fault_probability(valid, total)
    if p == 1.0:
        return math.inf
    return runtime / (1.0 - p)
