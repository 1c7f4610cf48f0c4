// rating.cpp -- fault-aware runtime estimation of processing units (Sec. IV.B)
// fed by the voter's per-replica statistics.
//
// The paper rates each combination of kernel and processing unit by
//   F_i = R_i / (1 - p_i),
// the fault-free runtime R_i stretched by the expected number of attempts
// until a run is correct, where p_i is the unit's observed fault
// probability.  p_i = 1 gives an infinite F_i; such a unit is only tried again
// at predefined check intervals.  The fault probability is the share of the
// unit's past runs that were faulty: p_i = (t_i - v_i) / t_i for t_i runs of
// which v_i were valid (the printed formula v_i / t_i contradicts the paper's
// own example of p = 0.75 making a unit four times slower, and is read as the
// share of faulty runs).  A unit with no runs yet has p_i = 0.
//
// A vote rates the units that produced its replicas: the run of the unit that
// produced replica r is valid iff the voter found no mismatching element in
// replica r.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "ftvote.h"

extern "C" {

double ft_fault_probability(uint64_t valid_runs, uint64_t total_runs)
{
    if (total_runs == 0 || valid_runs > total_runs) return 0.0;
    return (double)(total_runs - valid_runs) / (double)total_runs;
}

double ft_fault_aware_runtime(double runtime, uint64_t valid_runs, uint64_t total_runs)
{
    if (valid_runs > total_runs) return NAN;
    const double p = ft_fault_probability(valid_runs, total_runs);
    if (total_runs > 0 && valid_runs == 0) return INFINITY;   // p = 1
    return runtime / (1.0 - p);
}

int ft_rating_record(ft_unit_rating *units, int32_t nunits, const int32_t *unit_of_replica, int32_t R,
                     const ft_stats *stats)
{
    if (!units || !unit_of_replica || !stats || R < 1 || R > FT_MAX_R || nunits < 1) return FT_EINVAL;
    for (int r = 0; r < R; ++r)
        if (unit_of_replica[r] < 0 || unit_of_replica[r] >= nunits) return FT_EINVAL;
    for (int r = 0; r < R; ++r) {
        ft_unit_rating &u = units[unit_of_replica[r]];
        u.total_runs += 1;
        if (stats->mismatch[r] == 0) u.valid_runs += 1;
    }
    return FT_OK;
}

int ft_rating_rank(const ft_unit_rating *units, int32_t nunits, uint64_t round, uint64_t check_interval,
                   int32_t *order, int32_t *count)
{
    if (!units || !order || !count || nunits < 1) return FT_EINVAL;
    // Units whose F is infinite are left out, except in check rounds, where
    // they come first so that they actually run and show whether they still
    // fail.  The others follow by increasing F (insertion sort, stable: ties
    // keep the unit order).
    const bool check = check_interval > 0 && round % check_interval == 0;
    int k = 0;
    for (int i = 0; i < nunits; ++i) {
        const double f = ft_fault_aware_runtime(units[i].runtime, units[i].valid_runs, units[i].total_runs);
        if (std::isnan(f)) return FT_EINVAL;
        if (std::isinf(f) && check) order[k++] = i;
    }
    const int first_finite = k;
    for (int i = 0; i < nunits; ++i) {
        const double f = ft_fault_aware_runtime(units[i].runtime, units[i].valid_runs, units[i].total_runs);
        if (std::isinf(f)) continue;
        int j = k;
        while (j > first_finite) {
            const ft_unit_rating &o = units[order[j - 1]];
            const double g = ft_fault_aware_runtime(o.runtime, o.valid_runs, o.total_runs);
            if (g <= f) break;
            order[j] = order[j - 1];
            --j;
        }
        order[j] = i;
        ++k;
    }
    *count = k;
    return FT_OK;
}

}  // extern "C"
