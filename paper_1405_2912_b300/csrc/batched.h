// batched.h -- host-side layout of a batch of vote tasks in device memory:
// the task table ordered by (kind, R) group, each task's first tile, and the
// tile -> task map that the persistent batched kernel reads.
#pragma once

#include <cstdint>
#include <vector>

#include "common.cuh"
#include "runtime.h"

namespace ftv {

// Launch shapes of the batched kernels: warps per CTA (8, 12 or 16) and
// whether a warp prefetches its tile's next block into L2.  A plan's
// autotuner picks one per (kind, R) group; without tuning a group runs 16
// warps without prefetch, which on the batch of 4096 tasks of 4 KiB .. 16 MiB
// measured 0.621 M tasks/s (6.48 TB/s) against 0.599 M (6.25 TB/s) with the
// single-task shapes.  The small-batch kernel is built with 8 and 16 warps.
constexpr int kBatchWarps = 16;
constexpr int kShapeWarps[] = {8, 12, 16};

// The kernel of a (kind, R) group in one launch shape: the plan's persistent
// kernel (small = false) or the small-batch kernel whose group travels in its
// parameters (small = true; built without the prefetch).  Each warp count's
// kernels are instantiated in a translation unit of their own
// (batched_w8.cu, batched_w12.cu, batched_w16.cu) so that they compile in
// parallel; nullptr for a shape that is not built.
template <int W>
const void *group_fn_w(int kind, int R, bool pf, bool small);
template <>
const void *group_fn_w<8>(int kind, int R, bool pf, bool small);
template <>
const void *group_fn_w<12>(int kind, int R, bool pf, bool small);
template <>
const void *group_fn_w<16>(int kind, int R, bool pf, bool small);
const void *group_kernel(int kind, int R, int warps, bool pf, bool small);

// A (kind, R) group of a small batch, passed whole as the kernel parameter:
// no upload precedes the launch.  tile_first[t] is task t's first tile (an
// empty task's equals the next one's); counter and done_ctas are zero and
// each task's statistics (0, -1) at launch, and the group kernel's last CTA
// leaves them so after copying the statistics to stats_out.
constexpr int kSmallTasks = 16;
struct SmallGroup {
    TaskArgs tasks[kSmallTasks];
    unsigned long long tile_first[kSmallTasks];
    unsigned long long total_tiles;
    unsigned long long *counter;
    unsigned long long *done_ctas;
    const ft_stats *stats_base;      // the slot's statistics array (device)
    ft_stats *stats_out;             // its host-mapped copy
    // per-task completion as GroupDev's (flag_out set); the task's last warp
    // also puts its statistics and tiles_done entry back to their initial values
    unsigned long long *tiles_done;
    unsigned long long *flag_out;
    unsigned long long seq;
    int32_t ntasks;
    int32_t tile_blocks;
    int32_t kind;
    int32_t R;
    int32_t warps;                   // 8 or 16 (0 = 16)
    int32_t pad_;
};
int launch_small_group(const SmallGroup &g, cudaStream_t s, int max_ctas = 0);

// The whole batch as one persistent kernel (batched_mixed.cu): the tiles of
// every group back to back (tile_task), and each task's first tile in that
// sequence.  counter is zeroed before the launch.
struct MixedDev {
    const TaskArgs *tasks;
    const uint32_t *tile_task;
    const unsigned long long *tile_first_global;
    unsigned long long total_tiles;
    unsigned long long *counter;
    int32_t tile_blocks;
    int32_t pad_;
};
int launch_mixed(const MixedDev &g, int ctas_per_sm, cudaStream_t s);

struct GroupHost {
    int kind, R;
    int t0, t1;                 // task range in the ordered table
    size_t tile0;               // offset of the group's tiles in tile_task
    unsigned long long tiles;
};

struct BatchLayout {
    std::vector<TaskArgs> tasks;                  // ordered by (kind, R)
    std::vector<int> user_index;                  // tasks[i] is the caller's task user_index[i]
    std::vector<GroupHost> groups;
    std::vector<unsigned long long> tile_first;   // per ordered task: first tile in its group
    std::vector<uint32_t> tile_task;              // per tile (all groups back to back)
    std::vector<unsigned long long> tile_first_global;   // per ordered task: first tile in tile_task
    int tile_blocks_ = 8;
    // set by pack(): device addresses of the table and the counters
    const TaskArgs *tasks_dev = nullptr;
    unsigned long long *counters_dev = nullptr;
    MixedDev mixed{};                             // the batch as one kernel (counter: counters_dev[0])

    static size_t align(size_t x) { return (x + 255) & ~size_t(255); }
    void build(const std::vector<TaskArgs> &in, int tile_blocks);
    size_t device_bytes() const;
    void pack(uint8_t *host, uint8_t *dev, std::vector<GroupDev> &gd);
};

// The statistics / tile-counter reset followed by the group kernels.
int launch_batch(const BatchLayout &L, const std::vector<GroupDev> &gd, int ctas_per_sm, cudaStream_t s);
// The group kernels alone, for callers whose upload already carries zeroed
// counters and initialised statistics.
int launch_groups(const std::vector<GroupDev> &gd, int ctas_per_sm, cudaStream_t s, int max_ctas = 0);

}  // namespace ftv
