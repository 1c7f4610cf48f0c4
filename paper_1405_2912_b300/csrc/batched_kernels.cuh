// batched_kernels.cuh -- the persistent batched voter kernels (K3), shared by
// the translation units that instantiate them for each launch shape: warps
// per CTA and whether a warp prefetches its tile's next block into L2.
#pragma once

#include "batched.h"
#include "common.cuh"
#include "runtime.h"

namespace ftv {

// Statistics hand-off at the end of a group kernel.  The last CTA to finish
// copies the statistics of tasks[0..ntasks) to stats_out[tasks[t].stats -
// stats_base] (host-mapped memory), so that no download follows the kernel.
// Every thread's statistics atomics are made visible at device scope before
// its CTA is counted, and the last CTA reads the final values from L2.  With
// `reset`, it then puts each statistics word back to its initial value and
// zeroes the tile and done counters, leaving the buffers ready for the next
// launch without an upload.
struct CopyOut {
    unsigned long long *done_ctas;
    unsigned long long *counter;   // zeroed when reset
    const TaskArgs *tasks;
    int ntasks;
    bool reset;
    const ft_stats *stats_base;
    ft_stats *stats_out;
};

static __device__ __noinline__ void copy_out_if_last(const CopyOut &c)
{
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(c.done_ctas, 1ull) == (unsigned long long)gridDim.x - 1ull;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    constexpr int kWords = (int)(sizeof(ft_stats) / 8);   // mismatch[8], first[8], no_majority, first
    static_assert(kWords == 2 * FT_MAX_R + 2, "ft_stats layout");
    const int n = c.ntasks * kWords;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int w = i % kWords;
        ft_stats *src = c.tasks[i / kWords].stats;
        unsigned long long *word = reinterpret_cast<unsigned long long *>(src) + w;
        reinterpret_cast<unsigned long long *>(c.stats_out + (src - c.stats_base))[w] = __ldcg(word);
        if (c.reset) *word = (w < FT_MAX_R || w == 2 * FT_MAX_R) ? 0ull : ~0ull;   // counts 0, first indices -1
    }
    if (c.reset && threadIdx.x == 0) {
        *c.counter = 0;
        *c.done_ctas = 0;
    }
    // no system-scope fence: the host reads stats_out only once the event
    // recorded after the batch's kernels has completed, which makes the
    // kernel's writes to host memory visible to it
}

// Completion of each task on its own (the server, flag_out set): the warp
// whose tiles complete a task copies the task's statistics to stats_out[i]
// and then writes seq to flag_out[i], both host-mapped, i = the task's index
// in the statistics array.  The host then sees the request done while the rest
// of its batch is still voting.  tiles_done[i] is zero at launch; with
// `reset`, the last warp puts it and the statistics back to their initial
// values for the next launch.
struct TaskDone {
    unsigned long long *tiles_done;
    const ft_stats *stats_base;
    ft_stats *stats_out;
    unsigned long long *flag_out;   // nullptr: off
    unsigned long long seq;
    bool reset;
};

// Called by every lane of a warp after it has flushed its statistics of the
// task whose statistics are `stats`: adds the warp's `tiles` of the task to
// its count and, if that completes the task's `need` tiles, hands it off.
static __device__ __noinline__ void finish_task(const TaskDone &d, ft_stats *stats, unsigned long long tiles,
                                                unsigned long long need, int lane)
{
    const size_t i = (size_t)(stats - d.stats_base);
    int last = 0;
    if (lane == 0) {
        __threadfence();   // lane 0 made the statistics atomics of the flush
        last = atomicAdd(d.tiles_done + i, tiles) + tiles == need;
    }
    if (!__shfl_sync(0xFFFFFFFFu, last, 0)) return;
    // every other warp that voted tiles of the task counted them after its
    // own flush: their statistics are final in L2
    __threadfence();
    constexpr int kWords = (int)(sizeof(ft_stats) / 8);
    if (lane < kWords) {
        unsigned long long *w = reinterpret_cast<unsigned long long *>(stats) + lane;
        reinterpret_cast<unsigned long long *>(d.stats_out + i)[lane] = __ldcg(w);
        if (d.reset) *w = (lane < FT_MAX_R || lane == 2 * FT_MAX_R) ? 0ull : ~0ull;
    }
    if (lane == 0 && d.reset) d.tiles_done[i] = 0;
    // each lane's writes reach the host (and the resets the device) before the flag
    __threadfence_system();
    __syncwarp();
    if (lane == 0) *reinterpret_cast<volatile unsigned long long *>(d.flag_out + i) = d.seq;
}

// The task of a tile: from the tile map (plans and large batches) ...
struct MapLookup {
    const TaskArgs *tasks;
    const uint32_t *tile_task;
    const unsigned long long *tile_first;
    int t_end;                       // one past the group's last task
    unsigned long long total;        // the group's tiles
    __device__ __forceinline__ int task_of(unsigned long long tg, int) const { return (int)tile_task[tg]; }
    __device__ __forceinline__ unsigned long long tiles_of(int t) const
    {
        return (t + 1 < t_end ? tile_first[t + 1] : total) - tile_first[t];
    }
};

// ... or, for a batch of at most 32 tasks, as the last task whose first tile
// is at or before it (one ballot; an empty task shares its first tile with
// the next task, or starts at the group's end, so it is never picked).
struct ScanLookup {
    const TaskArgs *tasks;
    const unsigned long long *tile_first;
    int ntasks;
    unsigned long long total;
    __device__ __forceinline__ int task_of(unsigned long long tg, int lane) const
    {
        const unsigned m = __ballot_sync(0xFFFFFFFFu, lane < ntasks && tile_first[lane] <= tg);
        return 31 - __clz((int)m);
    }
    __device__ __forceinline__ unsigned long long tiles_of(int t) const
    {
        return (t + 1 < ntasks ? tile_first[t + 1] : total) - tile_first[t];
    }
};

// ---------------------------------------------------------------------------
// K3: persistent batched voter for one (kind, R) group.  A warp claims the
// next tile with one atomic, looks up its task, votes the tile's 4 KiB blocks
// (and the task's partial last block when the tile holds it), and flushes its
// per-task statistics whenever it moves to another task.  Tiles are claimed
// in increasing order, so a warp meets each task's blocks in increasing order
// and the first index it sees per replica is its minimum.  PF: lanes 0..R-1
// prefetch the tile's next block into L2 while the warp votes the current one.
// ---------------------------------------------------------------------------
// STATIC: warp w of the grid takes tiles w, w + (warps in the grid), ...
// instead of claiming them, which saves a round trip to the counter per tile
// where the tiles are too few for their sizes to need balancing.
template <int K, int R, bool PF, bool STATIC, class Lookup, bool SMALL = false>
__device__ __forceinline__ void vote_tiles(const Lookup &lk, unsigned long long *counter, unsigned long long total_tiles,
                                           int tile_blocks, const uint32_t *s_crc, const TaskDone &td)
{
    const int lane = threadIdx.x & 31;
    CrcLane L;
    L.init(lane);
    LaneStats<R> st;
    st.init();
    int cur = -1;
    ft_stats *cur_stats = nullptr;
    unsigned long long cur_tiles = 0;   // tiles of task cur this warp voted
    const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    unsigned long long next = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (;;) {
        unsigned long long tg = 0;
        if constexpr (STATIC) {
            tg = next;
            next += nwarps;
        } else {
            if (lane == 0) tg = atomicAdd(counter, 1ull);
            tg = __shfl_sync(0xFFFFFFFFu, tg, 0);
        }
        if (tg >= total_tiles) break;
        const int t = lk.task_of(tg, lane);
        const TaskArgs a = lk.tasks[t];
        if (t != cur) {
            if (cur >= 0) {
                st.flush(cur_stats, lane);
                if (td.flag_out) finish_task(td, cur_stats, cur_tiles, lk.tiles_of(cur), lane);
            }
            st.init();
            cur = t;
            cur_stats = a.stats;
            cur_tiles = 0;
        }
        ++cur_tiles;
        const unsigned long long k = tg - lk.tile_first[t];
        const unsigned long long b0 = k * (unsigned long long)tile_blocks;
        const unsigned long long b1 = min(b0 + (unsigned long long)tile_blocks, a.nfull);
        for (unsigned long long b = b0; b < b1; ++b)
            vote_full_block<K, R, kSubBatch<K, R>, SMALL>(a, b, (PF && b + 1 < b1) ? b + 1 : ~0ull, s_crc, L, st,
                                                          lane);
        if (a.tail_bytes && a.nfull / tile_blocks == k) {
            LaneStats<R> ts;
            ts.init();
            vote_tail_block<K, R>(a, a.nfull, s_crc, L, ts, lane);
            st.merge(ts);
        }
    }
    if (cur >= 0) {
        st.flush(cur_stats, lane);
        if (td.flag_out) finish_task(td, cur_stats, cur_tiles, lk.tiles_of(cur), lane);
    }
}

template <int K, int R, int W, bool PF>
__global__ void __launch_bounds__(W * 32, 1) batched_kernel(const GroupDev g)
{
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *s_crc = reinterpret_cast<uint32_t *>(smem);
    load_crc_tables<W>(s_crc);
    __syncthreads();
    vote_tiles<K, R, PF, false>(MapLookup{g.tasks, g.tile_task, g.tile_first, g.t1, g.total_tiles}, g.counter,
                                g.total_tiles, g.tile_blocks, s_crc,
                                TaskDone{g.tiles_done, g.stats_base, g.stats_out, g.flag_out, g.seq, false});
    if (g.done_ctas)
        copy_out_if_last(CopyOut{g.done_ctas, nullptr, g.tasks + g.t0, g.t1 - g.t0, false, g.stats_base, g.stats_out});
}

// The same voter for a small batch whose whole group travels in the kernel
// parameters (no upload); its counters and statistics are left reset for the
// next launch by the last CTA.  Its warps take their tiles in a fixed order
// (the batch is small enough not to need balancing).
template <int K, int R, int W>
__global__ void __launch_bounds__(W * 32, 1) batched_small_kernel(const __grid_constant__ SmallGroup g)
{
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *s_crc = reinterpret_cast<uint32_t *>(smem);
    const ScanLookup lk{g.tasks, g.tile_first, g.ntasks, g.total_tiles};
    {
        // ask L2 for the first block of the warp's first tile while the CRC
        // tables are copied
        const int lane = threadIdx.x & 31;
        const unsigned long long tg = (unsigned long long)blockIdx.x * W + (threadIdx.x >> 5);
        if (tg < g.total_tiles) {
            const int t = lk.task_of(tg, lane);
            const TaskArgs &a = g.tasks[t];
            const unsigned long long b0 = (tg - g.tile_first[t]) * (unsigned long long)g.tile_blocks;
            if (lane < R && b0 < a.nfull) prefetch_l2(a.rep[lane] + b0 * kBlockBytes, kBlockBytes);
        }
    }
    load_crc_tables<W>(s_crc);
    __syncthreads();
    // the 8-warp instance serves groups of at most a few tiles per warp: the
    // SMALL block form (see vote_full_block)
    vote_tiles<K, R, false, true, ScanLookup, W == 8>(
        lk, g.counter, g.total_tiles, g.tile_blocks, s_crc,
        TaskDone{g.tiles_done, g.stats_base, g.stats_out, g.flag_out, g.seq, true});
    // with per-task completion the tasks' last warps have handed off and reset
    // the statistics already; the last CTA still resets the counters
    copy_out_if_last(CopyOut{g.done_ctas, g.counter, g.tasks, g.flag_out ? 0 : g.ntasks, true, g.stats_base,
                             g.stats_out});
}

template <int K, int R, int W, bool PF, bool SMALL>
const void *group_fn_kr()
{
    if constexpr (SMALL) return reinterpret_cast<const void *>(batched_small_kernel<K, R, W>);
    else return reinterpret_cast<const void *>(batched_kernel<K, R, W, PF>);
}

// The switch over (kind, R) of one shape, for those translation units.
template <int W, bool PF, bool SMALL>
const void *group_fn_shape(int kind, int R)
{
#define FTV_GROUP_R(K)                                        \
    switch (R) {                                              \
    case 2: return group_fn_kr<K, 2, W, PF, SMALL>();         \
    case 3: return group_fn_kr<K, 3, W, PF, SMALL>();         \
    case 4: return group_fn_kr<K, 4, W, PF, SMALL>();         \
    case 5: return group_fn_kr<K, 5, W, PF, SMALL>();         \
    case 6: return group_fn_kr<K, 6, W, PF, SMALL>();         \
    case 7: return group_fn_kr<K, 7, W, PF, SMALL>();         \
    case 8: return group_fn_kr<K, 8, W, PF, SMALL>();         \
    default: return nullptr;                                  \
    }
    switch (kind) {
    case K_F32: FTV_GROUP_R(K_F32)
    case K_F64: FTV_GROUP_R(K_F64)
    case K_B1: FTV_GROUP_R(K_B1)
    case K_B4: FTV_GROUP_R(K_B4)
    case K_B8: FTV_GROUP_R(K_B8)
    default: return nullptr;
    }
#undef FTV_GROUP_R
}

}  // namespace ftv
