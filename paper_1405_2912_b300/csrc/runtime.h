// runtime.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <atomic>
#include <cstddef>
#include <cuda_runtime.h>

#include "ftvote.h"

namespace ftv {

struct TaskArgs;

// Optional launch override of the single-task voter (tests and tuning); zero
// fields keep the library's choice.
struct VoteLaunch {
    int ctas_per_sm;   // 0 = occupancy limit
    int warps;         // warps per CTA (f32 R = 3: 4, 8 or 16; other kinds: the shapes built for them)
    int sub_batch;     // 16-byte vectors per lane per sub-batch (f32 R = 3: 4 or 8)
    int stats_mode;    // 1 = statistics reset kernel + voter, 2 = one kernel with a statistics slot
    int small_form;    // votes of 1185..32768 blocks: 1 = 16 warps with the SMALL block form, 2 = without
    int max_ctas;      // 0 = no cap beyond the occupancy limit
};

extern std::atomic<unsigned long long> g_launches;
extern thread_local int g_last_cuda;

int cuda_fail(cudaError_t e);
int check_launch(int nlaunch);
int occupancy(const void *fn, int threads, size_t smem, int *sms, int *per_sm);
size_t dtype_size(int dtype);
int dtype_kind(int dtype);
int validate_desc(const ft_vote_desc *d);
TaskArgs make_task_args(const ft_vote_desc *d);
int vote_desc(const ft_vote_desc *desc, cudaStream_t s, const VoteLaunch *cfg);
// The single-task voter on an already validated task, through a statistics
// slot (one launch, programmatic dependent of the stream's previous kernel):
// the slot is copied to a.stats at the end.  FT_EAGAIN, with nothing
// launched, for an empty task or when every slot is taken.  Not for a stream
// that is being captured.
// With flag set, the kernel writes seq to *flag (host-mapped) after the
// statistics have reached a.stats.
int vote_task_slot(const TaskArgs &a, cudaStream_t s, const VoteLaunch *cfg, unsigned long long *flag = nullptr,
                   unsigned long long seq = 0);
// The same in two steps, for a caller that launches several votes and must
// know before the first that each gets a statistics slot: reserve_vote_slot
// takes a free slot of the current device (-1 when all are taken),
// vote_task_reserved launches a task on it, which must not be empty (the
// kernel frees the slot at its end; a failed launch frees it at once), and
// release_vote_slot
// frees a reserved slot that no vote was launched on.
int reserve_vote_slot();
void release_vote_slot(int slot);
int vote_task_reserved(const TaskArgs &a, cudaStream_t s, const VoteLaunch *cfg, int slot, unsigned long long *flag,
                       unsigned long long seq);

// With lazy module loading (the CUDA default) a kernel is loaded at its first
// launch, 0.1-0.4 ms of host time on B300.  These load, and size for the CRC
// tables' shared memory, every single-task voter shape the library picks by
// itself (and create the device's statistics slots), and every batched and
// small-batch kernel of the shapes the server launches, so that a long-lived
// caller (the server) pays that once at creation instead of inside a request.
int preload_vote_kernels();
int preload_group_kernels();

// One (element kind, R) group of a batch, as the batched kernel sees it.
// tasks[t] for t in [t0, t1) belong to the group; the group's work is split
// into total_tiles tiles of tile_blocks 4 KiB blocks; tile_task[g] is the task
// of the group's tile g and tile_first[t] the group tile where task t starts.
// With done_ctas set, the group's last CTA to finish copies the statistics of
// tasks t0..t1-1 to stats_out[tasks[t].stats - stats_base] (host-mapped
// memory), so that no download follows the kernel.
struct GroupDev {
    const TaskArgs *tasks;
    const uint32_t *tile_task;
    const unsigned long long *tile_first;
    unsigned long long total_tiles;
    unsigned long long *counter;     // tile dispenser, zeroed before the launch
    unsigned long long *done_ctas;   // CTAs finished, zeroed before the launch; nullptr: no copy-out
    const ft_stats *stats_base;      // the batch's statistics array (device)
    ft_stats *stats_out;             // its host-mapped copy
    // Completion of each task on its own (flag_out set): the warp whose tiles
    // complete task t copies its statistics to stats_out[i] and then writes
    // seq to flag_out[i] (host-mapped), i = tasks[t].stats - stats_base;
    // tiles_done[i] counts the task's voted tiles and is zero at launch.
    unsigned long long *tiles_done;
    unsigned long long *flag_out;
    unsigned long long seq;
    int32_t tile_blocks;
    int32_t kind;
    int32_t R;
    int32_t t0, t1;
    int32_t warps;                   // launch shape: warps per CTA (8, 12, 16; 0 = 16)
    int32_t pf;                      // and the L2 prefetch of the tile's next block
    int32_t pad_;
};

// Reset the statistics of tasks[0..ntasks) and zero ncounters counters.
int launch_batch_reset(const TaskArgs *tasks, int ntasks, unsigned long long *counters, int ncounters,
                       cudaStream_t s);
// Launch the persistent batched voter for one group.
int launch_group(const GroupDev &g, int ctas_per_sm, cudaStream_t s, int max_ctas = 0);
// Resident CTAs per SM of the batched kernel for (kind, R) with `warps` warps
// per CTA (0 = 16), and the SM count.
int group_occupancy(int kind, int R, int *sms, int *per_sm, int warps = 0);
// Tile size of a batch whose caller left it to the library: 8 blocks, halved
// while the batch's total_blocks would make fewer tiles than the kernel has
// warps in one wave (wave_warps), so that a small batch is spread over as
// many warps as it has blocks instead of being walked block after block by a
// few warps.
int auto_tile_blocks(unsigned long long total_blocks, unsigned long long wave_warps);
// Copy stats of tasks[i] to user[i] where user[i] is not null (server).
int launch_stats_scatter(const ft_stats *src, ft_stats *const *dst, int n, cudaStream_t s);
int digest(const void *buf, unsigned long long nbytes, uint32_t block_bytes, uint32_t *out, cudaStream_t s);

}  // namespace ftv
