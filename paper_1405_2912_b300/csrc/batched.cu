// batched.cu -- the batched voter: thousands of tasks of uneven size and mixed
// element type voted by persistent kernels that pull work tiles from a device
// counter, captured together with the statistics reset in one CUDA graph
// (ft_plan_create / ft_vote_batched), and the tile-size / CTA autotuner.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

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

__device__ __noinline__ void copy_out_if_last(const CopyOut &c)
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
    __threadfence_system();
}

// The task of a tile: from the tile map (plans and large batches) ...
struct MapLookup {
    const TaskArgs *tasks;
    const uint32_t *tile_task;
    const unsigned long long *tile_first;
    __device__ __forceinline__ int task_of(unsigned long long tg, int) const { return (int)tile_task[tg]; }
};

// ... or, for a batch of at most 32 tasks, as the last task whose first tile
// is at or before it (one ballot; an empty task shares its first tile with
// the next task, or starts at the group's end, so it is never picked).
struct ScanLookup {
    const TaskArgs *tasks;
    const unsigned long long *tile_first;
    int ntasks;
    __device__ __forceinline__ int task_of(unsigned long long tg, int lane) const
    {
        const unsigned m = __ballot_sync(0xFFFFFFFFu, lane < ntasks && tile_first[lane] <= tg);
        return 31 - __clz((int)m);
    }
};

// ---------------------------------------------------------------------------
// K3: persistent batched voter for one (kind, R) group.  A warp claims the
// next tile with one atomic, looks up its task, votes the tile's 4 KiB blocks
// (and the task's partial last block when the tile holds it), and flushes its
// per-task statistics whenever it moves to another task.  Tiles are claimed
// in increasing order, so a warp meets each task's blocks in increasing order
// and the first index it sees per replica is its minimum.
// ---------------------------------------------------------------------------
template <int K, int R, class Lookup>
__device__ __forceinline__ void vote_tiles(const Lookup &lk, unsigned long long *counter, unsigned long long total_tiles,
                                           int tile_blocks, const uint32_t *s_crc)
{
    const int lane = threadIdx.x & 31;
    CrcLane L;
    L.init(lane);
    LaneStats<R> st;
    st.init();
    int cur = -1;
    ft_stats *cur_stats = nullptr;
    for (;;) {
        unsigned long long tg = 0;
        if (lane == 0) tg = atomicAdd(counter, 1ull);
        tg = __shfl_sync(0xFFFFFFFFu, tg, 0);
        if (tg >= total_tiles) break;
        const int t = lk.task_of(tg, lane);
        const TaskArgs a = lk.tasks[t];
        if (t != cur) {
            if (cur >= 0) st.flush(cur_stats, lane);
            st.init();
            cur = t;
            cur_stats = a.stats;
        }
        const unsigned long long k = tg - lk.tile_first[t];
        const unsigned long long b0 = k * (unsigned long long)tile_blocks;
        const unsigned long long b1 = min(b0 + (unsigned long long)tile_blocks, a.nfull);
        for (unsigned long long b = b0; b < b1; ++b)
            vote_full_block<K, R>(a, b, ~0ull, s_crc, L, st, lane);
        if (a.tail_bytes && a.nfull / tile_blocks == k) {
            LaneStats<R> ts;
            ts.init();
            vote_tail_block<K, R>(a, a.nfull, s_crc, L, ts, lane);
            st.merge(ts);
        }
    }
    if (cur >= 0) st.flush(cur_stats, lane);
}

template <int K, int R, int W>
__global__ void __launch_bounds__(W * 32, 1) batched_kernel(const GroupDev g)
{
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *s_crc = reinterpret_cast<uint32_t *>(smem);
    load_crc_tables<W>(s_crc);
    __syncthreads();
    vote_tiles<K, R>(MapLookup{g.tasks, g.tile_task, g.tile_first}, g.counter, g.total_tiles, g.tile_blocks, s_crc);
    if (g.done_ctas)
        copy_out_if_last(CopyOut{g.done_ctas, nullptr, g.tasks + g.t0, g.t1 - g.t0, false, g.stats_base, g.stats_out});
}

// The same voter for a small batch whose whole group travels in the kernel
// parameters (no upload); its counters and statistics are left reset for the
// next launch by the last CTA.
template <int K, int R, int W>
__global__ void __launch_bounds__(W * 32, 1) batched_small_kernel(const __grid_constant__ SmallGroup g)
{
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *s_crc = reinterpret_cast<uint32_t *>(smem);
    load_crc_tables<W>(s_crc);
    __syncthreads();
    vote_tiles<K, R>(ScanLookup{g.tasks, g.tile_first, g.ntasks}, g.counter, g.total_tiles, g.tile_blocks, s_crc);
    copy_out_if_last(CopyOut{g.done_ctas, g.counter, g.tasks, g.ntasks, true, g.stats_base, g.stats_out});
}

template <int K, int R>
static const void *group_fn(bool small)
{
    return small ? reinterpret_cast<const void *>(batched_small_kernel<K, R, kBatchWarps>)
                 : reinterpret_cast<const void *>(batched_kernel<K, R, kBatchWarps>);
}

template <int K>
static const void *group_fn_k(int R, bool small)
{
    switch (R) {
    case 2: return group_fn<K, 2>(small);
    case 3: return group_fn<K, 3>(small);
    case 4: return group_fn<K, 4>(small);
    case 5: return group_fn<K, 5>(small);
    case 6: return group_fn<K, 6>(small);
    case 7: return group_fn<K, 7>(small);
    case 8: return group_fn<K, 8>(small);
    default: return nullptr;
    }
}

static const void *group_kernel(int kind, int R, bool small = false)
{
    switch (kind) {
    case K_F32: return group_fn_k<K_F32>(R, small);
    case K_F64: return group_fn_k<K_F64>(R, small);
    case K_B1: return group_fn_k<K_B1>(R, small);
    case K_B4: return group_fn_k<K_B4>(R, small);
    case K_B8: return group_fn_k<K_B8>(R, small);
    default: return nullptr;
    }
}

int group_occupancy(int kind, int R, int *sms, int *per_sm)
{
    const void *fn = group_kernel(kind, R);
    if (!fn) return FT_EINVAL;
    const int warps = kBatchWarps;
    return occupancy(fn, warps * 32, kSmemBytes, sms, per_sm);
}

// One CTA per kBatchWarps tiles, at most the resident CTAs of the whole GPU
// and at most max_ctas (0 = no limit).
static int group_grid(const void *fn, unsigned long long total_tiles, int ctas_per_sm, int max_ctas, unsigned *grid)
{
    int sms = 0, per_sm = 0;
    const int rc = occupancy(fn, kBatchWarps * 32, kSmemBytes, &sms, &per_sm);
    if (rc != FT_OK) return rc;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    unsigned long long g = (unsigned long long)sms * per_sm;
    if (max_ctas > 0 && g > (unsigned long long)max_ctas) g = (unsigned long long)max_ctas;
    const unsigned long long need = (total_tiles + kBatchWarps - 1) / kBatchWarps;
    *grid = (unsigned)(g < need ? g : need);
    return FT_OK;
}

int launch_group(const GroupDev &g, int ctas_per_sm, cudaStream_t s, int max_ctas)
{
    const void *fn = group_kernel(g.kind, g.R);
    if (!fn) return FT_EINVAL;
    if (g.total_tiles == 0) return FT_OK;
    unsigned grid = 0;
    const int rc = group_grid(fn, g.total_tiles, ctas_per_sm, max_ctas, &grid);
    if (rc != FT_OK) return rc;
    GroupDev arg = g;
    void *params[] = {&arg};
    const cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(kBatchWarps * 32), params, kSmemBytes, s);
    if (e != cudaSuccess) return cuda_fail(e);
    return check_launch(1);
}

int launch_small_group(const SmallGroup &g, cudaStream_t s, int max_ctas)
{
    const void *fn = group_kernel(g.kind, g.R, true);
    if (!fn || g.ntasks < 1 || g.ntasks > kSmallTasks) return FT_EINVAL;
    if (g.total_tiles == 0) return FT_OK;
    unsigned grid = 0;
    const int rc = group_grid(fn, g.total_tiles, 0, max_ctas, &grid);
    if (rc != FT_OK) return rc;
    void *params[] = {const_cast<SmallGroup *>(&g)};
    const cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(kBatchWarps * 32), params, kSmemBytes, s);
    if (e != cudaSuccess) return cuda_fail(e);
    return check_launch(1);
}

__global__ void batch_reset_kernel(const TaskArgs *tasks, int ntasks, unsigned long long *counters, int ncounters)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = i / (FT_MAX_R + 1), f = i % (FT_MAX_R + 1);
    if (t < ntasks) reset_stats(tasks[t].stats, f);
    if (i < ncounters) counters[i] = 0;
}

int launch_batch_reset(const TaskArgs *tasks, int ntasks, unsigned long long *counters, int ncounters,
                       cudaStream_t s)
{
    const int items = std::max(ntasks * (FT_MAX_R + 1), ncounters);
    if (items == 0) return FT_OK;
    batch_reset_kernel<<<(items + 255) / 256, 256, 0, s>>>(tasks, ntasks, counters, ncounters);
    return check_launch(1);
}

__global__ void stats_scatter_kernel(const ft_stats *src, ft_stats *const *dst, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = i / 18, f = i % 18;
    if (t < n && dst[t]) reinterpret_cast<long long *>(dst[t])[f] = reinterpret_cast<const long long *>(src + t)[f];
}

int launch_stats_scatter(const ft_stats *src, ft_stats *const *dst, int n, cudaStream_t s)
{
    if (n == 0) return FT_OK;
    stats_scatter_kernel<<<(n * 18 + 255) / 256, 256, 0, s>>>(src, dst, n);
    return check_launch(1);
}

// ---------------------------------------------------------------------------
// Host-side batch layout, shared by plans and the server.
// ---------------------------------------------------------------------------
void BatchLayout::build(const std::vector<TaskArgs> &in, int tile_blocks)
{
    tile_blocks_ = tile_blocks;
    tasks.clear();
    groups.clear();
    tile_first.clear();
    tile_task.clear();
    // order tasks by (kind, R), stable, so that each group is contiguous
    std::vector<int> order(in.size());
    for (size_t i = 0; i < in.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return std::make_pair(in[x].kind, in[x].R) < std::make_pair(in[y].kind, in[y].R);
    });
    user_index.assign(order.begin(), order.end());
    for (int idx : order) tasks.push_back(in[idx]);
    tile_first.resize(tasks.size());
    for (size_t t = 0; t < tasks.size();) {
        GroupHost gh;
        gh.kind = tasks[t].kind;
        gh.R = tasks[t].R;
        gh.t0 = (int)t;
        gh.tile0 = tile_task.size();
        unsigned long long g_tiles = 0;
        while (t < tasks.size() && tasks[t].kind == gh.kind && tasks[t].R == gh.R) {
            const TaskArgs &a = tasks[t];
            const unsigned long long nblk = a.nfull + (a.tail_bytes ? 1 : 0);
            const unsigned long long nt = (nblk + tile_blocks - 1) / tile_blocks;
            tile_first[t] = g_tiles;
            for (unsigned long long k = 0; k < nt; ++k) tile_task.push_back((uint32_t)t);
            g_tiles += nt;
            ++t;
        }
        gh.t1 = (int)t;
        gh.tiles = g_tiles;
        groups.push_back(gh);
    }
}

size_t BatchLayout::device_bytes() const
{
    return align(sizeof(TaskArgs) * tasks.size()) + align(8 * tile_first.size()) + align(4 * tile_task.size()) +
           align(16 * groups.size());
}

// Packs the layout into `host` (device_bytes() long) as it must appear at
// device address `dev`, and fills the GroupDev descriptors.
void BatchLayout::pack(uint8_t *host, uint8_t *dev, std::vector<GroupDev> &gd)
{
    size_t off = 0;
    const size_t o_tasks = off;
    off += align(sizeof(TaskArgs) * tasks.size());
    const size_t o_first = off;
    off += align(8 * tile_first.size());
    const size_t o_map = off;
    off += align(4 * tile_task.size());
    const size_t o_cnt = off;
    if (!tasks.empty()) std::memcpy(host + o_tasks, tasks.data(), sizeof(TaskArgs) * tasks.size());
    if (!tile_first.empty()) std::memcpy(host + o_first, tile_first.data(), 8 * tile_first.size());
    if (!tile_task.empty()) std::memcpy(host + o_map, tile_task.data(), 4 * tile_task.size());
    std::memset(host + o_cnt, 0, 16 * groups.size());   // tile counters, then done counters
    gd.clear();
    for (size_t i = 0; i < groups.size(); ++i) {
        const GroupHost &gh = groups[i];
        GroupDev g;
        std::memset(&g, 0, sizeof(g));
        g.tasks = reinterpret_cast<const TaskArgs *>(dev + o_tasks);
        g.tile_task = reinterpret_cast<const uint32_t *>(dev + o_map) + gh.tile0;
        g.tile_first = reinterpret_cast<const unsigned long long *>(dev + o_first);
        g.total_tiles = gh.tiles;
        g.counter = reinterpret_cast<unsigned long long *>(dev + o_cnt) + i;
        g.done_ctas = nullptr;     // no copy-out unless the caller sets it
        g.tile_blocks = tile_blocks_;
        g.kind = gh.kind;
        g.R = gh.R;
        g.t0 = gh.t0;
        g.t1 = gh.t1;
        gd.push_back(g);
    }
    counters_dev = reinterpret_cast<unsigned long long *>(dev + o_cnt);
    tasks_dev = reinterpret_cast<const TaskArgs *>(dev + o_tasks);
}

int launch_groups(const std::vector<GroupDev> &gd, int ctas_per_sm, cudaStream_t s, int max_ctas)
{
    int rc = FT_OK;
    for (const GroupDev &g : gd)
        if ((rc = launch_group(g, ctas_per_sm, s, max_ctas)) != FT_OK) return rc;
    return FT_OK;
}

int launch_batch(const BatchLayout &L, const std::vector<GroupDev> &gd, int ctas_per_sm, cudaStream_t s)
{
    const int rc = launch_batch_reset(L.tasks_dev, (int)L.tasks.size(), L.counters_dev, (int)gd.size(), s);
    if (rc != FT_OK) return rc;
    return launch_groups(gd, ctas_per_sm, s);
}

}  // namespace ftv

// ---------------------------------------------------------------------------
// Plans
// ---------------------------------------------------------------------------
struct ft_plan {
    ftv::BatchLayout layout;
    std::vector<ftv::TaskArgs> args;
    std::vector<ftv::GroupDev> gd;
    uint8_t *dev = nullptr;
    size_t dev_bytes = 0;
    ft_tune tune{0, 0};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int device = 0;
    unsigned long long graph_kernels = 0;   // kernel launches one replay makes
};

namespace ftv {

static int upload_layout(ft_plan *p, int tile_blocks)
{
    p->layout.build(p->args, tile_blocks);
    const size_t need = p->layout.device_bytes();
    if (need > p->dev_bytes) {
        if (p->dev) cudaFree(p->dev);
        p->dev = nullptr;
        p->dev_bytes = 0;
        cudaError_t e = cudaMalloc(&p->dev, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? FT_ENOMEM : cuda_fail(e);
        }
        p->dev_bytes = need;
    }
    std::vector<uint8_t> host(need);
    p->layout.pack(host.data(), p->dev, p->gd);
    cudaError_t e = cudaMemcpy(p->dev, host.data(), need, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? FT_OK : cuda_fail(e);
}

// In-process autotune cache keyed by a coarse signature of the batch.
static std::mutex g_tune_mu;
static std::map<std::string, ft_tune> g_tune_cache;

static std::string signature(const std::vector<TaskArgs> &args)
{
    unsigned long long bytes = 0, blocks = 0;
    std::map<std::pair<int, int>, int> mix;
    for (const TaskArgs &a : args) {
        blocks += a.nfull + (a.tail_bytes ? 1 : 0);
        bytes += (a.nfull * 4096ull + a.tail_bytes) * (a.R + 1);
        mix[{a.kind, a.R}]++;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    char buf[256];
    int lb = 0;
    while ((bytes >> lb) > 1) ++lb;
    std::snprintf(buf, sizeof buf, "dev%d:n%zu:b2^%d:blk%llu", dev, args.size(), lb, blocks / std::max<size_t>(1, args.size()));
    std::string s(buf);
    for (auto &kv : mix) s += ":" + std::to_string(kv.first.first) + "x" + std::to_string(kv.first.second);
    return s;
}

static int time_config(ft_plan *p, const ft_tune &t, cudaStream_t s, float *best_ms)
{
    int rc = upload_layout(p, t.tile_blocks);
    if (rc != FT_OK) return rc;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    rc = launch_batch(p->layout, p->gd, t.ctas_per_sm, s);   // warm-up
    for (int rep = 0; rep < 3 && rc == FT_OK; ++rep) {
        cudaEventRecord(e0, s);
        rc = launch_batch(p->layout, p->gd, t.ctas_per_sm, s);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) rc = cuda_fail(e);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *best_ms = best;
    return rc;
}

static int autotune(ft_plan *p, ft_tune *out)
{
    const std::string key = signature(p->args);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *out = it->second;
            return FT_OK;
        }
    }
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e);
    int max_occ = 1;
    for (const TaskArgs &a : p->args) {
        int sms = 0, occ = 0;
        if (group_occupancy(a.kind, a.R, &sms, &occ) == FT_OK) max_occ = std::max(max_occ, occ);
    }
    const int tiles[] = {1, 2, 4, 8, 16, 32};
    ft_tune best{8, 0};
    float best_ms = 1e30f;
    int rc = FT_OK;
    for (int tb : tiles) {
        for (int cps = 1; cps <= max_occ && rc == FT_OK; ++cps) {
            ft_tune t{tb, cps};
            float ms = 0;
            rc = time_config(p, t, s, &ms);
            if (rc == FT_OK && ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (rc != FT_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    *out = best;
    return FT_OK;
}

// Records the reset and the group kernels into the capture of stream s, the
// group kernels as parallel branches after the reset (each on its own forked
// stream), so that one group's CTAs can start on the SMs that the previous
// group's CTAs leave at its tail.
static int launch_batch_branches(ft_plan *p, cudaStream_t s)
{
    const BatchLayout &L = p->layout;
    int rc = launch_batch_reset(L.tasks_dev, (int)L.tasks.size(), L.counters_dev, (int)p->gd.size(), s);
    if (rc != FT_OK || p->gd.size() <= 1) {
        for (const GroupDev &g : p->gd)
            if (rc == FT_OK) rc = launch_group(g, p->tune.ctas_per_sm, s);
        return rc;
    }
    const size_t k = p->gd.size();
    std::vector<cudaStream_t> side(k, nullptr);
    std::vector<cudaEvent_t> done(k, nullptr);
    cudaEvent_t fork = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(fork, s);
    for (size_t i = 0; i < k && e == cudaSuccess && rc == FT_OK; ++i) {
        if ((e = cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming)) != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(side[i], fork, 0)) != cudaSuccess) break;
        rc = launch_group(p->gd[i], p->tune.ctas_per_sm, side[i]);
        if (rc == FT_OK) e = cudaEventRecord(done[i], side[i]);
    }
    for (size_t i = 0; i < k && e == cudaSuccess && rc == FT_OK; ++i) e = cudaStreamWaitEvent(s, done[i], 0);
    if (e != cudaSuccess && rc == FT_OK) rc = cuda_fail(e);
    for (size_t i = 0; i < k; ++i) {
        if (done[i]) cudaEventDestroy(done[i]);
        if (side[i]) cudaStreamDestroy(side[i]);
    }
    if (fork) cudaEventDestroy(fork);
    return rc;
}

static int capture(ft_plan *p)
{
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e);
    int rc = FT_OK;
    const unsigned long long before = g_launches.load();
    if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) rc = cuda_fail(e);
    if (rc == FT_OK) {
        rc = launch_batch_branches(p, s);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(s, &g);
        if (rc == FT_OK && e != cudaSuccess) rc = cuda_fail(e);
        if (rc == FT_OK) {
            p->graph = g;
            if ((e = cudaGraphInstantiate(&p->exec, g, 0)) != cudaSuccess) rc = cuda_fail(e);
        } else if (g) {
            cudaGraphDestroy(g);
        }
    }
    cudaStreamDestroy(s);
    // the launches recorded during capture did not run; a replay makes them
    p->graph_kernels = g_launches.load() - before;
    g_launches.fetch_sub(p->graph_kernels, std::memory_order_relaxed);
    return rc;
}

}  // namespace ftv

extern "C" {

int ft_plan_create(ft_plan **plan, const ft_vote_desc *tasks, int32_t ntasks, const ft_tune *tune)
{
    using namespace ftv;
    if (!plan || ntasks < 0 || (ntasks > 0 && !tasks)) return FT_EINVAL;
    *plan = nullptr;
    if (tune && ((tune->tile_blocks && (tune->tile_blocks < 1 || tune->tile_blocks > 64)) ||
                 tune->ctas_per_sm < 0 || tune->ctas_per_sm > 8))
        return FT_EINVAL;
    ft_plan *p = new (std::nothrow) ft_plan();
    if (!p) return FT_ENOMEM;
    cudaGetDevice(&p->device);
    for (int i = 0; i < ntasks; ++i) {
        int rc = validate_desc(&tasks[i]);
        if (rc != FT_OK) {
            delete p;
            return rc;
        }
        p->args.push_back(make_task_args(&tasks[i]));
    }
    int rc = FT_OK;
    if (!tune || tune->tile_blocks == 0 || tune->ctas_per_sm == 0) {
        ft_tune t{};
        rc = autotune(p, &t);
        if (rc == FT_OK && tune && tune->tile_blocks) t.tile_blocks = tune->tile_blocks;
        if (rc == FT_OK && tune && tune->ctas_per_sm) t.ctas_per_sm = tune->ctas_per_sm;
        p->tune = t;
    } else {
        p->tune = *tune;
    }
    if (rc == FT_OK) rc = upload_layout(p, p->tune.tile_blocks);
    if (rc == FT_OK) rc = capture(p);
    if (rc != FT_OK) {
        ft_plan_destroy(p);
        return rc;
    }
    *plan = p;
    return FT_OK;
}

int ft_vote_batched(ft_plan *p, ft_stream stream)
{
    if (!p || !p->exec) return FT_EINVAL;
    const cudaError_t e = cudaGraphLaunch(p->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return ftv::cuda_fail(e);
    ftv::g_launches.fetch_add(p->graph_kernels, std::memory_order_relaxed);
    return FT_OK;
}

int ft_vote_batched_nograph(ft_plan *p, ft_stream stream)
{
    if (!p) return FT_EINVAL;
    return ftv::launch_batch(p->layout, p->gd, p->tune.ctas_per_sm, static_cast<cudaStream_t>(stream));
}

int ft_plan_tune(const ft_plan *p, ft_tune *out)
{
    if (!p || !out) return FT_EINVAL;
    *out = p->tune;
    return FT_OK;
}

int ft_plan_destroy(ft_plan *p)
{
    if (!p) return FT_EINVAL;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->dev) cudaFree(p->dev);
    delete p;
    return FT_OK;
}

int ft_vote_many(const ft_vote_desc *descs, int32_t n, ft_stream stream)
{
    if (n < 0 || (n > 0 && !descs)) return FT_EINVAL;
    for (int i = 0; i < n; ++i) {
        const int rc = ftv::vote_desc(&descs[i], static_cast<cudaStream_t>(stream), nullptr);
        if (rc != FT_OK) return rc;
    }
    return FT_OK;
}

}  // extern "C"
