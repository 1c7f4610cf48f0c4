// batched.cu -- the batched voter: thousands of tasks of uneven size and mixed
// element type voted by persistent kernels that pull work tiles from a device
// counter, captured together with the statistics reset in one CUDA graph
// (ft_plan_create / ft_vote_batched), and the autotuner of the tile size and
// of each group's launch shape.
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

const void *group_kernel(int kind, int R, int warps, bool pf, bool small)
{
    switch (warps) {
    case 8: return group_fn_w<8>(kind, R, pf, small);
    case 12: return group_fn_w<12>(kind, R, pf, small);
    case 0:
    case 16: return group_fn_w<16>(kind, R, pf, small);
    default: return nullptr;
    }
}

static int shape_warps(int warps) { return warps ? warps : kBatchWarps; }

int group_occupancy(int kind, int R, int *sms, int *per_sm, int warps)
{
    const int w = shape_warps(warps);
    const void *fn = group_kernel(kind, R, w, false, false);
    if (!fn) return FT_EINVAL;
    return occupancy(fn, w * 32, kSmemBytes, sms, per_sm);
}

// One CTA per `warps` tiles, at most the resident CTAs of the whole GPU and at
// most max_ctas (0 = no limit).
static int group_grid(const void *fn, int warps, unsigned long long total_tiles, int ctas_per_sm, int max_ctas,
                      unsigned *grid)
{
    int sms = 0, per_sm = 0;
    const int rc = occupancy(fn, warps * 32, kSmemBytes, &sms, &per_sm);
    if (rc != FT_OK) return rc;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    unsigned long long g = (unsigned long long)sms * per_sm;
    if (max_ctas > 0 && g > (unsigned long long)max_ctas) g = (unsigned long long)max_ctas;
    const unsigned long long need = (total_tiles + warps - 1) / warps;
    *grid = (unsigned)(g < need ? g : need);
    return FT_OK;
}

int launch_group(const GroupDev &g, int ctas_per_sm, cudaStream_t s, int max_ctas)
{
    const int w = shape_warps(g.warps);
    const void *fn = group_kernel(g.kind, g.R, w, g.pf != 0, false);
    if (!fn) return FT_EINVAL;
    if (g.total_tiles == 0) return FT_OK;
    unsigned grid = 0;
    const int rc = group_grid(fn, w, g.total_tiles, ctas_per_sm, max_ctas, &grid);
    if (rc != FT_OK) return rc;
    GroupDev arg = g;
    void *params[] = {&arg};
    const cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(w * 32), params, kSmemBytes, s);
    if (e != cudaSuccess) return cuda_fail(e);
    return check_launch(1);
}

int launch_small_group(const SmallGroup &g, cudaStream_t s, int max_ctas)
{
    const int w = shape_warps(g.warps);
    const void *fn = group_kernel(g.kind, g.R, w, false, true);
    if (!fn || g.ntasks < 1 || g.ntasks > kSmallTasks) return FT_EINVAL;
    if (g.total_tiles == 0) return FT_OK;
    unsigned grid = 0;
    const int rc = group_grid(fn, w, g.total_tiles, 0, max_ctas, &grid);
    if (rc != FT_OK) return rc;
    void *params[] = {const_cast<SmallGroup *>(&g)};
    const cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(w * 32), params, kSmemBytes, s);
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
    tile_first_global.clear();
    // order tasks by (kind, R), stable, so that each group is contiguous
    std::vector<int> order(in.size());
    for (size_t i = 0; i < in.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return std::make_pair(in[x].kind, in[x].R) < std::make_pair(in[y].kind, in[y].R);
    });
    user_index.assign(order.begin(), order.end());
    for (int idx : order) tasks.push_back(in[idx]);
    tile_first.resize(tasks.size());
    tile_first_global.resize(tasks.size());
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
            tile_first_global[t] = gh.tile0 + g_tiles;
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
           align(8 * tile_first_global.size()) + align(16 * groups.size());
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
    const size_t o_gfirst = off;
    off += align(8 * tile_first_global.size());
    const size_t o_cnt = off;
    if (!tasks.empty()) std::memcpy(host + o_tasks, tasks.data(), sizeof(TaskArgs) * tasks.size());
    if (!tile_first.empty()) std::memcpy(host + o_first, tile_first.data(), 8 * tile_first.size());
    if (!tile_task.empty()) std::memcpy(host + o_map, tile_task.data(), 4 * tile_task.size());
    if (!tile_first_global.empty())
        std::memcpy(host + o_gfirst, tile_first_global.data(), 8 * tile_first_global.size());
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
    std::memset(&mixed, 0, sizeof(mixed));
    mixed.tasks = tasks_dev;
    mixed.tile_task = reinterpret_cast<const uint32_t *>(dev + o_map);
    mixed.tile_first_global = reinterpret_cast<const unsigned long long *>(dev + o_gfirst);
    mixed.total_tiles = tile_task.size();
    mixed.counter = counters_dev;
    mixed.tile_blocks = tile_blocks_;
}

int preload_group_kernels()
{
    for (int kind : {K_F32, K_F64, K_B1, K_B4, K_B8})
        for (int R = 2; R <= FT_MAX_R; ++R)
            for (int w : {8, 16})
                for (bool small : {false, true}) {
                    const void *fn = group_kernel(kind, R, w, false, small);
                    if (!fn) return FT_EINVAL;
                    int sms = 0, per_sm = 0;
                    const int rc = occupancy(fn, w * 32, kSmemBytes, &sms, &per_sm);
                    if (rc != FT_OK) return rc;
                }
    cudaFuncAttributes fa;
    const cudaError_t e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void *>(stats_scatter_kernel));
    return e == cudaSuccess ? FT_OK : cuda_fail(e);
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
    ft_tune tune{0, 0, 0, 0};
    std::map<std::pair<int, int>, std::pair<int, int>> shape;   // (kind, R) -> (warps, prefetch)
    bool mixed = false;                      // the whole batch as one kernel (batched_mixed.cu)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int device = 0;
    unsigned long long graph_kernels = 0;   // kernel launches one replay makes
};

namespace ftv {

// Launch shape of each group from the plan's choices (16 warps without the
// prefetch where none was made).
static void apply_shapes(ft_plan *p)
{
    for (GroupDev &g : p->gd) {
        auto it = p->shape.find({g.kind, g.R});
        g.warps = it == p->shape.end() ? kBatchWarps : it->second.first;
        g.pf = it == p->shape.end() ? 0 : it->second.second;
    }
}

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
    apply_shapes(p);
    cudaError_t e = cudaMemcpy(p->dev, host.data(), need, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? FT_OK : cuda_fail(e);
}

// Records the reset and the group kernels into the capture of stream s, the
// group kernels as parallel branches after the reset (each on its own forked
// stream), so that one group's CTAs can start on the SMs that the previous
// group's CTAs leave at its tail.
static int launch_batch_branches(ft_plan *p, cudaStream_t s)
{
    const BatchLayout &L = p->layout;
    int rc = launch_batch_reset(L.tasks_dev, (int)L.tasks.size(), L.counters_dev, (int)p->gd.size(), s);
    if (rc == FT_OK && p->mixed) return launch_mixed(L.mixed, p->tune.ctas_per_sm, s);
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

// Captures the plan's current layout and shapes into an executable graph:
// the reset, then the groups as parallel branches.  *kernels receives the
// kernel launches one replay makes.
static int build_exec(ft_plan *p, cudaGraph_t *graph, cudaGraphExec_t *exec, unsigned long long *kernels)
{
    *graph = nullptr;
    *exec = nullptr;
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
            *graph = g;
            if ((e = cudaGraphInstantiate(exec, g, 0)) != cudaSuccess) rc = cuda_fail(e);
        } else if (g) {
            cudaGraphDestroy(g);
        }
    }
    cudaStreamDestroy(s);
    // the launches recorded during capture did not run; a replay makes them
    *kernels = g_launches.load() - before;
    g_launches.fetch_sub(*kernels, std::memory_order_relaxed);
    return rc;
}

// In-process autotune cache keyed by a coarse signature of the batch.
struct TuneResult {
    int tile_blocks;
    std::map<std::pair<int, int>, std::pair<int, int>> shape;
    bool mixed;
};
static std::mutex g_tune_mu;
static std::map<std::string, TuneResult> g_tune_cache;

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

// Time of one replay of the plan as it stands (layout uploaded, shapes set):
// the graph that ft_vote_batched would replay is built and replayed, one
// warm-up and the best of three.
static int time_replay(ft_plan *p, cudaStream_t s, float *best_ms)
{
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    unsigned long long kernels = 0;
    int rc = build_exec(p, &g, &x, &kernels);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best = 1e30f;
    if (rc == FT_OK) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaError_t e = cudaGraphLaunch(x, s);
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
            if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
            if ((e = cudaGraphLaunch(x, s)) != cudaSuccess) break;
            if ((e = cudaEventRecord(e1, s)) != cudaSuccess) break;
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            best = std::min(best, ms);
        }
        if (e != cudaSuccess) rc = cuda_fail(e);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    if (x) cudaGraphExecDestroy(x);
    if (g) cudaGraphDestroy(g);
    *best_ms = best;
    return rc;
}

// The autotuner.  It times the graph that will be replayed, with the groups
// as the parallel branches they will be: first the tile size (4 KiB blocks per
// work tile) with every group at 16 warps, then, at that tile size, each
// group's launch shape in turn (warps per CTA 8, 12 or 16, with and without
// the L2 prefetch of the tile's next block), the other groups keeping theirs.
// A voter CTA fills an SM's shared memory with the CRC tables, so one CTA per
// SM is the only residency there is to choose.  Shapes forced by the caller
// (ft_tune.warps / l2_prefetch) are not searched.
static int autotune(ft_plan *p, const ft_tune *forced, TuneResult *out)
{
    const std::string key = signature(p->args);
    const bool forced_mixed = forced && forced->kernels == 1;
    // the one-kernel form runs 16 warps without prefetch: a caller's other shape rules it out
    const bool mixed_allowed = !forced || ((forced->warps == 0 || forced->warps == 16) && forced->l2_prefetch != 2);
    const bool free_kernels = (!forced || forced->kernels == 0) && mixed_allowed;
    const bool free_shape = !forced_mixed && (!forced || (forced->warps == 0 && forced->l2_prefetch == 0));
    const bool free_tile = !forced || forced->tile_blocks == 0;
    if (free_shape && free_tile && free_kernels) {
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
    int rc = FT_OK;
    TuneResult best;
    best.tile_blocks = free_tile ? 8 : forced->tile_blocks;
    best.shape = p->shape;
    best.mixed = forced_mixed;
    p->mixed = forced_mixed;
    float best_ms = 1e30f;
    if (free_tile) {
        for (int tb : {1, 2, 4, 8, 16, 32}) {
            float ms = 0;
            if ((rc = upload_layout(p, tb)) != FT_OK || (rc = time_replay(p, s, &ms)) != FT_OK) break;
            if (ms < best_ms) {
                best_ms = ms;
                best.tile_blocks = tb;
            }
        }
    }
    if (rc == FT_OK && free_shape) {
        rc = upload_layout(p, best.tile_blocks);
        if (rc == FT_OK && !free_tile) rc = time_replay(p, s, &best_ms);
        std::vector<std::pair<int, int>> groups;
        for (const GroupHost &gh : p->layout.groups)
            if (gh.tiles) groups.push_back({gh.kind, gh.R});
        for (size_t gi = 0; gi < groups.size() && rc == FT_OK; ++gi) {
            for (int w : kShapeWarps) {
                for (int pf = 0; pf <= 1 && rc == FT_OK; ++pf) {
                    if (w == kBatchWarps && pf == 0) continue;        // the shape timed already
                    p->shape = best.shape;
                    p->shape[groups[gi]] = {w, pf};
                    apply_shapes(p);
                    float ms = 0;
                    if ((rc = time_replay(p, s, &ms)) != FT_OK) break;
                    if (ms < best_ms) {
                        best_ms = ms;
                        best.shape = p->shape;
                    }
                }
            }
        }
        p->shape = best.shape;
    }
    if (rc == FT_OK && free_kernels) {
        // the whole batch as one kernel, against the best per-group graph
        if (best_ms >= 1e29f && (rc = upload_layout(p, best.tile_blocks)) == FT_OK)
            rc = time_replay(p, s, &best_ms);
        p->mixed = true;
        std::vector<int> tiles;
        if (free_tile) tiles = {4, 8, 16};
        else tiles = {best.tile_blocks};
        for (size_t i = 0; i < tiles.size() && rc == FT_OK; ++i) {
            float ms = 0;
            if ((rc = upload_layout(p, tiles[i])) != FT_OK || (rc = time_replay(p, s, &ms)) != FT_OK) break;
            if (ms < best_ms) {
                best_ms = ms;
                best.tile_blocks = tiles[i];
                best.mixed = true;
            }
        }
        p->mixed = best.mixed;
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (rc != FT_OK) return rc;
    if (free_shape && free_tile && free_kernels) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    *out = best;
    return FT_OK;
}

static int capture(ft_plan *p)
{
    return build_exec(p, &p->graph, &p->exec, &p->graph_kernels);
}

}  // namespace ftv

extern "C" {

int ft_plan_create(ft_plan **plan, const ft_vote_desc *tasks, int32_t ntasks, const ft_tune *tune)
{
    using namespace ftv;
    if (!plan || ntasks < 0 || (ntasks > 0 && !tasks)) return FT_EINVAL;
    *plan = nullptr;
    if (tune && ((tune->tile_blocks && (tune->tile_blocks < 1 || tune->tile_blocks > 64)) ||
                 tune->ctas_per_sm < 0 || tune->ctas_per_sm > 8 ||
                 (tune->warps != 0 && tune->warps != 8 && tune->warps != 12 && tune->warps != 16) ||
                 tune->l2_prefetch < 0 || tune->l2_prefetch > 2 || tune->kernels < 0 || tune->kernels > 2 ||
                 (tune->kernels == 1 && ((tune->warps != 0 && tune->warps != 16) || tune->l2_prefetch == 2))))
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
    if (tune) p->tune = *tune;
    p->tune.ctas_per_sm = tune ? tune->ctas_per_sm : 0;
    const bool forced_shape = tune && (tune->warps != 0 || tune->l2_prefetch != 0 || tune->kernels == 1);
    if (forced_shape) {
        // the caller's shape for every group
        for (const TaskArgs &a : p->args)
            p->shape[{a.kind, a.R}] = {tune->warps ? tune->warps : kBatchWarps, tune->l2_prefetch == 2 ? 1 : 0};
    }
    int rc = FT_OK;
    p->mixed = tune && tune->kernels == 1;
    if (!tune || tune->tile_blocks == 0 || !forced_shape || tune->kernels == 0) {
        TuneResult t;
        rc = autotune(p, tune, &t);
        if (rc == FT_OK) {
            p->tune.tile_blocks = t.tile_blocks;
            if (!forced_shape) p->shape = t.shape;
            p->mixed = t.mixed;
        }
    }
    if (rc == FT_OK) rc = upload_layout(p, p->tune.tile_blocks);
    if (rc == FT_OK) {
        // report a shape common to every group, else 0
        int w = -1, pf = -1;
        for (const GroupDev &g : p->gd) {
            if (!g.total_tiles) continue;
            w = (w == -1 || w == g.warps) ? g.warps : 0;
            pf = (pf == -1 || pf == g.pf + 1) ? g.pf + 1 : 0;
        }
        p->tune.warps = w < 0 ? kBatchWarps : w;
        p->tune.l2_prefetch = pf < 0 ? 1 : pf;
        if (p->mixed) {
            p->tune.warps = kBatchWarps;
            p->tune.l2_prefetch = 1;
        }
        p->tune.kernels = p->mixed ? 1 : 2;
    }
    if (rc == FT_OK) rc = capture(p);
    if (rc != FT_OK) {
        ft_plan_destroy(p);
        return rc;
    }
    *plan = p;
    return FT_OK;
}

int ft_plan_groups(const ft_plan *p, ft_plan_group *out, int32_t max, int32_t *n)
{
    if (!p || !n || max < 0 || (max > 0 && !out)) return FT_EINVAL;
    static const int32_t kDtypeOfKind[] = {FT_F32, FT_F64, FT_U8, FT_I32, FT_I64};
    int k = 0;
    for (size_t i = 0; i < p->gd.size() && k < max; ++i, ++k) {
        const ftv::GroupDev &g = p->gd[i];
        const ftv::GroupHost &gh = p->layout.groups[i];
        out[k].dtype = kDtypeOfKind[g.kind];
        out[k].R = g.R;
        out[k].tasks = gh.t1 - gh.t0;
        out[k].warps = p->mixed ? ftv::kBatchWarps : g.warps ? g.warps : ftv::kBatchWarps;
        out[k].l2_prefetch = p->mixed ? 0 : g.pf;
        out[k].tile_blocks = g.tile_blocks;
        out[k].tiles = g.total_tiles;
    }
    *n = (int32_t)p->gd.size();
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
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (p->mixed) {
        const ftv::BatchLayout &L = p->layout;
        const int rc = ftv::launch_batch_reset(L.tasks_dev, (int)L.tasks.size(), L.counters_dev, (int)p->gd.size(), s);
        return rc == FT_OK ? ftv::launch_mixed(L.mixed, p->tune.ctas_per_sm, s) : rc;
    }
    return ftv::launch_batch(p->layout, p->gd, p->tune.ctas_per_sm, s);
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
