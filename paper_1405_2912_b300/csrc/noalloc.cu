// noalloc.cu -- ft_vote_batched_noalloc: the batched vote for callers that
// must not allocate device memory.
//
// The batched plan (ft_plan_create) allocates its task table, tile map and
// tile counters with cudaMalloc.  Some callers cannot do that, or cannot let
// a library do it for them: code running inside a framework that owns every
// byte of device memory through its own pool, a latency-critical loop where
// cudaMalloc / cudaFree would synchronise the device, or a plug-in that must
// not change the process's allocation pattern.  This entry point keeps its
// scratch in a fixed file-scope device array instead, and builds the batch on
// the host in fixed static buffers, so a call allocates nothing on the device
// or the host.
//
// The scratch array is shared by every call in the process on a given device
// and keeps the last call's contents; the tile counters and statistics are
// reset at the start of each call.  Two calls whose work overlaps on the GPU
// (different streams, no ordering between them) race on the scratch and give
// wrong results: order them on one stream or synchronise between them.
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "runtime.h"

namespace ftv {

constexpr int kNoallocMaxTasks = FT_NOALLOC_MAX_TASKS;
constexpr int kNoallocMaxGroups = 64;   // (kind, R) pairs that can occur: 5 x 7
constexpr size_t kNoallocTasksBytes = sizeof(TaskArgs) * kNoallocMaxTasks;
constexpr size_t kNoallocFirstBytes = sizeof(unsigned long long) * kNoallocMaxTasks;
constexpr size_t kNoallocCounterBytes = sizeof(unsigned long long) * kNoallocMaxGroups;
constexpr size_t kNoallocScratchBytes = kNoallocTasksBytes + kNoallocFirstBytes + kNoallocCounterBytes;

// The scratch: task table (ordered by group), each task's first tile within
// its group, one tile counter per group.  Every GPU that loads the library
// holds it (about 580 KiB) until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Host staging of the same layout, filled under g_stage_mu and copied with one
// pageable cudaMemcpyAsync (which returns once the bytes are staged, so the
// buffer can be refilled by the next call).
static unsigned char g_stage[kNoallocScratchBytes];
static std::mutex g_stage_mu;

// Per-device scratch address from cudaGetSymbolAddress (set up by the first
// call on each device, with that device current).
constexpr int kMaxDevices = 64;
static void *g_scratch_addr[kMaxDevices];
static std::mutex g_addr_mu;

struct NoallocGroup {
    const TaskArgs *tasks;                   // whole table (device)
    const unsigned long long *first;         // per ordered task (device)
    unsigned long long *counter;             // this group's tile counter (device)
    unsigned long long total_tiles;
    int32_t t0, t1;                          // the group's task range
    int32_t tile_blocks;
    int32_t pad_;
};

// Largest t in [t0, t1) with first[t] <= tg (first[t0] = 0 <= tg), found by the
// warp 32 candidates at a time.
__device__ __forceinline__ int find_task(const unsigned long long *first, int t0, int t1, unsigned long long tg,
                                         int lane)
{
    int lo = t0, hi = t1;
    while (hi - lo > 1) {
        const int stride = (hi - lo + 31) / 32;
        const int idx = lo + lane * stride;
        const bool p = idx < hi && first[idx] <= tg;
        const unsigned ballot = __ballot_sync(0xFFFFFFFFu, p);
        const int k = 31 - __clz((int)ballot);
        lo += k * stride;
        hi = min(lo + stride, hi);
    }
    return lo;
}

template <int K, int R, int W>
__global__ void __launch_bounds__(W * 32, 1) noalloc_batched_kernel(const NoallocGroup g)
{
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *s_crc = reinterpret_cast<uint32_t *>(smem);
    load_crc_tables<W>(s_crc);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    CrcLane L;
    L.init(lane);
    LaneStats<R> st;
    st.init();
    int cur = -1;
    ft_stats *cur_stats = nullptr;
    for (;;) {
        unsigned long long tg = 0;
        if (lane == 0) tg = atomicAdd(g.counter, 1ull);
        tg = __shfl_sync(0xFFFFFFFFu, tg, 0);
        if (tg >= g.total_tiles) break;
        const int t = find_task(g.first, g.t0, g.t1, tg, lane);
        const TaskArgs a = g.tasks[t];
        if (t != cur) {
            if (cur >= 0) st.flush(cur_stats, lane);
            st.init();
            cur = t;
            cur_stats = a.stats;
        }
        const unsigned long long k = tg - g.first[t];
        const unsigned long long b0 = k * (unsigned long long)g.tile_blocks;
        const unsigned long long b1 = min(b0 + (unsigned long long)g.tile_blocks, a.nfull);
        for (unsigned long long b = b0; b < b1; ++b)
            vote_full_block<K, R>(a, b, ~0ull, s_crc, L, st, lane);   // no prefetch: as the batched kernel
        if (a.tail_bytes && a.nfull / g.tile_blocks == k) {
            LaneStats<R> ts;
            ts.init();
            vote_tail_block<K, R>(a, a.nfull, s_crc, L, ts, lane);
            st.merge(ts);
        }
    }
    if (cur >= 0) st.flush(cur_stats, lane);
}

constexpr int kNoallocWarps = 16;

template <int K, int R>
static const void *noalloc_fn()
{
    return reinterpret_cast<const void *>(noalloc_batched_kernel<K, R, kNoallocWarps>);
}

template <int K>
static const void *noalloc_fn_k(int R)
{
    switch (R) {
    case 2: return noalloc_fn<K, 2>();
    case 3: return noalloc_fn<K, 3>();
    case 4: return noalloc_fn<K, 4>();
    case 5: return noalloc_fn<K, 5>();
    case 6: return noalloc_fn<K, 6>();
    case 7: return noalloc_fn<K, 7>();
    case 8: return noalloc_fn<K, 8>();
    default: return nullptr;
    }
}

static const void *noalloc_kernel(int kind, int R)
{
    switch (kind) {
    case K_F32: return noalloc_fn_k<K_F32>(R);
    case K_F64: return noalloc_fn_k<K_F64>(R);
    case K_B1: return noalloc_fn_k<K_B1>(R);
    case K_B4: return noalloc_fn_k<K_B4>(R);
    case K_B8: return noalloc_fn_k<K_B8>(R);
    default: return nullptr;
    }
}

static int group_key(int kind, int R) { return kind * 8 + R; }   // < 64

// Resident CTAs per SM and SM count for one group kernel, cached in fixed
// arrays (no container that could allocate).
static int noalloc_occupancy(int dev, int key, const void *fn, size_t smem, int *sms, int *per_sm)
{
    static std::mutex mu;
    static int cached[kMaxDevices][kNoallocMaxGroups][2];
    std::lock_guard<std::mutex> lk(mu);
    int *c = cached[dev][key];
    if (c[1] == 0) {
        cudaError_t e;
        if ((e = cudaDeviceGetAttribute(&c[0], cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_fail(e);
        if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return cuda_fail(e);
        int occ = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kNoallocWarps * 32, smem)) != cudaSuccess)
            return cuda_fail(e);
        if (occ < 1) return FT_EINVAL;
        c[1] = occ;
    }
    *sms = c[0];
    *per_sm = c[1];
    return FT_OK;
}

// The scratch address on the current device; the first call on a device
// looks it up with cudaGetSymbolAddress.
static int scratch_address(int dev, unsigned char **out)
{
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e);
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[dev]);
    return FT_OK;
}

static int vote_batched_noalloc(const ft_vote_desc *descs, int ntasks, int tile_blocks, cudaStream_t s)
{
    if (ntasks < 0 || ntasks > kNoallocMaxTasks || (ntasks > 0 && !descs)) return FT_EINVAL;
    const bool auto_tile = tile_blocks == 0;
    if (tile_blocks < 0 || tile_blocks > 64) return FT_EINVAL;
    for (int i = 0; i < ntasks; ++i) {
        const int rc = validate_desc(&descs[i]);
        if (rc != FT_OK) return rc;
    }
    // The batch reaches the device through copies from one static host
    // staging area that every call refills.  Recorded into a graph, such a
    // copy would read that area when the graph is replayed, by which time a
    // later call may have refilled it with another batch; so a stream that is
    // being captured is refused.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return cuda_fail(e);
    if (cap != cudaStreamCaptureStatusNone) return FT_EINVAL;
    if (ntasks == 0) return FT_OK;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= kMaxDevices) return FT_EINVAL;
    unsigned char *scratch = nullptr;
    int rc = scratch_address(dev, &scratch);
    if (rc != FT_OK) return rc;

    TaskArgs *tasks_h = reinterpret_cast<TaskArgs *>(g_stage);
    unsigned long long *first_h = reinterpret_cast<unsigned long long *>(g_stage + kNoallocTasksBytes);
    const TaskArgs *tasks_d = reinterpret_cast<const TaskArgs *>(scratch);
    const unsigned long long *first_d = reinterpret_cast<const unsigned long long *>(scratch + kNoallocTasksBytes);
    unsigned long long *cnt_d = reinterpret_cast<unsigned long long *>(scratch + kNoallocTasksBytes + kNoallocFirstBytes);

    // counting sort of the tasks by (kind, R) group into the staging table
    int count[kNoallocMaxGroups] = {};
    int start[kNoallocMaxGroups] = {};
    int fill[kNoallocMaxGroups] = {};
    NoallocGroup groups[kNoallocMaxGroups];
    int ngroups = 0;
    std::lock_guard<std::mutex> lk(g_stage_mu);
    for (int i = 0; i < ntasks; ++i) count[group_key(dtype_kind(descs[i].dtype), descs[i].R)]++;
    for (int k = 0, acc = 0; k < kNoallocMaxGroups; ++k) {
        start[k] = acc;
        fill[k] = acc;
        acc += count[k];
    }
    for (int i = 0; i < ntasks; ++i) {
        const int k = group_key(dtype_kind(descs[i].dtype), descs[i].R);
        tasks_h[fill[k]++] = make_task_args(&descs[i]);
    }
    const size_t smem = kSmemBytes;
    if (auto_tile) {
        // every group kernel holds a whole SM's shared memory (one CTA per
        // SM) with the same warps, so the first group's wave stands for all
        unsigned long long total = 0;
        for (int i = 0; i < ntasks; ++i) total += tasks_h[i].nfull + (tasks_h[i].tail_bytes ? 1 : 0);
        const TaskArgs &a0 = tasks_h[0];
        const void *fn = noalloc_kernel(a0.kind, a0.R);
        if (!fn) return FT_EINVAL;
        int sms = 0, per_sm = 0;
        if ((rc = noalloc_occupancy(dev, group_key(a0.kind, a0.R), fn, smem, &sms, &per_sm)) != FT_OK) return rc;
        tile_blocks = auto_tile_blocks(total, (unsigned long long)sms * per_sm * kNoallocWarps);
    }
    for (int k = 0; k < kNoallocMaxGroups; ++k) {
        if (!count[k]) continue;
        unsigned long long tiles = 0;
        for (int t = start[k]; t < start[k] + count[k]; ++t) {
            first_h[t] = tiles;
            const unsigned long long nblk = tasks_h[t].nfull + (tasks_h[t].tail_bytes ? 1 : 0);
            tiles += (nblk + tile_blocks - 1) / tile_blocks;
        }
        NoallocGroup &g = groups[ngroups];
        std::memset(&g, 0, sizeof(g));
        g.tasks = tasks_d;
        g.first = first_d;
        g.counter = cnt_d + ngroups;
        g.total_tiles = tiles;
        g.t0 = start[k];
        g.t1 = start[k] + count[k];
        g.tile_blocks = tile_blocks;
        ++ngroups;
    }
    // copy the table and the first tiles; the reset kernel then clears the
    // statistics and the tile counters left by the previous call
    const size_t bytes_tasks = sizeof(TaskArgs) * ntasks;
    if ((e = cudaMemcpyAsync(scratch, g_stage, bytes_tasks, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaMemcpyAsync(scratch + kNoallocTasksBytes, g_stage + kNoallocTasksBytes,
                             sizeof(unsigned long long) * ntasks, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e);
    if ((rc = launch_batch_reset(tasks_d, ntasks, cnt_d, ngroups, s)) != FT_OK) return rc;
    for (int gi = 0; gi < ngroups; ++gi) {
        const NoallocGroup &g = groups[gi];
        if (g.total_tiles == 0) continue;
        const TaskArgs &a0 = tasks_h[g.t0];
        const void *fn = noalloc_kernel(a0.kind, a0.R);
        if (!fn) return FT_EINVAL;
        int sms = 0, per_sm = 0;
        if ((rc = noalloc_occupancy(dev, group_key(a0.kind, a0.R), fn, smem, &sms, &per_sm)) != FT_OK) return rc;
        unsigned long long grid = (unsigned long long)sms * per_sm;
        const unsigned long long need = (g.total_tiles + kNoallocWarps - 1) / kNoallocWarps;
        if (grid > need) grid = need;
        NoallocGroup arg = g;
        void *params[] = {&arg};
        if ((e = cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kNoallocWarps * 32), params, smem, s)) != cudaSuccess)
            return cuda_fail(e);
        if ((rc = check_launch(1)) != FT_OK) return rc;
    }
    return FT_OK;
}

}  // namespace ftv

extern "C" int ft_vote_batched_noalloc(const ft_vote_desc *tasks, int32_t ntasks, int32_t tile_blocks,
                                       ft_stream stream)
{
    return ftv::vote_batched_noalloc(tasks, ntasks, tile_blocks, static_cast<cudaStream_t>(stream));
}
