// vote.cu -- the single-task voter (ft_vote), the digest-only CRC32C
// (ft_digest) and the library-wide C-ABI helpers.
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"
#include "runtime.h"
#include "vote_kernel.cuh"

namespace ftv {

std::atomic<unsigned long long> g_launches{0};
thread_local int g_last_cuda = 0;

int cuda_fail(cudaError_t e)
{
    g_last_cuda = (int)e;
    return FT_ECUDA;
}

int check_launch(int nlaunch)
{
    g_launches.fetch_add((unsigned long long)nlaunch, std::memory_order_relaxed);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FT_OK : cuda_fail(e);
}

// Per-(device, kernel) launch facts: the SM count and the resident CTAs per SM
// at the kernel's dynamic shared memory size (the attribute is raised once).
int occupancy(const void *fn, int threads, size_t smem, int *sms, int *per_sm)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, std::pair<int, int>> cache;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find({dev, fn});
    if (it == cache.end()) {
        int n_sm = 0, occ = 0;
        if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_fail(e);
        if (smem > 48 * 1024 &&
            (e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return cuda_fail(e);
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem)) != cudaSuccess)
            return cuda_fail(e);
        if (occ < 1) return FT_EINVAL;
        it = cache.emplace(std::make_pair(dev, fn), std::make_pair(n_sm, occ)).first;
    }
    *sms = it->second.first;
    *per_sm = it->second.second;
    return FT_OK;
}

int auto_tile_blocks(unsigned long long total_blocks, unsigned long long wave_warps)
{
    int tb = 8;
    while (tb > 1 && total_blocks < (unsigned long long)tb * wave_warps) tb >>= 1;
    return tb;
}

size_t dtype_size(int dtype)
{
    switch (dtype) {
    case FT_I32: case FT_U32: case FT_F32: return 4;
    case FT_I64: case FT_U64: case FT_F64: return 8;
    case FT_U8: return 1;
    default: return 0;
    }
}

int dtype_kind(int dtype)
{
    switch (dtype) {
    case FT_F32: return K_F32;
    case FT_F64: return K_F64;
    case FT_I32: case FT_U32: return K_B4;
    case FT_I64: case FT_U64: return K_B8;
    case FT_U8: return K_B1;
    default: return -1;
    }
}

static bool aligned(const void *p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

int validate_desc(const ft_vote_desc *d)
{
    if (!d) return FT_EINVAL;
    if (d->R < 2 || d->R > FT_MAX_R) return FT_EINVAL;
    const size_t sz = dtype_size(d->dtype);
    if (sz == 0) return FT_EINVAL;
    if (!d->stats || !aligned(d->stats, 8)) return FT_EINVAL;
    if (d->dtype == FT_F32 || d->dtype == FT_F64) {
        // 0 <= rel_tol <= 1 and a finite abs_tol >= 0 in the element type (NaN fails too)
        if (!(d->abs_tol >= 0.0) || !(d->rel_tol >= 0.0) || !(d->rel_tol <= 1.0)) return FT_EINVAL;
        if (d->dtype == FT_F32 && !std::isfinite((float)d->abs_tol)) return FT_EINVAL;
        if (d->dtype == FT_F64 && !std::isfinite(d->abs_tol)) return FT_EINVAL;
    }
    if (d->n == 0) return FT_OK;
    if (d->n > (~0ull >> 4) / sz) return FT_EINVAL;
    const unsigned long long nbytes = d->n * sz;
    if (!d->out || !aligned(d->out, 16)) return FT_EINVAL;
    if (d->block_crc && !aligned(d->block_crc, 4)) return FT_EINVAL;
    const uintptr_t o0 = (uintptr_t)d->out, o1 = o0 + nbytes;
    for (int r = 0; r < d->R; ++r) {
        const void *p = d->replicas[r];
        if (!p || !aligned(p, 16)) return FT_EINVAL;
        const uintptr_t p0 = (uintptr_t)p, p1 = p0 + nbytes;
        if (p0 < o1 && o0 < p1) return FT_EINVAL;   // out overlaps a replica
    }
    if (d->block_crc) {
        const uintptr_t c0 = (uintptr_t)d->block_crc;
        const uintptr_t c1 = c0 + 4 * ((nbytes + FT_BLOCK_BYTES - 1) / FT_BLOCK_BYTES);
        if (c0 < o1 && o0 < c1) return FT_EINVAL;
    }
    return FT_OK;
}

TaskArgs make_task_args(const ft_vote_desc *d)
{
    TaskArgs a;
    std::memset(&a, 0, sizeof(a));
    for (int r = 0; r < FT_MAX_R; ++r)
        a.rep[r] = static_cast<const uint8_t *>(r < d->R ? d->replicas[r] : nullptr);
    a.out = static_cast<uint8_t *>(d->out);
    a.crc = d->block_crc;
    a.stats = d->stats;
    a.n = d->n;
    const unsigned long long nbytes = d->n * dtype_size(d->dtype);
    a.nfull = nbytes / FT_BLOCK_BYTES;
    a.tail_bytes = (uint32_t)(nbytes % FT_BLOCK_BYTES);
    a.R = d->R;
    a.kind = dtype_kind(d->dtype);
    a.abs_tol = d->abs_tol;
    a.rel_tol = d->rel_tol;
    return a;
}

// The statistics reset before a single vote whose statistics go straight to
// the caller's ft_stats.  It lets the voter kernel, which is launched right
// after it as a programmatic dependent, start at once: the voter touches the
// statistics only after pdl_wait().
__global__ void reset_stats_kernel(ft_stats *s)
{
    pdl_release();
    reset_stats(s, threadIdx.x);
}

// The same reset launched as a programmatic dependent of the caller's previous
// kernel: it lets the voter launch at once, then waits for its predecessor
// (which may still be adding to these statistics) before it resets them.
__global__ void reset_stats_chained_kernel(ft_stats *s)
{
    pdl_release();
    pdl_wait();
    reset_stats(s, threadIdx.x);
}

// ---------------------------------------------------------------------------
// Statistics slots.  A vote needs its statistics at (0, -1) before the first
// warp adds to them; with the caller's ft_stats that takes a reset kernel
// ahead of the voter, a second launch that costs a small vote about as much
// as its own work.  Instead a vote takes a slot from a per-device pool of
// library-owned statistics that are kept at their initial values between
// votes: the warps add into the slot, and the last CTA to finish copies it to
// the caller's ft_stats, puts it back to its initial values and marks it free
// in host-mapped memory.  The host takes a slot only when it reads it free,
// so a slot is never used by two votes at once, whatever streams they run
// on.  When every slot is taken, and in a stream capture (a graph would bake
// one slot into every replay), the vote falls back to the reset kernel.
// ---------------------------------------------------------------------------
constexpr int kSlots = 1024;
constexpr int kMaxDevices = 64;

struct SlotPool {
    StatsSlot *dev = nullptr;
    unsigned int *busy = nullptr;      // host view
    unsigned int *busy_dev = nullptr;  // device view of the same memory
    std::atomic<unsigned int> next{0};
    std::atomic<bool> ready{false};
    bool failed = false;            // guarded by g_pool_mu
};
static SlotPool g_pools[kMaxDevices];
static std::mutex g_pool_mu;

__global__ void init_slots_kernel(StatsSlot *slots, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int f = 0; f <= FT_MAX_R; ++f) reset_stats(&slots[i].s, f);
    slots[i].done = 0;
}

// The pool of the current device, created on first use (outside a capture).
static SlotPool *slot_pool(int dev)
{
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    SlotPool &p = g_pools[dev];
    if (p.ready.load(std::memory_order_acquire)) return &p;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (p.ready.load(std::memory_order_relaxed)) return &p;
    if (p.failed) return nullptr;
    cudaStream_t st = nullptr;
    cudaError_t e = cudaMalloc(&p.dev, sizeof(StatsSlot) * kSlots);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&p.busy), sizeof(unsigned int) * kSlots,
                                            cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&p.busy_dev), p.busy, 0);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        std::memset(p.busy, 0, sizeof(unsigned int) * kSlots);
        init_slots_kernel<<<(kSlots + 255) / 256, 256, 0, st>>>(p.dev, kSlots);
        g_launches.fetch_add(1, std::memory_order_relaxed);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        p.failed = true;       // the reset-kernel path serves this device from now on
        return nullptr;
    }
    p.ready.store(true, std::memory_order_release);
    return &p;
}

// Takes a free slot (-1 when all are taken).
static int acquire_slot(SlotPool &p)
{
    for (int k = 0; k < kSlots; ++k) {
        const unsigned int i = p.next.fetch_add(1, std::memory_order_relaxed) % kSlots;
        unsigned int expect = 0;
        if (__atomic_compare_exchange_n(&p.busy[i], &expect, 1u, false, __ATOMIC_ACQ_REL, __ATOMIC_ACQUIRE))
            return (int)i;
    }
    return -1;
}

static void release_slot(SlotPool &p, int i) { __atomic_store_n(&p.busy[i], 0u, __ATOMIC_RELEASE); }

// Launches one shape.  With a slot the statistics reset is not needed; the
// kernel is a programmatic dependent of the caller's previous kernel.
template <int K, int R, int kVoteWarps, bool PF, int JB, bool SMALL = false>
static int launch_vote_shape(const TaskArgs &a, cudaStream_t s, const VoteLaunch *cfg, const SlotRef &sr)
{
    const void *fn = reinterpret_cast<const void *>(vote_kernel<K, R, kVoteWarps, PF, JB, SMALL>);
    if (sr.flag) {
        // the server's vote, which also writes its completion flag
        if constexpr (kDefaultShape<K, R, kVoteWarps, PF, JB, SMALL>)
            fn = flagged_vote_kernel<K, R, kVoteWarps, PF, JB, SMALL>();
        else
            return FT_EINVAL;
    }
    const size_t smem = kSmemBytes;
    int sms = 0, per_sm = 0;
    int rc = occupancy(fn, kVoteWarps * 32, smem, &sms, &per_sm);
    if (rc != FT_OK) return rc;
    if (cfg && cfg->ctas_per_sm > 0 && cfg->ctas_per_sm < per_sm) per_sm = cfg->ctas_per_sm;
    const unsigned long long nblk = a.nfull + (a.tail_bytes ? 1 : 0);
    unsigned long long grid = (nblk + kVoteWarps - 1) / kVoteWarps;
    unsigned long long cap = (unsigned long long)sms * per_sm;
    if (cfg && cfg->max_ctas > 0 && (unsigned long long)cfg->max_ctas < cap) cap = cfg->max_ctas;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3(kVoteWarps * 32);
    lc.dynamicSmemBytes = smem;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    void *args[] = {const_cast<TaskArgs *>(&a), const_cast<SlotRef *>(&sr)};
    const cudaError_t e = cudaLaunchKernelExC(&lc, fn, args);
    if (e != cudaSuccess) return cuda_fail(e);
    return check_launch(1);
}

// Votes of up to 32768 blocks (128 MiB of output) have at most a few blocks
// per warp, so latency, not bandwidth, sets their time: for them the shape
// with more warps and no prefetch measured faster even where the policy
// prefers the prefetching one (f32 R = 3: 3 x 16M 52 against 58 us, 3 x 4M 18
// against 20 us; equal at 3 x 64M; 6.7 against 6.25 TB/s the other way at
// 3 x 256M).  Votes of at most one block per warp of a full wave of 8-warp
// CTAs (1184 blocks, 4.6 MiB of output) take 8-warp CTAs, which spreads them
// over up to all 148 SMs instead of the 74 that 16-warp CTAs would use, and
// the SMALL form of the block voter (two CRC chains per lane, R = 3 pairwise
// masks kept in registers).
constexpr unsigned long long kSmallVoteBlocks = 32768;
// Up to 4096 blocks (16 MiB of output) the 16-warp shape also takes the SMALL
// block form: f32 R = 3 3 x 2M 13.1 -> 10.7 us, 3 x 4M 18.6 -> 16.9 us;
// from 16384 blocks on it no longer gains (3 x 16M 48.2 against 48.5 us, 5 x 8M
// f64 76.6 against 75.3, 5 x 8M i32 43.1 against 42.9).
constexpr unsigned long long kSmallFormBlocks = 4096;

template <int K, int R>
static int launch_vote_kr(const TaskArgs &a, cudaStream_t s, const VoteLaunch *cfg, const SlotRef &sr)
{
    using P = VotePolicy<K, R>;
    constexpr int JB = kSubBatch<K, R>;
    const unsigned long long nblk = a.nfull + (a.tail_bytes ? 1 : 0);
    if constexpr (K == K_F32 && R == 3) {
        // the shapes a tuning override may pick
        const int w = cfg ? cfg->warps : 0, jb = cfg ? cfg->sub_batch : 0;
        if (w == 4 && jb == 8) return launch_vote_shape<K, R, 4, false, 8>(a, s, cfg, sr);
        if (w == 4 && jb == 4) return launch_vote_shape<K, R, 4, false, 4>(a, s, cfg, sr);
        if (w == 8 && jb == 8) return launch_vote_shape<K, R, 8, false, 8>(a, s, cfg, sr);
        if (w == 8 && jb == 4) return launch_vote_shape<K, R, 8, false, 4>(a, s, cfg, sr);
        if (w == 16 && jb == 8) return launch_vote_shape<K, R, 16, false, 8>(a, s, cfg, sr);
        if (w == 16 && jb == 4) return launch_vote_shape<K, R, 16, false, 4>(a, s, cfg, sr);
        if (w == 12) return launch_vote_shape<K, R, 12, true, JB>(a, s, cfg, sr);
    }
    int sms = 0, per_sm = 0;
    int rc = occupancy(reinterpret_cast<const void *>(vote_kernel<K, R, kTinyWarps, false, JB, true>),
                       kTinyWarps * 32, kSmemBytes, &sms, &per_sm);
    if (rc != FT_OK) return rc;
    if (nblk <= (unsigned long long)sms * per_sm * kTinyWarps)
        return launch_vote_shape<K, R, kTinyWarps, false, JB, true>(a, s, cfg, sr);
    if (cfg && nblk <= kSmallVoteBlocks) {
        if (cfg->small_form == 1) return launch_vote_shape<K, R, 16, false, JB, true>(a, s, cfg, sr);
        if (cfg->small_form == 2) return launch_vote_shape<K, R, 16, false, JB, false>(a, s, cfg, sr);
    }
    if (nblk <= kSmallFormBlocks) return launch_vote_shape<K, R, 16, false, JB, true>(a, s, cfg, sr);
    if constexpr (P::kPrefetch) {
        if (nblk <= kSmallVoteBlocks) return launch_vote_shape<K, R, 16, false, JB>(a, s, cfg, sr);
    }
    return launch_vote_shape<K, R, P::kWarps, P::kPrefetch, JB>(a, s, cfg, sr);
}

template <int K>
static int launch_vote_k(const TaskArgs &a, cudaStream_t s, const VoteLaunch *cfg, const SlotRef &sr)
{
    switch (a.R) {
    case 2: return launch_vote_kr<K, 2>(a, s, cfg, sr);
    case 3: return launch_vote_kr<K, 3>(a, s, cfg, sr);
    case 4: return launch_vote_kr<K, 4>(a, s, cfg, sr);
    case 5: return launch_vote_kr<K, 5>(a, s, cfg, sr);
    case 6: return launch_vote_kr<K, 6>(a, s, cfg, sr);
    case 7: return launch_vote_kr<K, 7>(a, s, cfg, sr);
    case 8: return launch_vote_kr<K, 8>(a, s, cfg, sr);
    default: return FT_EINVAL;
    }
}

// Launched directly after the statistics reset on the same stream (sr.slot
// null) or, with a slot, after whatever the stream ran before.
static int launch_vote(const TaskArgs &a, cudaStream_t s, const VoteLaunch *cfg, const SlotRef &sr)
{
    switch (a.kind) {
    case K_F32: return launch_vote_k<K_F32>(a, s, cfg, sr);
    case K_F64: return launch_vote_k<K_F64>(a, s, cfg, sr);
    case K_B1: return launch_vote_k<K_B1>(a, s, cfg, sr);
    case K_B4: return launch_vote_k<K_B4>(a, s, cfg, sr);
    case K_B8: return launch_vote_k<K_B8>(a, s, cfg, sr);
    default: return FT_EINVAL;
    }
}

// Loads (and sets up for the library's shared memory) every shape of K1 that
// launch_vote_kr picks without a tuning override for (K, R).
template <int K, int R>
static int preload_vote_kr()
{
    using P = VotePolicy<K, R>;
    constexpr int JB = kSubBatch<K, R>;
    int sms = 0, per_sm = 0, rc;
    if ((rc = occupancy(reinterpret_cast<const void *>(vote_kernel<K, R, kTinyWarps, false, JB, true>),
                        kTinyWarps * 32, kSmemBytes, &sms, &per_sm)) != FT_OK ||
        (rc = occupancy(reinterpret_cast<const void *>(vote_kernel<K, R, 16, false, JB, true>), 16 * 32, kSmemBytes,
                        &sms, &per_sm)) != FT_OK ||
        (rc = occupancy(reinterpret_cast<const void *>(vote_kernel<K, R, 16, false, JB, false>), 16 * 32,
                        kSmemBytes, &sms, &per_sm)) != FT_OK)
        return rc;
    return occupancy(reinterpret_cast<const void *>(vote_kernel<K, R, P::kWarps, P::kPrefetch, JB, false>),
                     P::kWarps * 32, kSmemBytes, &sms, &per_sm);
}

template <int K>
static int preload_vote_k()
{
    int rc;
    if ((rc = preload_vote_kr<K, 2>()) != FT_OK || (rc = preload_vote_kr<K, 3>()) != FT_OK ||
        (rc = preload_vote_kr<K, 4>()) != FT_OK || (rc = preload_vote_kr<K, 5>()) != FT_OK ||
        (rc = preload_vote_kr<K, 6>()) != FT_OK || (rc = preload_vote_kr<K, 7>()) != FT_OK)
        return rc;
    return preload_vote_kr<K, 8>();
}

int preload_vote_kernels()
{
    int rc;
    if ((rc = preload_vote_k<K_F32>()) != FT_OK || (rc = preload_vote_k<K_F64>()) != FT_OK ||
        (rc = preload_vote_k<K_B1>()) != FT_OK || (rc = preload_vote_k<K_B4>()) != FT_OK ||
        (rc = preload_vote_k<K_B8>()) != FT_OK)
        return rc;
    if ((rc = preload_flagged_vote_kernels()) != FT_OK) return rc;
    int dev = 0;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    slot_pool(dev);   // the statistics slots too (a device without them votes through the reset kernel)
    return FT_OK;
}

int reserve_vote_slot()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    SlotPool *pool = slot_pool(dev);
    return pool ? acquire_slot(*pool) : -1;
}

void release_vote_slot(int slot)
{
    int dev = 0;
    if (slot < 0 || cudaGetDevice(&dev) != cudaSuccess) return;
    SlotPool *pool = slot_pool(dev);
    if (pool) release_slot(*pool, slot);
}

int vote_task_reserved(const TaskArgs &a, cudaStream_t s, const VoteLaunch *cfg, int slot, unsigned long long *flag,
                       unsigned long long seq)
{
    int dev = 0;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    SlotPool *pool = slot_pool(dev);
    if (!pool || slot < 0 || slot >= kSlots || a.n == 0) return FT_EINVAL;
    const int rc = launch_vote(a, s, cfg, SlotRef{pool->dev + slot, pool->busy_dev + slot, 1, flag, seq});
    if (rc != FT_OK) release_slot(*pool, slot);   // the kernel did not start
    return rc;
}

int vote_task_slot(const TaskArgs &a, cudaStream_t s, const VoteLaunch *cfg, unsigned long long *flag,
                   unsigned long long seq)
{
    if (a.n == 0) return FT_EAGAIN;
    const int i = reserve_vote_slot();
    if (i < 0) return FT_EAGAIN;
    return vote_task_reserved(a, s, cfg, i, flag, seq);
}

int vote_desc(const ft_vote_desc *desc, cudaStream_t s, const VoteLaunch *cfg)
{
    int rc = validate_desc(desc);
    if (rc != FT_OK) return rc;
    const int mode = cfg ? cfg->stats_mode : 0;
    if (mode == 3) {
        // the reset and the voter both chained to the previous kernel
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(1);
        lc.blockDim = dim3(FT_MAX_R + 1);
        lc.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        lc.attrs = attr;
        lc.numAttrs = 1;
        const cudaError_t e = cudaLaunchKernelEx(&lc, reset_stats_chained_kernel, desc->stats);
        if (e != cudaSuccess) return cuda_fail(e);
        if ((rc = check_launch(1)) != FT_OK) return rc;
        if (desc->n == 0) return FT_OK;
        return launch_vote(make_task_args(desc), s, cfg, SlotRef{nullptr, nullptr, 1, nullptr, 0});
    }
    if (desc->n > 0 && mode != 1) {
        // one launch: the statistics go through a slot, unless the stream is
        // being captured or no slot is free
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaError_t e = cudaStreamIsCapturing(s, &cap);
        if (e != cudaSuccess) return cuda_fail(e);
        int dev = 0;
        if (cap == cudaStreamCaptureStatusNone && (e = cudaGetDevice(&dev)) == cudaSuccess) {
            SlotPool *pool = slot_pool(dev);
            const int i = pool ? acquire_slot(*pool) : -1;
            if (i >= 0) {
                rc = launch_vote(make_task_args(desc), s, cfg, SlotRef{pool->dev + i, pool->busy_dev + i, 1, nullptr, 0});
                if (rc != FT_OK) release_slot(*pool, i);   // the kernel did not start
                return rc;
            }
        }
        if (e != cudaSuccess) return cuda_fail(e);
    }
    reset_stats_kernel<<<1, FT_MAX_R + 1, 0, s>>>(desc->stats);
    if ((rc = check_launch(1)) != FT_OK) return rc;
    if (desc->n == 0) return FT_OK;
    return launch_vote(make_task_args(desc), s, cfg, SlotRef{nullptr, nullptr, 0, nullptr, 0});
}

// ---------------------------------------------------------------------------
// K2: digest-only CRC32C of blocks of `block_bytes` (a multiple of 4096).
// Each warp digests whole blocks, 4 KiB chunk by chunk, and chains the chunk
// registers with the x^(8*4096) operator.  A full chunk is digested from the
// registers its coalesced loads fill (crc_vec); each lane reads its own
// segment of a partial last chunk.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(W * 32, 1)
    digest_kernel(const uint8_t *__restrict__ buf, unsigned long long nbytes, uint32_t block_bytes,
                  unsigned long long nblocks, uint32_t *__restrict__ out, uint32_t init_full)
{
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *s_crc = reinterpret_cast<uint32_t *>(smem);
    load_crc_tables<W>(s_crc);
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    CrcLane L;
    L.init(lane);
    const unsigned long long step = (unsigned long long)gridDim.x * W;
    // The warp's full 4 KiB chunks form one sequence across its blocks; the
    // next chunk of the sequence is loaded into registers while the current
    // one is digested.  (An L2 prefetch of the warp's next block, as the f32
    // voter uses, measured slower here: 3.9 against 4.2 TB/s.)
    uint4 q[8];
    bool have = false;   // q holds chunk 0 of block b
    for (unsigned long long b = (unsigned long long)blockIdx.x * W + w; b < nblocks; b += step) {
        const unsigned long long start = b * block_bytes;
        const unsigned long long len = min((unsigned long long)block_bytes, nbytes - start);
        const unsigned long long nfull = len / kBlockBytes;
        const uint32_t rem = (uint32_t)(len % kBlockBytes);
        if (nfull && !have) {
            const uint4 *src = reinterpret_cast<const uint4 *>(buf + start);
#pragma unroll
            for (int t = 0; t < 8; ++t) q[t] = __ldcs(src + lane + 32 * t);
        }
        have = false;
        uint32_t acc = 0;
        for (unsigned long long c = 0; c < nfull; ++c) {
            uint4 cur[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) cur[t] = q[t];
            const uint4 *next = nullptr;
            if (c + 1 < nfull) {
                next = reinterpret_cast<const uint4 *>(buf + start + (c + 1) * kBlockBytes);
            } else if (b + step < nblocks && nbytes - (b + step) * block_bytes >= (unsigned long long)kBlockBytes) {
                next = reinterpret_cast<const uint4 *>(buf + (b + step) * block_bytes);
                have = true;
            }
            if (next) {
#pragma unroll
                for (int t = 0; t < 8; ++t) q[t] = __ldcs(next + lane + 32 * t);
            }
            uint32_t cc = 0;
#pragma unroll
            for (int t = 0; t < 8; ++t) cc = crc_vec(s_crc, L, cc, cur[t], t == 7);
            acc = shift_4096(acc) ^ crc_combine(s_crc, cc, lane);
        }
        if (rem) {
            // partial last chunk: lane l reads its bytes [128 l, 128 l + 128)
            // below rem itself, four at a time, and moves its register over
            // the bytes that follow them
            const uint8_t *src = buf + start + nfull * kBlockBytes + 128u * lane;
            const uint32_t seg = rem > 128u * lane ? min(128u, rem - 128u * lane) : 0u;
            uint32_t cc = 0, k = 0;
            for (; k + 4 <= seg; k += 4) cc = crc_step4(s_crc, L, cc ^ *reinterpret_cast<const uint32_t *>(src + k));
            for (; k < seg; ++k) cc = crc_step1(s_crc, cc, src[k]);
            cc = shift_bytes(cc, rem > 128u * (lane + 1) ? rem - 128u * (lane + 1) : 0u);
            acc = shift_bytes(acc, rem) ^ warp_xor(cc);
        }
        const uint32_t init = (len == block_bytes) ? init_full : shift_bytes(0xFFFFFFFFu, (uint32_t)len);
        if (lane == 0) out[b] = ~(acc ^ init);
    }
}

// K2a: digest-only CRC32C of 4 KiB blocks.  Each warp runs through its full
// blocks in grid-stride order with the next block's coalesced loads in flight
// while the current one is digested (crc_vec, crc_combine); the partial last
// block, if any, goes to the warp whose turn it would be, each lane reading its
// own 128-byte segment.  Without the general kernel's per-chunk chaining, 24
// warps per CTA measured 6.24 TB/s on 1 GiB against 5.08 for the general
// kernel (16 warps 5.75, 20 warps 6.12; two blocks per warp at once 4.8-5.5).
template <int W>
__global__ void __launch_bounds__(W * 32, 1)
    digest4k_kernel(const uint8_t *__restrict__ buf, unsigned long long nbytes, uint32_t *__restrict__ out)
{
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *s_crc = reinterpret_cast<uint32_t *>(smem);
    load_crc_tables<W>(s_crc);
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    CrcLane L;
    L.init(lane);
    const unsigned long long nfull = nbytes / kBlockBytes;
    const unsigned long long step = (unsigned long long)gridDim.x * W;
    const unsigned long long gw = (unsigned long long)blockIdx.x * W + w;
    uint4 q[8];
    if (gw < nfull) {
        const uint4 *src = reinterpret_cast<const uint4 *>(buf + gw * kBlockBytes);
#pragma unroll
        for (int t = 0; t < 8; ++t) q[t] = __ldcs(src + lane + 32 * t);
    }
    for (unsigned long long b = gw; b < nfull; b += step) {
        uint4 cur[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) cur[t] = q[t];
        if (b + step < nfull) {
            const uint4 *src = reinterpret_cast<const uint4 *>(buf + (b + step) * kBlockBytes);
#pragma unroll
            for (int t = 0; t < 8; ++t) q[t] = __ldcs(src + lane + 32 * t);
        }
        uint32_t cc = 0;
#pragma unroll
        for (int t = 0; t < 8; ++t) cc = crc_vec(s_crc, L, cc, cur[t], t == 7);
        const uint32_t raw = crc_combine(s_crc, cc, lane);
        if (lane == 0) out[b] = ~(raw ^ g_crc.init4096);
    }
    const uint32_t rem = (uint32_t)(nbytes % kBlockBytes);
    if (rem && nfull % step == gw) {
        // lane l reads its bytes [128 l, 128 l + 128) below rem, four at a
        // time, and moves its register over the bytes that follow them
        const uint8_t *src = buf + nfull * kBlockBytes + 128u * lane;
        const uint32_t seg = rem > 128u * lane ? min(128u, rem - 128u * lane) : 0u;
        uint32_t cc = 0, k = 0;
        for (; k + 4 <= seg; k += 4) cc = crc_step4(s_crc, L, cc ^ *reinterpret_cast<const uint32_t *>(src + k));
        for (; k < seg; ++k) cc = crc_step1(s_crc, cc, src[k]);
        cc = shift_bytes(cc, rem > 128u * (lane + 1) ? rem - 128u * (lane + 1) : 0u);
        const uint32_t raw = warp_xor(cc);
        if (lane == 0) out[nfull] = ~(raw ^ shift_bytes(0xFFFFFFFFu, rem));
    }
}

constexpr int kDigest4kWarps = 24;

static int launch_digest4k(const void *buf, unsigned long long nbytes, uint32_t *out, cudaStream_t s)
{
    const unsigned long long nblocks = (nbytes + kBlockBytes - 1) / kBlockBytes;
    auto fn = digest4k_kernel<kDigest4kWarps>;
    const size_t smem = kSmemBytes;
    int sms = 0, per_sm = 0;
    int rc = occupancy(reinterpret_cast<const void *>(fn), kDigest4kWarps * 32, smem, &sms, &per_sm);
    if (rc != FT_OK) return rc;
    unsigned long long grid = (nblocks + kDigest4kWarps - 1) / kDigest4kWarps;
    const unsigned long long cap = (unsigned long long)sms * per_sm;
    if (grid > cap) grid = cap;
    fn<<<(unsigned)grid, kDigest4kWarps * 32, smem, s>>>(static_cast<const uint8_t *>(buf), nbytes, out);
    return check_launch(1);
}

// Warps per CTA of the general digest kernel (blocks of a multiple of 4 KiB
// above 4 KiB): 16, which measured 5.45 TB/s on 1 GiB in 64 KiB blocks
// against 5.13 with 20 (fewer, longer blocks per warp).
template <int W>
static int launch_digest(const void *buf, unsigned long long nbytes, uint32_t block_bytes, uint32_t *out,
                         cudaStream_t s)
{
    const unsigned long long nblocks = (nbytes + block_bytes - 1) / block_bytes;
    auto fn = digest_kernel<W>;
    const size_t smem = kSmemBytes;
    int sms = 0, per_sm = 0;
    int rc = occupancy(reinterpret_cast<const void *>(fn), W * 32, smem, &sms, &per_sm);
    if (rc != FT_OK) return rc;
    unsigned long long grid = (nblocks + W - 1) / W;
    const unsigned long long cap = (unsigned long long)sms * per_sm;
    if (grid > cap) grid = cap;
    const uint32_t init_full = gf_mul(0xFFFFFFFFu, gf_xpow8(block_bytes));
    fn<<<(unsigned)grid, W * 32, smem, s>>>(static_cast<const uint8_t *>(buf), nbytes, block_bytes, nblocks, out,
                                           init_full);
    return check_launch(1);
}

int digest(const void *buf, unsigned long long nbytes, uint32_t block_bytes, uint32_t *out, cudaStream_t s)
{
    if (block_bytes < FT_BLOCK_BYTES || block_bytes % FT_BLOCK_BYTES || block_bytes > (1u << 24)) return FT_EINVAL;
    if (nbytes == 0) return FT_OK;
    if (!buf || !out || !aligned(buf, 16) || !aligned(out, 4)) return FT_EINVAL;
    if (block_bytes == FT_BLOCK_BYTES) return launch_digest4k(buf, nbytes, out, s);
    return launch_digest<16>(buf, nbytes, block_bytes, out, s);
}

}  // namespace ftv

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int ft_vote(const ft_vote_desc *desc, ft_stream stream)
{
    return ftv::vote_desc(desc, static_cast<cudaStream_t>(stream), nullptr);
}

int ft_digest(const void *buf, uint64_t nbytes, uint32_t block_bytes, uint32_t *out, ft_stream stream)
{
    return ftv::digest(buf, nbytes, block_bytes, out, static_cast<cudaStream_t>(stream));
}

const char *ft_strerror(int code)
{
    switch (code) {
    case FT_OK: return "ok";
    case FT_EINVAL: return "invalid argument";
    case FT_ENOMEM: return "out of memory";
    case FT_EAGAIN: return "try again (over budget or not done)";
    case FT_ETIMEDOUT: return "timed out";
    case FT_ECUDA: return "CUDA error";
    case FT_ENOTFOUND: return "unknown ticket";
    default: return "unknown error code";
    }
}

int ft_last_cuda_error(void) { return ftv::g_last_cuda; }

uint64_t ft_launch_count(void) { return ftv::g_launches.load(std::memory_order_relaxed); }

const char *ft_version(void) { return "ftvote 0.1 sm_103a"; }

}  // extern "C"
