// resident.cu -- the server's resident voter (resident.h): a persistent
// kernel, one CTA per SM, that stays on the GPU while vote requests arrive.
//
// Warp 0 of CTA 0 admits: it polls the host-mapped mailboxes, copies each
// newly published request into its device slot and makes it claimable.  Every
// other warp votes: it scans the 32 slots (one per lane), claims the next tile
// of the request with the fewest unclaimed tiles (shortest remaining work
// first, so a small request that arrives behind a large one is voted at once
// beside it), votes the tile through the (kind, R) tile routine and counts it;
// the warp that completes a request copies its statistics to host-mapped
// memory (and to the caller's statistics, if given), puts the slot's
// statistics back to their initial values and then writes the request's
// generation to its host-mapped flag.  A small request (fewer 4 KiB blocks
// than there are voting warps) is also marked urgent: a warp voting a tile of
// another request checks the urgent mask after each block, and while it is
// set puts its tile aside, votes a tile of the small request and then
// resumes, so a small request waits for one block of the warps' work, not
// for their whole tiles.
//
// Every wait is bounded.  The admitting warp leaves once nothing has arrived
// for idle_ns and every admitted request is done (the host relaunches the
// kernel for the next request), when the host sets *quit, or, with an error
// code, when requests are on the device but none has completed for
// max_wait_ns.  A voting warp waits for work only while the admitting warp
// keeps beating (its loop counter); it leaves when that warp has left, or,
// with an error code, when the beat stops for max_wait_ns.
#include "resident.h"
#include "tile_vote.cuh"

namespace ftv {
namespace {

__device__ __forceinline__ unsigned long long gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_sys(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned int ld_relaxed_sys32(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_gpu(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned int ld_acquire_gpu32(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_gpu(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed_sys(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed_sys32(unsigned int *p, unsigned int v)
{
    asm volatile("st.relaxed.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_release_gpu(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Atomic add with acquire and release semantics at device scope: the
// thread's earlier writes are visible to whoever sees the new value, and it
// sees the writes of those whose adds came before.
__device__ __forceinline__ unsigned long long atom_add_acq_rel_gpu(unsigned long long *p, unsigned long long v)
{
    unsigned long long old;
    asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

constexpr int kSlotWords = (int)(sizeof(ResSlot) / 8);
constexpr int kStatWords = (int)(sizeof(ft_stats) / 8);   // mismatch[8], first[8], no_majority, first
static_assert(kStatWords == 2 * FT_MAX_R + 2, "ft_stats layout");

// Warp 0 of CTA 0: lane j watches mailbox j.
__device__ __noinline__ void admit_loop(const ResDev &g, int lane)
{
    const unsigned full = 0xFFFFFFFFu;
    const unsigned long long beat0 = ld_relaxed_gpu(g.beat);
    unsigned long long last_act = gtime();
    unsigned long long prog_seen = ld_relaxed_gpu(g.progress), prog_at = last_act;
    for (unsigned long long it = 1;; ++it) {
        if (lane == 0) st_relaxed_gpu(g.beat, beat0 + it);
        // both host reads in flight at once
        const unsigned quit = ld_relaxed_sys32(g.quit);
        const unsigned long long gen = ld_acquire_sys(g.mail_gen + lane);
        if (__any_sync(full, quit != 0u)) break;
        const bool fresh = gen != 0ull && gen != ld_relaxed_gpu(g.admitted + lane);
        bool small = false;
        // each newly published mailbox is copied by the whole warp, one word
        // per lane, in one round trip to host memory (after the acquire of
        // its gen, plain loads that bypass the caches)
        for (unsigned m = __ballot_sync(full, fresh); m; m &= m - 1u) {
            const int jj = __ffs(m) - 1;
            const unsigned long long gj = __shfl_sync(full, gen, jj);
            const unsigned long long *src = reinterpret_cast<const unsigned long long *>(g.mail + jj);
            unsigned long long wv = 0;
            if (lane < kSlotWords) {
                wv = __ldcv(src + lane);
                reinterpret_cast<unsigned long long *>(g.slots + jj)[lane] = wv;
            }
            const unsigned long long ntiles =
                __shfl_sync(full, wv, (int)(offsetof(ResMail, ntiles) / 8)) & kResTileMask;
            const unsigned long long tw = __shfl_sync(full, wv, (int)(offsetof(ResMail, tile_blocks) / 8));
            if (lane == jj) small = (tw >> 32) != 0ull;
            __threadfence();
            if (lane == 0) {
                const unsigned long long g24 = (gj & 0xFFFFFFull) << kResGenShift;
                st_relaxed_gpu(g.meta + jj, g24 | ntiles);
                // claimable from here: the release orders the slot and its
                // tile count before the claim counter
                st_release_gpu(g.next + jj, g24);
                st_relaxed_gpu(g.admitted + jj, gj);
            }
        }
        static_assert(kSlotWords <= 32, "one mailbox word per lane");
        static_assert(offsetof(ResMail, urgent) == offsetof(ResMail, tile_blocks) + 4 &&
                          offsetof(ResMail, tile_blocks) % 8 == 0,
                      "tile_blocks and urgent share a word");
        __syncwarp();
        const unsigned fresh_mask = __ballot_sync(full, fresh);
        const unsigned urgent_mask = __ballot_sync(full, small);
        if (fresh_mask && lane == 0) {
            atomicOr(g.active, fresh_mask);
            if (urgent_mask) atomicOr(g.urgent, urgent_mask);
        }
        const bool busy = ld_relaxed_gpu(g.admitted + lane) != ld_relaxed_gpu(g.fin + lane);
        const unsigned busy_mask = __ballot_sync(full, busy);
        const unsigned long long t = gtime();
        if (fresh_mask || busy_mask) {
            last_act = t;
        } else if (t - last_act > g.idle_ns) {
            break;
        }
        if (busy_mask && !fresh_mask) {
            const unsigned long long p = ld_relaxed_gpu(g.progress);
            if (p != prog_seen) {
                prog_seen = p;
                prog_at = t;
            } else if (t - prog_at > g.max_wait_ns) {
                if (lane == 0) st_relaxed_sys32(g.error, kResErrNoProgress);
                break;
            }
        } else {
            prog_at = t;
        }
        if (!fresh_mask) __nanosleep(128);
    }
    __threadfence();
    if (lane == 0) atomicExch(g.stop, g.epoch);
}

// The request of slot j is done: its statistics to the host (and the
// caller), the slot back to its initial values, then the flag.
__device__ __noinline__ void hand_off(const ResDev &g, int j, const ResSlot &sl, int lane)
{
    // every warp that voted a tile of the request counted it after its
    // statistics with a release, and lane 0 of this warp counted the last
    // with an acquire: the statistics are final in L2 (the other lanes read
    // them after the shuffle that follows lane 0's count)
    __threadfence();
    if (lane < kStatWords) {
        unsigned long long *w = reinterpret_cast<unsigned long long *>(g.stats + j) + lane;
        const unsigned long long v = __ldcg(w);
        reinterpret_cast<unsigned long long *>(g.stats_out + j)[lane] = v;
        if (sl.user) reinterpret_cast<unsigned long long *>(sl.user)[lane] = v;
        *w = (lane < FT_MAX_R || lane == 2 * FT_MAX_R) ? 0ull : ~0ull;   // counts 0, first indices -1
    }
    if (lane == 0) {
        g.done[j] = 0ull;
        atomicAdd(g.progress, 1ull);   // requests completed
    }
    // the statistics reach the host, and the resets the device, before the flag
    __threadfence_system();
    __syncwarp();
    if (lane == 0) {
        st_relaxed_sys(g.flags + j, sl.gen);
        st_relaxed_gpu(g.fin + j, sl.gen);
    }
}

// Scans the slots in `mask` (lane j: slot j) and claims the next tile of the
// one with the fewest unclaimed tiles.  Returns 1 with the slot, tile, the
// request's tile count and the slot's contents (*sl_out); 0 when the claim
// lost a race (look again); -1 when nothing in the mask is claimable.
__device__ __noinline__ int claim_tile(const ResDev &g, unsigned mask, int lane, int *j_out,
                                          unsigned long long *k_out, unsigned long long *nt_out, ResSlot *sl_out)
{
    const unsigned full = 0xFFFFFFFFu;
    unsigned key = 0xFFFFFFFFu;
    unsigned long long mt = 0;
    if ((mask >> lane) & 1u) {
        const unsigned long long nx = ld_acquire_gpu(g.next + lane);
        mt = ld_relaxed_gpu(g.meta + lane);
        if ((nx >> kResGenShift) == (mt >> kResGenShift)) {
            const unsigned long long c = nx & kResTileMask, n = mt & kResTileMask;
            if (c < n) {
                const unsigned long long rem = n - c < (1ull << 26) ? n - c : (1ull << 26) - 1ull;
                key = ((unsigned)rem << 5) | (unsigned)lane;
            }
        }
    }
    const unsigned best = __reduce_min_sync(full, key);
    if (best == 0xFFFFFFFFu) return -1;
    const int j = (int)(best & 31u);
    const unsigned long long mj = __shfl_sync(full, mt, j);
    // the slot, one word per lane, read while the claim is in flight: it is
    // the request of the generation scanned (written before its claim
    // counter), and the claim below keeps it only if that generation holds
    unsigned long long w = 0;
    if (lane < kSlotWords) w = __ldcg(reinterpret_cast<const unsigned long long *>(g.slots + j) + lane);
    unsigned long long v = 0;
    if (lane == 0) v = atomicAdd(g.next + j, 1ull);
    v = __shfl_sync(full, v, 0);
    const unsigned long long nt = mj & kResTileMask, k = v & kResTileMask;
    // another request took the slot since the scan, or its tiles are all taken
    if ((v >> kResGenShift) != (mj >> kResGenShift) || k >= nt) return 0;
    unsigned long long *d = reinterpret_cast<unsigned long long *>(sl_out);
#pragma unroll
    for (int i = 0; i < kSlotWords; ++i) d[i] = __shfl_sync(full, w, i);
    if (k + 1ull == nt && lane == 0) {
        atomicAnd(g.active, ~(1u << j));
        atomicAnd(g.urgent, ~(1u << j));
    }
    *j_out = j;
    *k_out = k;
    *nt_out = nt;
    return 1;
}

// The slot as the admitting warp wrote it before making it claimable.
__device__ __forceinline__ void read_slot(const ResDev &g, int j, ResSlot &sl)
{
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(g.slots + j);
    unsigned long long *d = reinterpret_cast<unsigned long long *>(&sl);
#pragma unroll
    for (int i = 0; i < kSlotWords; ++i) d[i] = __ldcg(src + i);
}

// The (kind, R) tile routine of the slot's request, out of line so that the
// scheduling loop around it stays small; the latency form of the block voter
// (most of this kernel's tiles are single blocks of small requests).
__device__ __noinline__ unsigned long long vote_slot_tile(const ResSlot &sl, unsigned long long k,
                                                          unsigned long long b_begin, const unsigned int *preempt,
                                                          const uint32_t *s_crc, const CrcLane &L, int lane)
{
    return mixed_tile_any<true>(sl.args, k, sl.tile_blocks, b_begin, preempt, s_crc, L, lane);
}

// Counts a voted tile of slot j (after its statistics); the warp that
// completes the request hands it off.
__device__ __forceinline__ void finish_tile(const ResDev &g, int j, unsigned long long nt, const ResSlot &sl, int lane)
{
    // lane 0 made the tile's statistics atomics; its acquire-release count
    // orders them before the count, and makes the last counter see every
    // earlier tile's
    int last = 0;
    if (lane == 0) last = atom_add_acq_rel_gpu(g.done + j, 1ull) + 1ull == nt;
    if (__shfl_sync(0xFFFFFFFFu, last, 0)) hand_off(g, j, sl, lane);
}

__device__ __noinline__ void vote_loop(const ResDev &g, const uint32_t *s_crc, int lane)
{
    CrcLane L;
    L.init(lane);
    unsigned long long beat_seen = ld_relaxed_gpu(g.beat), beat_at = gtime();
    unsigned sleep_ns = 64;
    // a tile put aside for an urgent request: slot, tile, next block, tiles of its request
    bool held = false;
    int hj = 0;
    unsigned long long hk = 0, hb = 0, hnt = 0;
    for (;;) {
        int j = 0;
        unsigned long long k = 0, nt = 0, b_begin = 0;
        bool resume = false;
        ResSlot sl;
        if (held) {
            // urgent tiles first, then the tile put aside
            const unsigned urg = ld_acquire_gpu32(g.urgent);
            const int c = urg ? claim_tile(g, urg, lane, &j, &k, &nt, &sl) : -1;
            if (c == 0) continue;
            if (c < 0) {
                j = hj;
                k = hk;
                nt = hnt;
                b_begin = hb;
                resume = true;
                read_slot(g, j, sl);
            }
        } else {
            const int c = claim_tile(g, ld_acquire_gpu32(g.active), lane, &j, &k, &nt, &sl);
            if (c == 0) continue;
            if (c < 0) {
                // nothing to claim: leave when the admitting warp has left,
                // and give up if it has stopped beating
                if (ld_acquire_gpu32(g.stop) == g.epoch) return;
                const unsigned long long bt = ld_relaxed_gpu(g.beat), t = gtime();
                if (bt != beat_seen) {
                    beat_seen = bt;
                    beat_at = t;
                } else if (t - beat_at > g.max_wait_ns) {
                    if (lane == 0) st_relaxed_sys32(g.error, kResErrNoBeat);
                    return;
                }
                __nanosleep(sleep_ns);
                if (sleep_ns < 1024u) sleep_ns <<= 1;
                continue;
            }
            sleep_ns = 64;
        }
        // the tile put aside, and a fresh tile of a large request, stop
        // between blocks while an urgent request waits; an urgent tile, and
        // any tile voted while another is put aside, runs through
        const bool stoppable = resume || (!held && !sl.urgent);
        const unsigned long long b = vote_slot_tile(sl, k, b_begin, stoppable ? g.urgent : nullptr, s_crc, L, lane);
        if (b != kTileDone) {
            held = true;
            hj = j;
            hk = k;
            hb = b;
            hnt = nt;
            continue;
        }
        if (resume) held = false;
        finish_tile(g, j, nt, sl, lane);
    }
}

__global__ void __launch_bounds__(kResWarps * 32, 1) resident_kernel(const ResDev g)
{
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *s_crc = reinterpret_cast<uint32_t *>(smem);
    load_crc_tables<kResWarps>(s_crc);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x < 32) admit_loop(g, lane);
    else vote_loop(g, s_crc, lane);
}

}  // namespace

static int resident_grid(int max_ctas, int *grid)
{
    int sms = 0, per_sm = 0;
    const int rc = occupancy(reinterpret_cast<const void *>(resident_kernel), kResWarps * 32, kSmemBytes, &sms, &per_sm);
    if (rc != FT_OK) return rc;
    *grid = sms * per_sm;
    if (max_ctas > 0 && max_ctas < *grid) *grid = max_ctas;
    return FT_OK;
}

int resident_preload(int max_ctas, int *voting_warps)
{
    int grid = 0;
    const int rc = resident_grid(max_ctas, &grid);
    if (rc != FT_OK) return rc;
    if (voting_warps) *voting_warps = grid * kResWarps - 1;
    return FT_OK;
}

int resident_launch(const ResDev &g, cudaStream_t s, int max_ctas, int *ctas)
{
    int grid = 0;
    const int rc = resident_grid(max_ctas, &grid);
    if (rc != FT_OK) return rc;
    resident_kernel<<<grid, kResWarps * 32, kSmemBytes, s>>>(g);
    if (ctas) *ctas = grid;
    return check_launch(1);
}

}  // namespace ftv
