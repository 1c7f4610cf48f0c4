// vote_kernel.cuh -- K1, the single-task voter kernel, and the hand-off of
// its statistics through a slot of the library's pool.  vote.cu builds the
// kernels of ft_vote; vote_flag.cu builds the shapes that the voter picks by
// itself again with a completion flag, for the server.
#pragma once

#include "common.cuh"

namespace ftv {

struct StatsSlot {
    ft_stats s;                    // same layout as the caller's
    unsigned long long done;       // CTAs finished
    unsigned long long pad_[5];    // one slot per 192 bytes
};

struct SlotRef {
    StatsSlot *slot;               // nullptr: statistics go straight to a.stats
    unsigned int *busy;            // host-mapped free flag of the slot (0 = free)
    int wait_early;                // wait for the predecessor before reading the replicas
    unsigned long long *flag;      // the FLAG kernels: set to seq (host-mapped) once a.stats holds the result
    unsigned long long seq;
};

constexpr int kTinyWarps = 8;   // warps per CTA of the smallest votes' shape

// End of a slot vote, after every warp of the CTA has added its statistics to
// the slot: the last CTA to arrive copies the slot to the caller's ft_stats
// (entries beyond R are still at their initial values), resets it and marks
// it free.  FLAG: it then writes sr.seq to *sr.flag (host-mapped), after a
// system-scope fence, so that a host that reads the flag finds the copy.
// Only the server's votes are built with it: the flag code alone, never
// executed, measured 0.25 us longer per 3 x 1M f32 vote back to back (8.16
// against 7.91 us).
template <bool FLAG>
__device__ __noinline__ void slot_finish(const SlotRef &sr, ft_stats *user)
{
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&sr.slot->done, 1ull) == (unsigned long long)gridDim.x - 1ull;
    }
    __syncthreads();
    if (!s_last) return;
    constexpr int kWords = (int)(sizeof(ft_stats) / 8);
    if (threadIdx.x < kWords) {
        __threadfence();
        unsigned long long *w = reinterpret_cast<unsigned long long *>(&sr.slot->s) + threadIdx.x;
        reinterpret_cast<unsigned long long *>(user)[threadIdx.x] = __ldcg(w);
        *w = (threadIdx.x < FT_MAX_R || threadIdx.x == 2 * FT_MAX_R) ? 0ull : ~0ull;
        if constexpr (FLAG) __threadfence_system();   // the copy reaches the host before the flag
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sr.slot->done = 0;
        // the slot's reset values are visible on the device before the free
        // flag is written, so the vote the host launches on the slot once it
        // reads the flag sees them; only the GPU reads the slot
        __threadfence();
        *reinterpret_cast<volatile unsigned int *>(sr.busy) = 0u;
        if constexpr (FLAG) *reinterpret_cast<volatile unsigned long long *>(sr.flag) = sr.seq;
    }
}

// ---------------------------------------------------------------------------
// K1: persistent single-task voter.  Warps take 4 KiB blocks in grid-stride
// order; consecutive warps of a CTA take consecutive blocks.  PF: each warp
// prefetches its next block into L2.  JB: 16-byte vectors per lane loaded per
// sub-batch.
//
// The kernel is always launched as a programmatic dependent of the kernel
// before it in the stream, and lets the kernel after it launch once its own
// CTAs have voted their blocks.
// Before it waits for its predecessor it asks L2 for the warp's first block
// of every replica (L2 is the device's point of coherence, so early lines are
// never stale) and copies the CRC tables into shared memory; it reads the
// replicas only after the wait.  With a slot the predecessor is whatever the
// caller ran before; without one it is the statistics reset, which touches
// only the statistics, and the wait moves to just before they are added.
// ---------------------------------------------------------------------------
template <int K, int R, int W, bool PF, int JB, bool SMALL, bool FLAG = false>
__global__ void __launch_bounds__(W * 32, 1) vote_kernel(const TaskArgs a, const SlotRef sr)
{
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *s_crc = reinterpret_cast<uint32_t *>(smem);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned long long step = (unsigned long long)gridDim.x * W;
    const unsigned long long gw = (unsigned long long)blockIdx.x * W + w;
    if (lane < R && gw < a.nfull) prefetch_l2(rep_for_lane<R>(a, lane) + gw * kBlockBytes, kBlockBytes);
    load_crc_tables<W>(s_crc);
    if (sr.wait_early) pdl_wait();  // the predecessor's writes (possibly our replicas) are visible
    __syncthreads();
    CrcLane L;
    L.init(lane);
    LaneStats<R> st;
    st.init();
    for (unsigned long long b = gw; b < a.nfull; b += step)
        vote_full_block<K, R, JB, SMALL>(a, b, PF ? b + step : ~0ull, s_crc, L, st, lane);
    if (a.tail_bytes && a.nfull % step == gw) {
        // the partial last block goes to the warp whose turn it would be
        LaneStats<R> ts;
        ts.init();
        vote_tail_block<K, R>(a, a.nfull, s_crc, L, ts, lane);
        st.merge(ts);
    }
    // Only now may the next kernel's CTAs launch: one released at the start
    // would take SMs (a voter CTA holds an SM's shared memory) and sit in its
    // wait while this kernel votes, keeping other streams' work off them.
    pdl_release();
    if (sr.slot) {
        st.flush(&sr.slot->s, lane);
        slot_finish<FLAG>(sr, a.stats);
    } else {
        if (!sr.wait_early) pdl_wait();   // the statistics reset has completed
        st.flush(a.stats, lane);
    }
}

// The shapes the voter picks by itself for (K, R), without a tuning
// override: the 8-warp and 16-warp SMALL forms, 16 warps without the
// prefetch, and the policy shape.  vote_flag.cu builds these with FLAG.
template <int K, int R, int W, bool PF, int JB, bool SMALL>
constexpr bool kDefaultShape =
    JB == kSubBatch<K, R> && ((W == kTinyWarps && !PF && SMALL) || (W == 16 && !PF) ||
                              (W == VotePolicy<K, R>::kWarps && PF == VotePolicy<K, R>::kPrefetch && !SMALL));

// vote_kernel<K, R, W, PF, JB, SMALL, true> for a default shape (vote_flag.cu).
template <int K, int R, int W, bool PF, int JB, bool SMALL>
const void *flagged_vote_kernel();
// Loads every flagged kernel and sets it up for the tables' shared memory.
int preload_flagged_vote_kernels();

}  // namespace ftv
