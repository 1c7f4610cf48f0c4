// tile_vote.cuh -- one tile of one task, whatever its element kind and R:
// the tile routine of the kernels that take tiles of tasks of mixed kinds
// (the one-kernel batch and the server's resident voter).
#pragma once

#include "common.cuh"

namespace ftv {

// The return value of a tile routine that voted all of its tile.
constexpr unsigned long long kTileDone = ~0ull;

// Read in place of a preemption word by a tile routine that is not to stop.
static __device__ const unsigned int g_never_preempt = 0u;

// Votes tile k of task a from its block b_begin on (its blocks, and its
// partial last block when the tile holds it) and adds what it voted to
// *a.stats.  With preempt set, lane 0 reads *preempt after each block while
// the tile has more to vote: if it is nonzero the routine stops there and
// returns the block to resume from (the statistics of the blocks voted are
// added); otherwise it returns kTileDone.  Kept out of line, so that each
// (kind, R) instance has its own register allocation inside the one kernel.
// A task of no elements has one tile of no blocks, which adds nothing.
// SMALL: the latency form of the block voter (see vote_full_block), for a
// kernel whose tiles are mostly single blocks of small tasks.
template <int K, int R, bool SMALL>
__device__ __noinline__ unsigned long long mixed_tile(const TaskArgs &a, unsigned long long k, int tile_blocks,
                                                      unsigned long long b_begin, const unsigned int *preempt,
                                                      const uint32_t *s_crc, const CrcLane &L, int lane)
{
    LaneStats<R> st;
    st.init();
    const unsigned long long b0 = k * (unsigned long long)tile_blocks;
    const unsigned long long b1 = min(b0 + (unsigned long long)tile_blocks, a.nfull);
    const bool tail = a.tail_bytes && a.nfull / tile_blocks == k;
    // the word is read after every block either way (a zero word when the
    // tile is not to stop), so the loop has one form
    const volatile unsigned int *pw = preempt ? preempt : &g_never_preempt;
    unsigned long long stop_at = kTileDone;
    for (unsigned long long b = max(b0, b_begin); b < b1; ++b) {
        // the word is loaded before the block and looked at after it, so the
        // load is in flight while the block is voted
        unsigned int u = 0;
        if (lane == 0 && (b + 1 < b1 || tail)) u = *pw;
        vote_full_block<K, R, kSubBatch<K, R>, SMALL>(a, b, ~0ull, s_crc, L, st, lane);
        if (__shfl_sync(0xFFFFFFFFu, u, 0)) {
            stop_at = b + 1;
            break;
        }
    }
    if (tail && stop_at == kTileDone) {
        LaneStats<R> ts;
        ts.init();
        vote_tail_block<K, R>(a, a.nfull, s_crc, L, ts, lane);
        st.merge(ts);
    }
    st.flush(a.stats, lane);
    return stop_at;
}

template <int K, bool SMALL>
__device__ __forceinline__ unsigned long long mixed_tile_k(const TaskArgs &a, unsigned long long k, int tile_blocks,
                                                           unsigned long long b_begin, const unsigned int *preempt,
                                                           const uint32_t *s_crc, const CrcLane &L, int lane)
{
    switch (a.R) {
    case 2: return mixed_tile<K, 2, SMALL>(a, k, tile_blocks, b_begin, preempt, s_crc, L, lane);
    case 3: return mixed_tile<K, 3, SMALL>(a, k, tile_blocks, b_begin, preempt, s_crc, L, lane);
    case 4: return mixed_tile<K, 4, SMALL>(a, k, tile_blocks, b_begin, preempt, s_crc, L, lane);
    case 5: return mixed_tile<K, 5, SMALL>(a, k, tile_blocks, b_begin, preempt, s_crc, L, lane);
    case 6: return mixed_tile<K, 6, SMALL>(a, k, tile_blocks, b_begin, preempt, s_crc, L, lane);
    case 7: return mixed_tile<K, 7, SMALL>(a, k, tile_blocks, b_begin, preempt, s_crc, L, lane);
    case 8: return mixed_tile<K, 8, SMALL>(a, k, tile_blocks, b_begin, preempt, s_crc, L, lane);
    default: return kTileDone;
    }
}

// The (kind, R) instance of the tile routine for task a.
template <bool SMALL = false>
__device__ __forceinline__ unsigned long long mixed_tile_any(const TaskArgs &a, unsigned long long k, int tile_blocks,
                                                             unsigned long long b_begin, const unsigned int *preempt,
                                                             const uint32_t *s_crc, const CrcLane &L, int lane)
{
    switch (a.kind) {
    case K_F32: return mixed_tile_k<K_F32, SMALL>(a, k, tile_blocks, b_begin, preempt, s_crc, L, lane);
    case K_F64: return mixed_tile_k<K_F64, SMALL>(a, k, tile_blocks, b_begin, preempt, s_crc, L, lane);
    case K_B1: return mixed_tile_k<K_B1, SMALL>(a, k, tile_blocks, b_begin, preempt, s_crc, L, lane);
    case K_B4: return mixed_tile_k<K_B4, SMALL>(a, k, tile_blocks, b_begin, preempt, s_crc, L, lane);
    case K_B8: return mixed_tile_k<K_B8, SMALL>(a, k, tile_blocks, b_begin, preempt, s_crc, L, lane);
    default: return kTileDone;
    }
}

}  // namespace ftv
