// batched_mixed.cu -- the batched voter as one persistent kernel for a whole
// batch of mixed element kinds and replica counts: a warp claims the next
// tile of the batch, whatever its task's kind and R, and votes it through the
// (kind, R) instance of the tile routine.  The plan's autotuner times it
// against one kernel per (kind, R) group and keeps the faster.
#include "batched.h"
#include "common.cuh"
#include "runtime.h"

namespace ftv {

// Votes tile k of task a (its blocks, and its partial last block when the
// tile holds it) and adds the tile's statistics to the task's.  Kept out of
// line, so that each (kind, R) instance has its own register allocation
// inside the one kernel.
template <int K, int R>
__device__ __noinline__ void mixed_tile(const TaskArgs &a, unsigned long long k, int tile_blocks, const uint32_t *s_crc,
                                        const CrcLane &L, int lane)
{
    LaneStats<R> st;
    st.init();
    const unsigned long long b0 = k * (unsigned long long)tile_blocks;
    const unsigned long long b1 = min(b0 + (unsigned long long)tile_blocks, a.nfull);
    for (unsigned long long b = b0; b < b1; ++b) vote_full_block<K, R>(a, b, ~0ull, s_crc, L, st, lane);
    if (a.tail_bytes && a.nfull / tile_blocks == k) {
        LaneStats<R> ts;
        ts.init();
        vote_tail_block<K, R>(a, a.nfull, s_crc, L, ts, lane);
        st.merge(ts);
    }
    st.flush(a.stats, lane);
}

template <int K>
__device__ __forceinline__ void mixed_tile_k(const TaskArgs &a, unsigned long long k, int tile_blocks,
                                             const uint32_t *s_crc, const CrcLane &L, int lane)
{
    switch (a.R) {
    case 2: mixed_tile<K, 2>(a, k, tile_blocks, s_crc, L, lane); break;
    case 3: mixed_tile<K, 3>(a, k, tile_blocks, s_crc, L, lane); break;
    case 4: mixed_tile<K, 4>(a, k, tile_blocks, s_crc, L, lane); break;
    case 5: mixed_tile<K, 5>(a, k, tile_blocks, s_crc, L, lane); break;
    case 6: mixed_tile<K, 6>(a, k, tile_blocks, s_crc, L, lane); break;
    case 7: mixed_tile<K, 7>(a, k, tile_blocks, s_crc, L, lane); break;
    case 8: mixed_tile<K, 8>(a, k, tile_blocks, s_crc, L, lane); break;
    default: break;
    }
}

template <int W>
__global__ void __launch_bounds__(W * 32, 1) batched_mixed_kernel(const MixedDev g)
{
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *s_crc = reinterpret_cast<uint32_t *>(smem);
    load_crc_tables<W>(s_crc);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    CrcLane L;
    L.init(lane);
    for (;;) {
        unsigned long long tg = 0;
        if (lane == 0) tg = atomicAdd(g.counter, 1ull);
        tg = __shfl_sync(0xFFFFFFFFu, tg, 0);
        if (tg >= g.total_tiles) break;
        const int t = (int)g.tile_task[tg];
        const TaskArgs a = g.tasks[t];
        const unsigned long long k = tg - g.tile_first_global[t];
        switch (a.kind) {
        case K_F32: mixed_tile_k<K_F32>(a, k, g.tile_blocks, s_crc, L, lane); break;
        case K_F64: mixed_tile_k<K_F64>(a, k, g.tile_blocks, s_crc, L, lane); break;
        case K_B1: mixed_tile_k<K_B1>(a, k, g.tile_blocks, s_crc, L, lane); break;
        case K_B4: mixed_tile_k<K_B4>(a, k, g.tile_blocks, s_crc, L, lane); break;
        case K_B8: mixed_tile_k<K_B8>(a, k, g.tile_blocks, s_crc, L, lane); break;
        default: break;
        }
    }
}

constexpr int kMixedWarps = 16;

int launch_mixed(const MixedDev &g, int ctas_per_sm, cudaStream_t s)
{
    if (g.total_tiles == 0) return FT_OK;
    auto fn = batched_mixed_kernel<kMixedWarps>;
    int sms = 0, per_sm = 0;
    int rc = occupancy(reinterpret_cast<const void *>(fn), kMixedWarps * 32, kSmemBytes, &sms, &per_sm);
    if (rc != FT_OK) return rc;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    unsigned long long grid = (g.total_tiles + kMixedWarps - 1) / kMixedWarps;
    const unsigned long long cap = (unsigned long long)sms * per_sm;
    if (grid > cap) grid = cap;
    fn<<<(unsigned)grid, kMixedWarps * 32, kSmemBytes, s>>>(g);
    return check_launch(1);
}

}  // namespace ftv
