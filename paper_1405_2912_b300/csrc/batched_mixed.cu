// batched_mixed.cu -- the batched voter as one persistent kernel for a whole
// batch of mixed element kinds and replica counts: a warp claims the next
// tile of the batch, whatever its task's kind and R, and votes it through the
// (kind, R) instance of the tile routine.  The plan's autotuner times it
// against one kernel per (kind, R) group and keeps the faster.
#include "batched.h"
#include "common.cuh"
#include "runtime.h"
#include "tile_vote.cuh"

namespace ftv {

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
        mixed_tile_any(a, tg - g.tile_first_global[t], g.tile_blocks, 0ull, nullptr, s_crc, L, lane);
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
