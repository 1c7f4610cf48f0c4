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

// The statistics reset before a single vote.  It lets the voter kernel, which
// is launched right after it as a programmatic dependent, start at once: the
// voter touches the statistics only after pdl_wait().
__global__ void reset_stats_kernel(ft_stats *s)
{
    pdl_release();
    reset_stats(s, threadIdx.x);
}

// ---------------------------------------------------------------------------
// K1: persistent single-task voter.  Warps take 4 KiB blocks in grid-stride
// order; consecutive warps of a CTA take consecutive blocks.  PF: each warp
// prefetches its next block into L2.
// ---------------------------------------------------------------------------
template <int K, int R, int W, bool PF>
__global__ void __launch_bounds__(W * 32, 1) vote_kernel(const TaskArgs a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *s_crc = reinterpret_cast<uint32_t *>(smem);
    load_crc_tables<W>(s_crc);
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    CrcLane L;
    L.init(lane);
    LaneStats<R> st;
    st.init();
    const unsigned long long step = (unsigned long long)gridDim.x * W;
    const unsigned long long gw = (unsigned long long)blockIdx.x * W + w;
    for (unsigned long long b = gw; b < a.nfull; b += step)
        vote_full_block<K, R>(a, b, PF ? b + step : ~0ull, s_crc, L, st, lane);
    if (a.tail_bytes && a.nfull % step == gw) {
        // the partial last block goes to the warp whose turn it would be
        LaneStats<R> ts;
        ts.init();
        vote_tail_block<K, R>(a, a.nfull, s_crc, L, ts, lane);
        st.merge(ts);
    }
    pdl_wait();               // the statistics reset has completed
    st.flush(a.stats, lane);
}

template <int K, int R, int kVoteWarps, bool PF>
static int launch_vote_shape(const TaskArgs &a, cudaStream_t s, const VoteLaunch *cfg)
{
    auto fn = vote_kernel<K, R, kVoteWarps, PF>;
    const size_t smem = kSmemBytes;
    int sms = 0, per_sm = 0;
    int rc = occupancy(reinterpret_cast<const void *>(fn), kVoteWarps * 32, smem, &sms, &per_sm);
    if (rc != FT_OK) return rc;
    if (cfg && cfg->ctas_per_sm > 0 && cfg->ctas_per_sm < per_sm) per_sm = cfg->ctas_per_sm;
    const unsigned long long nblk = a.nfull + (a.tail_bytes ? 1 : 0);
    unsigned long long grid = (nblk + kVoteWarps - 1) / kVoteWarps;
    const unsigned long long cap = (unsigned long long)sms * per_sm;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    // a programmatic dependent of the statistics reset launched just before
    // it: the kernel may start while the reset runs (it reads the replicas and
    // writes the output and digests, which the reset does not touch) and waits
    // for it only before its statistics flush
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
    const cudaError_t e = cudaLaunchKernelEx(&lc, fn, a);
    if (e != cudaSuccess) return cuda_fail(e);
    return check_launch(1);
}

// Votes of up to 32768 blocks (128 MiB of output) have at most a few blocks
// per warp, so latency, not bandwidth, sets their time: for them the shape
// with more warps and no prefetch measured faster even where the policy
// prefers the prefetching one (f32 R = 3: 3 x 16M 52 against 58 us, 3 x 4M 18
// against 20 us; equal at 3 x 64M; 6.7 against 6.25 TB/s the other way at
// 3 x 256M).
constexpr unsigned long long kSmallVoteBlocks = 32768;

template <int K, int R>
static int launch_vote_kr(const TaskArgs &a, cudaStream_t s, const VoteLaunch *cfg)
{
    using P = VotePolicy<K, R>;
    if constexpr (P::kPrefetch) {
        if (a.nfull + (a.tail_bytes ? 1 : 0) <= kSmallVoteBlocks) return launch_vote_shape<K, R, 16, false>(a, s, cfg);
    }
    return launch_vote_shape<K, R, P::kWarps, P::kPrefetch>(a, s, cfg);
}

template <int K>
static int launch_vote_k(const TaskArgs &a, cudaStream_t s, const VoteLaunch *cfg)
{
    switch (a.R) {
    case 2: return launch_vote_kr<K, 2>(a, s, cfg);
    case 3: return launch_vote_kr<K, 3>(a, s, cfg);
    case 4: return launch_vote_kr<K, 4>(a, s, cfg);
    case 5: return launch_vote_kr<K, 5>(a, s, cfg);
    case 6: return launch_vote_kr<K, 6>(a, s, cfg);
    case 7: return launch_vote_kr<K, 7>(a, s, cfg);
    case 8: return launch_vote_kr<K, 8>(a, s, cfg);
    default: return FT_EINVAL;
    }
}

// Only ever launched directly after the statistics reset on the same stream
// (vote_desc): the programmatic dependency it is launched with relaxes the
// wait on exactly that kernel.
static int launch_vote(const TaskArgs &a, cudaStream_t s, const VoteLaunch *cfg)
{
    switch (a.kind) {
    case K_F32: return launch_vote_k<K_F32>(a, s, cfg);
    case K_F64: return launch_vote_k<K_F64>(a, s, cfg);
    case K_B1: return launch_vote_k<K_B1>(a, s, cfg);
    case K_B4: return launch_vote_k<K_B4>(a, s, cfg);
    case K_B8: return launch_vote_k<K_B8>(a, s, cfg);
    default: return FT_EINVAL;
    }
}

int vote_desc(const ft_vote_desc *desc, cudaStream_t s, const VoteLaunch *cfg)
{
    int rc = validate_desc(desc);
    if (rc != FT_OK) return rc;
    reset_stats_kernel<<<1, FT_MAX_R + 1, 0, s>>>(desc->stats);
    if ((rc = check_launch(1)) != FT_OK) return rc;
    if (desc->n == 0) return FT_OK;
    return launch_vote(make_task_args(desc), s, cfg);
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

// Warps per CTA of the digest kernel: 20 for 4 KiB blocks (each warp's chunks
// are then a stream of independent blocks), 16 for larger ones.  Measured on
// 1 GiB: 4 KiB blocks 5.07 against 4.98 TB/s with 16 warps; 64 KiB blocks
// 5.45 with 16 against 5.13 with 20 (fewer, longer blocks per warp).
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
    if (block_bytes == FT_BLOCK_BYTES) return launch_digest<20>(buf, nbytes, block_bytes, out, s);
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
