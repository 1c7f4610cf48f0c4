// host_vote.cu -- ft_vote_host: a vote whose replicas, output, digests and
// statistics live in host memory (for instance a replica that a CPU kernel
// produced in the paper's heterogeneous DMR mode, Sec. IV.D).
//
// The vote is cut into chunks of whole 4 KiB blocks.  Chunk k's replicas are
// uploaded on one stream while chunk k-1 is voted on a second and chunk k-2's
// voted bytes and digests are downloaded on a third, through two sets of
// device staging buffers, so that both directions of PCIe and the voter run
// at once.  Each chunk is an ordinary single-task vote (vote_desc) into its
// own statistics; the host adds the chunks' counts and takes the smallest
// first index, shifted by each chunk's first element.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>

#include <cuda_runtime.h>

#include "ftvote.h"
#include "runtime.h"

namespace {

constexpr uint64_t kDefaultChunk = 64ull << 20;

// Device staging of one device, kept between calls and grown on demand.
struct Staging {
    uint8_t *buf = nullptr;        // 2 sets x (R + 1) chunk buffers: replicas, then output
    size_t buf_bytes = 0;
    uint32_t *crc = nullptr;       // 2 sets x chunk / 4096 digests
    size_t crc_words = 0;
    ft_stats *stats = nullptr;     // one per chunk of the call
    size_t nstats = 0;
    ft_stats *host_stats = nullptr;   // pinned copy of the chunks' statistics
    cudaStream_t up = nullptr, comp = nullptr, down = nullptr;
    cudaEvent_t uploaded[2] = {}, voted[2] = {}, downloaded[2] = {};
    bool ready = false;
};

std::mutex g_mu;
std::map<int, Staging> g_staging;

int ensure(Staging &st, size_t buf_bytes, size_t crc_words, size_t nstats)
{
    cudaError_t e;
    if (!st.ready) {
        if ((e = cudaStreamCreateWithFlags(&st.up, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&st.comp, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&st.down, cudaStreamNonBlocking)) != cudaSuccess)
            return ftv::cuda_fail(e);
        for (int s = 0; s < 2; ++s)
            if ((e = cudaEventCreateWithFlags(&st.uploaded[s], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&st.voted[s], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&st.downloaded[s], cudaEventDisableTiming)) != cudaSuccess)
                return ftv::cuda_fail(e);
        st.ready = true;
    }
    if (buf_bytes > st.buf_bytes) {
        if (st.buf) cudaFree(st.buf);
        st.buf = nullptr;
        st.buf_bytes = 0;
        if ((e = cudaMalloc(&st.buf, buf_bytes)) != cudaSuccess) return ftv::cuda_fail(e);
        st.buf_bytes = buf_bytes;
    }
    if (crc_words > st.crc_words) {
        if (st.crc) cudaFree(st.crc);
        st.crc = nullptr;
        st.crc_words = 0;
        if ((e = cudaMalloc(&st.crc, crc_words * sizeof(uint32_t))) != cudaSuccess) return ftv::cuda_fail(e);
        st.crc_words = crc_words;
    }
    if (nstats > st.nstats) {
        if (st.stats) cudaFree(st.stats);
        if (st.host_stats) cudaFreeHost(st.host_stats);
        st.stats = nullptr;
        st.host_stats = nullptr;
        st.nstats = 0;
        if ((e = cudaMalloc(&st.stats, nstats * sizeof(ft_stats))) != cudaSuccess) return ftv::cuda_fail(e);
        if ((e = cudaMallocHost(&st.host_stats, nstats * sizeof(ft_stats))) != cudaSuccess)
            return ftv::cuda_fail(e);
        st.nstats = nstats;
    }
    return FT_OK;
}

}  // namespace

extern "C" int ft_vote_host(const ft_vote_desc *desc, uint64_t chunk_bytes)
{
    int rc = ftv::validate_desc(desc);
    if (rc != FT_OK) return rc;
    if (chunk_bytes == 0) chunk_bytes = kDefaultChunk;
    if (chunk_bytes % FT_BLOCK_BYTES || chunk_bytes > (1ull << 34)) return FT_EINVAL;
    const int R = desc->R;
    const size_t esize = ftv::dtype_size(desc->dtype);
    const uint64_t nbytes = desc->n * esize;
    const uint64_t nchunks = (nbytes + chunk_bytes - 1) / chunk_bytes;
    ft_stats total;
    for (int r = 0; r < FT_MAX_R; ++r) {
        total.mismatch[r] = 0;
        total.first_mismatch[r] = -1;
    }
    total.no_majority = 0;
    total.first_no_majority = -1;
    if (nbytes == 0) {
        *desc->stats = total;
        return FT_OK;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ftv::cuda_fail(e);
    std::lock_guard<std::mutex> lk(g_mu);
    Staging &st = g_staging[dev];
    const size_t crc_per_chunk = chunk_bytes / FT_BLOCK_BYTES;
    if ((rc = ensure(st, 2ull * (R + 1) * chunk_bytes, 2 * crc_per_chunk, nchunks)) != FT_OK) return rc;

    const uint8_t *const *hrep = reinterpret_cast<const uint8_t *const *>(desc->replicas);
    uint8_t *hout = static_cast<uint8_t *>(desc->out);
    for (uint64_t k = 0; k < nchunks; ++k) {
        const int s = (int)(k & 1);
        const uint64_t off = k * chunk_bytes;
        const uint64_t len = std::min<uint64_t>(chunk_bytes, nbytes - off);
        uint8_t *set = st.buf + (size_t)s * (R + 1) * chunk_bytes;
        uint32_t *dcrc = st.crc + (size_t)s * crc_per_chunk;
        // upload: the set's replica buffers are free once chunk k-2 was voted
        if ((e = cudaStreamWaitEvent(st.up, st.voted[s], 0)) != cudaSuccess) return ftv::cuda_fail(e);
        for (int r = 0; r < R; ++r)
            if ((e = cudaMemcpyAsync(set + (size_t)r * chunk_bytes, hrep[r] + off, len, cudaMemcpyHostToDevice,
                                     st.up)) != cudaSuccess)
                return ftv::cuda_fail(e);
        if ((e = cudaEventRecord(st.uploaded[s], st.up)) != cudaSuccess) return ftv::cuda_fail(e);
        // vote: after the upload, and once chunk k-2's output has been downloaded
        if ((e = cudaStreamWaitEvent(st.comp, st.uploaded[s], 0)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(st.comp, st.downloaded[s], 0)) != cudaSuccess)
            return ftv::cuda_fail(e);
        ft_vote_desc d = *desc;
        for (int r = 0; r < R; ++r) d.replicas[r] = set + (size_t)r * chunk_bytes;
        d.n = len / esize;
        d.out = set + (size_t)R * chunk_bytes;
        d.block_crc = desc->block_crc ? dcrc : nullptr;
        d.stats = st.stats + k;
        if ((rc = ftv::vote_desc(&d, st.comp, nullptr)) != FT_OK) return rc;
        if ((e = cudaEventRecord(st.voted[s], st.comp)) != cudaSuccess) return ftv::cuda_fail(e);
        // download the voted bytes and the chunk's digests
        if ((e = cudaStreamWaitEvent(st.down, st.voted[s], 0)) != cudaSuccess) return ftv::cuda_fail(e);
        if ((e = cudaMemcpyAsync(hout + off, d.out, len, cudaMemcpyDeviceToHost, st.down)) != cudaSuccess)
            return ftv::cuda_fail(e);
        if (desc->block_crc) {
            const uint64_t nblk = (len + FT_BLOCK_BYTES - 1) / FT_BLOCK_BYTES;
            if ((e = cudaMemcpyAsync(desc->block_crc + off / FT_BLOCK_BYTES, dcrc, nblk * sizeof(uint32_t),
                                     cudaMemcpyDeviceToHost, st.down)) != cudaSuccess)
                return ftv::cuda_fail(e);
        }
        if ((e = cudaEventRecord(st.downloaded[s], st.down)) != cudaSuccess) return ftv::cuda_fail(e);
    }
    // the chunks' statistics, after the last vote
    if ((e = cudaMemcpyAsync(st.host_stats, st.stats, nchunks * sizeof(ft_stats), cudaMemcpyDeviceToHost,
                             st.comp)) != cudaSuccess)
        return ftv::cuda_fail(e);
    if ((e = cudaStreamSynchronize(st.comp)) != cudaSuccess || (e = cudaStreamSynchronize(st.down)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st.up)) != cudaSuccess)
        return ftv::cuda_fail(e);
    for (uint64_t k = 0; k < nchunks; ++k) {
        const ft_stats &c = st.host_stats[k];
        const int64_t first_elem = (int64_t)(k * chunk_bytes / esize);
        for (int r = 0; r < R; ++r) {
            total.mismatch[r] += c.mismatch[r];
            if (c.first_mismatch[r] >= 0 && total.first_mismatch[r] < 0)
                total.first_mismatch[r] = c.first_mismatch[r] + first_elem;
        }
        total.no_majority += c.no_majority;
        if (c.first_no_majority >= 0 && total.first_no_majority < 0)
            total.first_no_majority = c.first_no_majority + first_elem;
    }
    *desc->stats = total;
    return FT_OK;
}
