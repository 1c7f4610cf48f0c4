// host_vote.cu -- ft_vote_host: a vote whose buffers may live in host memory
// (for instance a replica that a CPU kernel produced in the paper's
// heterogeneous DMR mode, Sec. IV.D), each pointer host or device.
//
// The vote is cut into chunks of whole 4 KiB blocks.  Chunk k's host-resident
// replicas are uploaded on one stream while chunk k-1 is voted on a second and
// chunk k-2's voted bytes and digests are downloaded on a third, through two
// sets of device staging buffers, so that both directions of PCIe and the
// voter run at once.  Device-resident replicas are read in place and a
// device-resident output or digest array is written in place.  Each chunk is
// an ordinary single-task vote (vote_desc) into its own statistics; the host
// adds the chunks' counts and takes the smallest first index, shifted by each
// chunk's first element.
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

// Where a pointer lives: 1 = device or managed memory of device `dev` (used
// in place), 0 = host memory, pinned or pageable (staged), -1 = another
// device's memory (rejected).
int residence(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();           // an address the runtime does not know: plain host memory
        return 0;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return a.device == dev ? 1 : -1;
    return 0;
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
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ftv::cuda_fail(e);

    const uint8_t *const *hrep = reinterpret_cast<const uint8_t *const *>(desc->replicas);
    uint8_t *hout = static_cast<uint8_t *>(desc->out);
    bool rep_dev[FT_MAX_R];
    for (int r = 0; r < R; ++r) {
        const int where = residence(hrep[r], dev);
        if (where < 0) return FT_EINVAL;
        rep_dev[r] = where == 1;
    }
    const int out_where = residence(hout, dev);
    const int crc_where = desc->block_crc ? residence(desc->block_crc, dev) : 0;
    const int stats_where = residence(desc->stats, dev);
    if (out_where < 0 || crc_where < 0 || stats_where < 0) return FT_EINVAL;
    auto put_stats = [&]() -> int {
        if (stats_where == 0) {
            *desc->stats = total;
            return FT_OK;
        }
        const cudaError_t pe = cudaMemcpy(desc->stats, &total, sizeof(total), cudaMemcpyHostToDevice);
        return pe == cudaSuccess ? FT_OK : ftv::cuda_fail(pe);
    };
    if (nbytes == 0) return put_stats();

    std::lock_guard<std::mutex> lk(g_mu);
    Staging &st = g_staging[dev];
    const size_t crc_per_chunk = chunk_bytes / FT_BLOCK_BYTES;
    if ((rc = ensure(st, 2ull * (R + 1) * chunk_bytes, 2 * crc_per_chunk, nchunks)) != FT_OK) return rc;
    // The pipeline; an error part-way leaves copies in flight into the caller's
    // buffers, so every exit below waits for the three streams first.
    auto pipeline = [&]() -> int {
        for (uint64_t k = 0; k < nchunks; ++k) {
            const int s = (int)(k & 1);
            const uint64_t off = k * chunk_bytes;
            const uint64_t len = std::min<uint64_t>(chunk_bytes, nbytes - off);
            uint8_t *set = st.buf + (size_t)s * (R + 1) * chunk_bytes;
            uint32_t *dcrc = st.crc + (size_t)s * crc_per_chunk;
            // upload: the set's replica buffers are free once chunk k-2 was voted
            if ((e = cudaStreamWaitEvent(st.up, st.voted[s], 0)) != cudaSuccess) return ftv::cuda_fail(e);
            for (int r = 0; r < R; ++r)
                if (!rep_dev[r] && (e = cudaMemcpyAsync(set + (size_t)r * chunk_bytes, hrep[r] + off, len,
                                                        cudaMemcpyHostToDevice, st.up)) != cudaSuccess)
                    return ftv::cuda_fail(e);
            if ((e = cudaEventRecord(st.uploaded[s], st.up)) != cudaSuccess) return ftv::cuda_fail(e);
            // vote: after the upload, and once chunk k-2's output has been downloaded
            if ((e = cudaStreamWaitEvent(st.comp, st.uploaded[s], 0)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(st.comp, st.downloaded[s], 0)) != cudaSuccess)
                return ftv::cuda_fail(e);
            ft_vote_desc d = *desc;
            for (int r = 0; r < R; ++r) d.replicas[r] = rep_dev[r] ? hrep[r] + off : set + (size_t)r * chunk_bytes;
            d.n = len / esize;
            d.out = out_where == 1 ? hout + off : set + (size_t)R * chunk_bytes;
            d.block_crc = !desc->block_crc ? nullptr : crc_where == 1 ? desc->block_crc + off / FT_BLOCK_BYTES : dcrc;
            d.stats = st.stats + k;
            if ((rc = ftv::vote_desc(&d, st.comp, nullptr)) != FT_OK) return rc;
            if ((e = cudaEventRecord(st.voted[s], st.comp)) != cudaSuccess) return ftv::cuda_fail(e);
            // download the voted bytes and the chunk's digests
            if ((e = cudaStreamWaitEvent(st.down, st.voted[s], 0)) != cudaSuccess) return ftv::cuda_fail(e);
            if (out_where == 0 &&
                (e = cudaMemcpyAsync(hout + off, d.out, len, cudaMemcpyDeviceToHost, st.down)) != cudaSuccess)
                return ftv::cuda_fail(e);
            if (desc->block_crc && crc_where == 0) {
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
        return FT_OK;
    };
    if ((rc = pipeline()) != FT_OK) {
        cudaStreamSynchronize(st.up);
        cudaStreamSynchronize(st.comp);
        cudaStreamSynchronize(st.down);
        return rc;
    }
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
    return put_stats();
}
