// ckpt.cu -- digest-driven checkpoint of a device buffer into a host copy
// (ft_ckpt_create / ft_ckpt_sync / ft_ckpt_restore).
//
// The paper's memory manager keeps "siblings" of every registered area and
// transfers data only when necessary (Sec. IV.A); before a kernel runs in the
// light-weight mode it makes sure that a backup copy of the data exists, so a
// faulty run can be rolled back (Sec. IV.C).  Here the per-4-KiB CRC32C of the
// buffer decides which blocks have changed since the last checkpoint: only
// those cross PCIe.
//   sync:    device -> host.  Digest the device buffer, compare with the
//            digests of the last checkpoint, compact the changed block numbers
//            on the GPU, gather those blocks into a staging area, copy them to
//            pinned memory in chunks and scatter them into the host copy.
//   restore: host -> device.  Digest the device buffer, compare with the
//            checkpoint's digests, and upload only the blocks that differ
//            (gathered on the host, scattered on the GPU).
// A change that leaves a block's CRC32C unchanged is not seen (CRC32C detects
// every change of up to a few bits in a 4 KiB block and misses a random
// change with probability 2^-32).
#include <algorithm>
#include <cstring>
#include <new>

#include "common.cuh"
#include "runtime.h"

namespace ftv {

// changed[] <- numbers of the blocks whose digest differs (or all blocks when
// `all`), in any order; *count <- how many.
__global__ void ckpt_compare_kernel(const uint32_t *__restrict__ now, const uint32_t *__restrict__ then,
                                    unsigned long long nblocks, int all, unsigned long long *__restrict__ changed,
                                    unsigned long long *__restrict__ count)
{
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ch = i < nblocks && (all || now[i] != then[i]);
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, ch);
    if (!mask) return;
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == __ffs(mask) - 1) base = atomicAdd(count, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xFFFFFFFFu, base, __ffs(mask) - 1);
    if (ch) changed[base + __popc(mask & ((1u << lane) - 1))] = i;
}

// stage[k] <- block changed[first + k] of buf, k < min(*count - first, cap), one
// warp per block (whole blocks; the partial last block is copied by bytes).
__global__ void ckpt_gather_kernel(const uint8_t *__restrict__ buf, unsigned long long nbytes,
                                   const unsigned long long *__restrict__ changed,
                                   const unsigned long long *__restrict__ count, unsigned long long first,
                                   unsigned long long cap, uint8_t *__restrict__ stage)
{
    const unsigned long long n = *count > first ? min(*count - first, cap) : 0ull;
    const int lane = threadIdx.x & 31;
    const unsigned long long wid = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    for (unsigned long long k = wid; k < n; k += nw) {
        const unsigned long long b = changed[first + k];
        const unsigned long long off = b * kBlockBytes;
        const unsigned long long len = min((unsigned long long)kBlockBytes, nbytes - off);
        uint8_t *dst = stage + k * kBlockBytes;
        if (len == (unsigned long long)kBlockBytes) {
            const uint4 *s = reinterpret_cast<const uint4 *>(buf + off);
#pragma unroll
            for (int t = 0; t < 8; ++t) reinterpret_cast<uint4 *>(dst)[lane + 32 * t] = s[lane + 32 * t];
        } else {
            for (unsigned long long i = lane; i < len; i += 32) dst[i] = buf[off + i];
        }
    }
}

// block blocks[k] of buf <- stage[k], k < n.
__global__ void ckpt_scatter_kernel(uint8_t *__restrict__ buf, unsigned long long nbytes,
                                    const unsigned long long *__restrict__ blocks, unsigned long long n,
                                    const uint8_t *__restrict__ stage)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long wid = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    for (unsigned long long k = wid; k < n; k += nw) {
        const unsigned long long off = blocks[k] * kBlockBytes;
        const unsigned long long len = min((unsigned long long)kBlockBytes, nbytes - off);
        const uint8_t *src = stage + k * kBlockBytes;
        if (len == (unsigned long long)kBlockBytes) {
#pragma unroll
            for (int t = 0; t < 8; ++t)
                reinterpret_cast<uint4 *>(buf + off)[lane + 32 * t] = reinterpret_cast<const uint4 *>(src)[lane + 32 * t];
        } else {
            for (unsigned long long i = lane; i < len; i += 32) buf[off + i] = src[i];
        }
    }
}

}  // namespace ftv

struct ft_ckpt {
    unsigned long long nbytes = 0, nblocks = 0;
    uint32_t *d_now = nullptr, *d_then = nullptr;   // digests (device)
    unsigned long long *d_changed = nullptr;        // changed block numbers (device)
    unsigned long long *d_count = nullptr;          // one counter (device)
    uint8_t *d_stage = nullptr;                     // staging blocks (device)
    unsigned long long stage_blocks = 0;
    uint8_t *h_stage = nullptr;                     // pinned staging
    unsigned long long *h_changed = nullptr;        // pinned copy of the block list
    unsigned long long *h_count = nullptr;          // pinned
    bool have = false;                              // d_then holds a checkpoint's digests
};

namespace {

void ckpt_free(ft_ckpt *c)
{
    cudaFree(c->d_now);
    cudaFree(c->d_then);
    cudaFree(c->d_changed);
    cudaFree(c->d_count);
    cudaFree(c->d_stage);
    cudaFreeHost(c->h_stage);
    cudaFreeHost(c->h_changed);
    cudaFreeHost(c->h_count);
    delete c;
}

// Digest buf into d_now and list the blocks that differ from d_then (all
// blocks if there is no checkpoint yet); returns their number in *n.
int ckpt_diff(ft_ckpt *c, const void *buf, cudaStream_t s, bool all, unsigned long long *n)
{
    int rc = ftv::digest(buf, c->nbytes, FT_BLOCK_BYTES, c->d_now, s);
    if (rc != FT_OK) return rc;
    cudaError_t e = cudaMemsetAsync(c->d_count, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return ftv::cuda_fail(e);
    const unsigned grid = (unsigned)((c->nblocks + 255) / 256);
    ftv::ckpt_compare_kernel<<<grid, 256, 0, s>>>(c->d_now, c->d_then, c->nblocks, all ? 1 : 0, c->d_changed,
                                                  c->d_count);
    if ((rc = ftv::check_launch(1)) != FT_OK) return rc;
    if ((e = cudaMemcpyAsync(c->h_count, c->d_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
        return ftv::cuda_fail(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return ftv::cuda_fail(e);
    *n = *c->h_count;
    return FT_OK;
}

unsigned gather_grid(unsigned long long nblocks)
{
    return (unsigned)std::max(1ull, std::min(4096ull, (nblocks * 32 + 255) / 256));
}

}  // namespace

extern "C" {

int ft_ckpt_create(ft_ckpt **out, uint64_t nbytes, uint64_t stage_bytes)
{
    if (!out || nbytes == 0) return FT_EINVAL;
    *out = nullptr;
    ft_ckpt *c = new (std::nothrow) ft_ckpt();
    if (!c) return FT_ENOMEM;
    c->nbytes = nbytes;
    c->nblocks = (nbytes + FT_BLOCK_BYTES - 1) / FT_BLOCK_BYTES;
    if (stage_bytes == 0) stage_bytes = 64ull << 20;
    c->stage_blocks = std::max(1ull, std::min(c->nblocks, (unsigned long long)(stage_bytes / FT_BLOCK_BYTES)));
    cudaError_t e = cudaSuccess;
    const size_t dig = 4 * c->nblocks;
    if ((e = cudaMalloc(&c->d_now, dig)) == cudaSuccess && (e = cudaMalloc(&c->d_then, dig)) == cudaSuccess &&
        (e = cudaMalloc(&c->d_changed, 8 * c->nblocks)) == cudaSuccess &&
        (e = cudaMalloc(&c->d_count, 8)) == cudaSuccess &&
        (e = cudaMalloc(&c->d_stage, c->stage_blocks * FT_BLOCK_BYTES)) == cudaSuccess &&
        (e = cudaMallocHost(&c->h_stage, c->stage_blocks * FT_BLOCK_BYTES)) == cudaSuccess &&
        (e = cudaMallocHost(&c->h_changed, 8 * c->nblocks)) == cudaSuccess &&
        (e = cudaMallocHost(&c->h_count, 8)) == cudaSuccess) {
        *out = c;
        return FT_OK;
    }
    ckpt_free(c);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? FT_ENOMEM : ftv::cuda_fail(e);
}

}  // extern "C"

namespace {

// More than an eighth of a buffer of 64 MiB or more changed: one direct copy
// of the whole buffer is faster than staging the changed blocks and placing
// them one by one on the host (measured on 1 GiB: every block changed, 175 ms
// staged against 19 ms direct; 1 % changed, 2 ms staged).
bool dense_change(const ft_ckpt *c, unsigned long long n)
{
    return c->nbytes >= (64ull << 20) && n * 8 > c->nblocks;
}

}  // namespace

extern "C" {

int ft_ckpt_sync(ft_ckpt *c, const void *dev_buf, void *host_copy, ft_stream stream, uint64_t *blocks_copied)
{
    if (!c || !dev_buf || !host_copy || ((uintptr_t)dev_buf & 15)) return FT_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long n = 0;
    int rc = ckpt_diff(c, dev_buf, s, !c->have, &n);
    if (rc != FT_OK) return rc;
    cudaError_t e;
    if (dense_change(c, n)) {
        if ((e = cudaMemcpyAsync(host_copy, dev_buf, c->nbytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return ftv::cuda_fail(e);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return ftv::cuda_fail(e);
        std::swap(c->d_now, c->d_then);
        c->have = true;
        if (blocks_copied) *blocks_copied = c->nblocks;
        return FT_OK;
    }
    if (n && (e = cudaMemcpyAsync(c->h_changed, c->d_changed, 8 * n, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return ftv::cuda_fail(e);
    uint8_t *host = static_cast<uint8_t *>(host_copy);
    for (unsigned long long first = 0; first < n; first += c->stage_blocks) {
        const unsigned long long k = std::min(c->stage_blocks, n - first);
        ftv::ckpt_gather_kernel<<<gather_grid(k), 256, 0, s>>>(static_cast<const uint8_t *>(dev_buf), c->nbytes,
                                                               c->d_changed, c->d_count, first, c->stage_blocks,
                                                               c->d_stage);
        if ((rc = ftv::check_launch(1)) != FT_OK) return rc;
        if ((e = cudaMemcpyAsync(c->h_stage, c->d_stage, k * FT_BLOCK_BYTES, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
            return ftv::cuda_fail(e);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return ftv::cuda_fail(e);
        for (unsigned long long i = 0; i < k; ++i) {
            const unsigned long long b = c->h_changed[first + i];
            const unsigned long long off = b * FT_BLOCK_BYTES;
            std::memcpy(host + off, c->h_stage + i * FT_BLOCK_BYTES,
                        std::min((unsigned long long)FT_BLOCK_BYTES, c->nbytes - off));
        }
    }
    // the new digests become the checkpoint's
    std::swap(c->d_now, c->d_then);
    c->have = true;
    if (blocks_copied) *blocks_copied = n;
    return FT_OK;
}

int ft_ckpt_restore(ft_ckpt *c, void *dev_buf, const void *host_copy, ft_stream stream, uint64_t *blocks_copied)
{
    if (!c || !dev_buf || !host_copy || ((uintptr_t)dev_buf & 15)) return FT_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!c->have) {
        // no digests of the host copy yet: upload everything
        cudaError_t e = cudaMemcpyAsync(dev_buf, host_copy, c->nbytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return ftv::cuda_fail(e);
        int rc = ftv::digest(dev_buf, c->nbytes, FT_BLOCK_BYTES, c->d_then, s);
        if (rc != FT_OK) return rc;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return ftv::cuda_fail(e);
        c->have = true;
        if (blocks_copied) *blocks_copied = c->nblocks;
        return FT_OK;
    }
    unsigned long long n = 0;
    int rc = ckpt_diff(c, dev_buf, s, false, &n);
    if (rc != FT_OK) return rc;
    cudaError_t e;
    if (dense_change(c, n)) {
        if ((e = cudaMemcpyAsync(dev_buf, host_copy, c->nbytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return ftv::cuda_fail(e);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return ftv::cuda_fail(e);
        if (blocks_copied) *blocks_copied = c->nblocks;
        return FT_OK;
    }
    if (n && (e = cudaMemcpyAsync(c->h_changed, c->d_changed, 8 * n, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return ftv::cuda_fail(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return ftv::cuda_fail(e);
    const uint8_t *host = static_cast<const uint8_t *>(host_copy);
    for (unsigned long long first = 0; first < n; first += c->stage_blocks) {
        const unsigned long long k = std::min(c->stage_blocks, n - first);
        for (unsigned long long i = 0; i < k; ++i) {
            const unsigned long long off = c->h_changed[first + i] * FT_BLOCK_BYTES;
            std::memcpy(c->h_stage + i * FT_BLOCK_BYTES, host + off,
                        std::min((unsigned long long)FT_BLOCK_BYTES, c->nbytes - off));
        }
        if ((e = cudaMemcpyAsync(c->d_stage, c->h_stage, k * FT_BLOCK_BYTES, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
            return ftv::cuda_fail(e);
        ftv::ckpt_scatter_kernel<<<gather_grid(k), 256, 0, s>>>(static_cast<uint8_t *>(dev_buf), c->nbytes,
                                                                c->d_changed + first, k, c->d_stage);
        if ((rc = ftv::check_launch(1)) != FT_OK) return rc;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return ftv::cuda_fail(e);
    }
    // the device buffer equals the checkpoint again: d_then stays valid
    if (blocks_copied) *blocks_copied = n;
    return FT_OK;
}

int ft_ckpt_forget(ft_ckpt *c)
{
    if (!c) return FT_EINVAL;
    c->have = false;
    return FT_OK;
}

int ft_ckpt_destroy(ft_ckpt *c)
{
    if (!c) return FT_EINVAL;
    ckpt_free(c);
    return FT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Areas with a host and a device sibling (Sec. IV.A): each sibling carries the
// version of the data it holds; a request brings the requested sibling up to
// the newest version, moving only the 4 KiB blocks whose digest differs, and a
// write request bumps its version.  Before a write, the previous version is
// made to exist in the other memory too, so that a faulty run can be rolled
// back from it (the fault-tolerant rule of Sec. IV.A / IV.C).
// ---------------------------------------------------------------------------
struct ft_area {
    void *host = nullptr;              // caller's host memory (the host sibling)
    void *dev = nullptr;               // device sibling (library-owned)
    unsigned long long bytes = 0;
    unsigned long long version[2] = {0, 0};
    bool valid[2] = {false, false};
    ft_ckpt *ck = nullptr;             // digests of the host sibling's content, as seen on the device
};

extern "C" {

int ft_area_create(ft_area **out, void *host_ptr, uint64_t bytes)
{
    if (!out || !host_ptr || bytes == 0) return FT_EINVAL;
    *out = nullptr;
    ft_area *a = new (std::nothrow) ft_area();
    if (!a) return FT_ENOMEM;
    a->host = host_ptr;
    a->bytes = bytes;
    a->version[FT_MEM_HOST] = 1;
    a->valid[FT_MEM_HOST] = true;
    int rc = ft_ckpt_create(&a->ck, bytes, 0);
    if (rc == FT_OK) {
        const cudaError_t e = cudaMalloc(&a->dev, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = e == cudaErrorMemoryAllocation ? FT_ENOMEM : ftv::cuda_fail(e);
        }
    }
    if (rc != FT_OK) {
        if (a->ck) ft_ckpt_destroy(a->ck);
        delete a;
        return rc;
    }
    *out = a;
    return FT_OK;
}

// Bring sibling m up to the newest version from the other one.
static int area_refresh(ft_area *a, int m, cudaStream_t s, unsigned long long *moved)
{
    const int o = 1 - m;
    uint64_t k = 0;
    int rc = FT_OK;
    if (m == FT_MEM_DEVICE) rc = ft_ckpt_restore(a->ck, a->dev, a->host, s, &k);
    else rc = ft_ckpt_sync(a->ck, a->dev, a->host, s, &k);
    if (rc != FT_OK) return rc;
    a->version[m] = a->version[o];
    a->valid[m] = true;
    *moved += k;
    return FT_OK;
}

int ft_area_request(ft_area *a, int32_t memory, int32_t access, void **ptr, ft_stream stream, uint64_t *blocks_moved)
{
    if (!a || !ptr || (memory != FT_MEM_HOST && memory != FT_MEM_DEVICE) ||
        (access & ~(FT_ACCESS_READ | FT_ACCESS_WRITE)) || !access)
        return FT_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int m = memory, o = 1 - memory;
    if (!a->valid[m] && !a->valid[o]) return FT_EINVAL;   // both siblings lost
    unsigned long long moved = 0;
    const unsigned long long newest =
        std::max(a->valid[m] ? a->version[m] : 0ull, a->valid[o] ? a->version[o] : 0ull);
    int rc = FT_OK;
    if (!a->valid[m] || a->version[m] < newest) rc = area_refresh(a, m, s, &moved);
    if (rc == FT_OK && (access & FT_ACCESS_WRITE)) {
        // keep the version about to be overwritten in the other memory
        if (!a->valid[o] || a->version[o] < a->version[m]) rc = area_refresh(a, o, s, &moved);
        if (rc == FT_OK) {
            a->version[m] += 1;
            // the device side no longer knows the digests of a rewritten host copy
            if (m == FT_MEM_HOST) ft_ckpt_forget(a->ck);
        }
    }
    if (rc != FT_OK) return rc;
    *ptr = m == FT_MEM_HOST ? a->host : a->dev;
    if (blocks_moved) *blocks_moved = moved;
    return FT_OK;
}

int ft_area_invalidate(ft_area *a, int32_t memory)
{
    if (!a || (memory != FT_MEM_HOST && memory != FT_MEM_DEVICE)) return FT_EINVAL;
    a->valid[memory] = false;
    if (memory == FT_MEM_HOST) ft_ckpt_forget(a->ck);
    return FT_OK;
}

int ft_area_versions(const ft_area *a, uint64_t *host_version, uint64_t *device_version)
{
    if (!a) return FT_EINVAL;
    if (host_version) *host_version = a->valid[FT_MEM_HOST] ? a->version[FT_MEM_HOST] : 0;
    if (device_version) *device_version = a->valid[FT_MEM_DEVICE] ? a->version[FT_MEM_DEVICE] : 0;
    return FT_OK;
}

int ft_area_destroy(ft_area *a)
{
    if (!a) return FT_EINVAL;
    cudaFree(a->dev);
    ft_ckpt_destroy(a->ck);
    delete a;
    return FT_OK;
}

}  // extern "C"
