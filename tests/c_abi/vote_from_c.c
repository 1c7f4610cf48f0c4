/*
 * A plain C client of libftvote.so: no Python, no torch.  Device memory comes
 * from the CUDA runtime; the expected results are worked out here from the
 * construction of the inputs (and a bit-at-a-time CRC32C of the voted bytes).
 * The same vote through ft_vote_host on the host arrays must agree with it.
 * Prints "C ABI OK" and exits 0 on success.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "ftvote.h"

static uint32_t crc32c_bits(const unsigned char *p, size_t n)
{
    uint32_t c = 0xFFFFFFFFu;
    for (size_t i = 0; i < n; ++i) {
        c ^= p[i];
        for (int k = 0; k < 8; ++k) c = (c & 1u) ? (c >> 1) ^ 0x82F63B78u : (c >> 1);
    }
    return c ^ 0xFFFFFFFFu;
}

#define CHECK(cond, msg) do { if (!(cond)) { printf("FAIL: %s\n", msg); return 1; } } while (0)

int main(void)
{
    const uint64_t n = 100003;                 /* 97 full 4 KiB blocks and a partial one */
    const size_t bytes = n * sizeof(float);
    const uint64_t nblk = (bytes + 4095) / 4096;
    float *h[3];
    for (int r = 0; r < 3; ++r) h[r] = (float *)malloc(bytes);
    for (uint64_t i = 0; i < n; ++i) h[0][i] = h[1][i] = h[2][i] = (float)i * 0.5f - 1000.0f;
    h[1][777] = nextafterf(h[1][777], INFINITY);   /* 1 ULP: equal under the tolerance */
    h[2][10] += 1.0f;                               /* two real faults in replica 2 */
    h[2][50000] = -h[2][50000];

    void *d_rep[3], *d_out;
    uint32_t *d_crc;
    ft_stats *d_stats;
    for (int r = 0; r < 3; ++r) {
        CHECK(cudaMalloc(&d_rep[r], bytes) == cudaSuccess, "cudaMalloc");
        CHECK(cudaMemcpy(d_rep[r], h[r], bytes, cudaMemcpyHostToDevice) == cudaSuccess, "cudaMemcpy");
    }
    CHECK(cudaMalloc(&d_out, bytes) == cudaSuccess, "cudaMalloc out");
    CHECK(cudaMalloc((void **)&d_crc, 4 * nblk) == cudaSuccess, "cudaMalloc crc");
    CHECK(cudaMalloc((void **)&d_stats, sizeof(ft_stats)) == cudaSuccess, "cudaMalloc stats");

    ft_vote_desc d;
    memset(&d, 0, sizeof d);
    for (int r = 0; r < 3; ++r) d.replicas[r] = d_rep[r];
    d.R = 3;
    d.dtype = FT_F32;
    d.n = n;
    d.abs_tol = 1e-6;
    d.rel_tol = 1e-5;
    d.out = d_out;
    d.block_crc = d_crc;
    d.stats = d_stats;
    CHECK(ft_vote(&d, NULL) == FT_OK, "ft_vote");

    uint32_t *d_dig;
    CHECK(cudaMalloc((void **)&d_dig, 4 * nblk) == cudaSuccess, "cudaMalloc digest");
    CHECK(ft_digest(d_out, bytes, 4096, d_dig, NULL) == FT_OK, "ft_digest");
    CHECK(cudaDeviceSynchronize() == cudaSuccess, "sync");

    float *out = (float *)malloc(bytes);
    uint32_t *crc = (uint32_t *)malloc(4 * nblk), *dig = (uint32_t *)malloc(4 * nblk);
    ft_stats s;
    CHECK(cudaMemcpy(out, d_out, bytes, cudaMemcpyDeviceToHost) == cudaSuccess, "copy out");
    CHECK(cudaMemcpy(crc, d_crc, 4 * nblk, cudaMemcpyDeviceToHost) == cudaSuccess, "copy crc");
    CHECK(cudaMemcpy(dig, d_dig, 4 * nblk, cudaMemcpyDeviceToHost) == cudaSuccess, "copy digest");
    CHECK(cudaMemcpy(&s, d_stats, sizeof s, cudaMemcpyDeviceToHost) == cudaSuccess, "copy stats");

    /* replica 0 is equal to a majority everywhere, so the vote is replica 0 */
    CHECK(memcmp(out, h[0], bytes) == 0, "voted values");
    CHECK(s.mismatch[0] == 0 && s.mismatch[1] == 0 && s.mismatch[2] == 2, "mismatch counts");
    CHECK(s.first_mismatch[0] == -1 && s.first_mismatch[1] == -1 && s.first_mismatch[2] == 10, "first indices");
    CHECK(s.no_majority == 0 && s.first_no_majority == -1, "majority");
    for (uint64_t b = 0; b < nblk; ++b) {
        const size_t len = (b + 1) * 4096 <= bytes ? 4096 : bytes - b * 4096;
        CHECK(crc[b] == crc32c_bits((const unsigned char *)out + b * 4096, len), "block CRC32C");
        CHECK(dig[b] == crc[b], "ft_digest equals the fused digest");
    }
    /* the same vote on the host arrays themselves (malloc'd, pageable), through
       the device in 8 KiB chunks: the same voted bytes, digests and statistics */
    ft_vote_desc hd = d;
    float *out2 = (float *)malloc(bytes);
    uint32_t *crc2 = (uint32_t *)malloc(4 * nblk);
    ft_stats s2;
    for (int r = 0; r < 3; ++r) hd.replicas[r] = h[r];
    hd.out = out2;
    hd.block_crc = crc2;
    hd.stats = &s2;
    CHECK(ft_vote_host(&hd, 8192) == FT_OK, "ft_vote_host");
    CHECK(memcmp(out2, out, bytes) == 0, "host vote: voted values");
    CHECK(memcmp(crc2, crc, 4 * nblk) == 0, "host vote: digests");
    CHECK(memcmp(&s2, &s, sizeof s) == 0, "host vote: statistics");

    d.R = 1;
    CHECK(ft_vote(&d, NULL) == FT_EINVAL, "R = 1 rejected");
    CHECK(strcmp(ft_strerror(FT_EINVAL), "invalid argument") == 0, "ft_strerror");
    printf("C ABI OK (%llu launches)\n", (unsigned long long)ft_launch_count());
    return 0;
}
