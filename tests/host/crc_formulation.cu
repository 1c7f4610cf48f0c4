// Host-side check of the CRC32C formulation the voter and digest kernels use,
// with the kernels' own compile-time tables (common.cuh), so that the tables
// can be pinned on a machine without a GPU.
//
// Reads bytes from stdin and prints one CRC32C per 4096-byte block (the last
// block partial), computed as the kernels do:
//   full block: lane l runs its register over vectors l + 32 t (t = 0..7),
//     one slicing-by-4 step per word, the last step of every vector but the
//     final one through the shifted tables; the lane registers are moved by
//     the per-lane combine tables and XORed;
//   partial block: lane l runs its register over bytes [128 l, 128 l + 128)
//     below the length and is moved over the bytes after them by shift_bytes.
// Then prints "shift ok" or "shift bad" for shift_bytes against the bit-serial
// power on random registers and byte counts.
#include <cstdint>
#include <cstdio>
#include <vector>

#include "common.cuh"

using namespace ftv;

static uint32_t step4(const uint32_t (&T)[4][256], uint32_t c)
{
    return T[3][c & 0xFFu] ^ T[2][(c >> 8) & 0xFFu] ^ T[1][(c >> 16) & 0xFFu] ^ T[0][c >> 24];
}

static uint32_t step1(uint32_t c, uint8_t b) { return kCrcHost.slice[0][(c ^ b) & 0xFFu] ^ (c >> 8); }

static uint32_t host_shift(uint32_t c, uint32_t k)
{
    for (int j = 0; k != 0u; ++j, k >>= 1) {
        if (!(k & 1u)) continue;
        uint32_t r = 0;
        for (int p = 0; p < 8; ++p) r ^= kCrcHost.shift_pow[j][p][(c >> (4 * p)) & 15u];
        c = r;
    }
    return c;
}

static uint32_t full_block(const uint8_t *blk)
{
    uint32_t raw = 0;
    for (int l = 0; l < 32; ++l) {
        uint32_t c = 0;
        for (int t = 0; t < 8; ++t) {
            uint32_t w[4];
            for (int k = 0; k < 4; ++k) {
                const uint8_t *p = blk + 16 * (l + 32 * t) + 4 * k;
                w[k] = (uint32_t)p[0] | (uint32_t)p[1] << 8 | (uint32_t)p[2] << 16 | (uint32_t)p[3] << 24;
            }
            c = step4(kCrcHost.slice, c ^ w[0]);
            c = step4(kCrcHost.slice, c ^ w[1]);
            c = step4(kCrcHost.slice, c ^ w[2]);
            c = step4(t == 7 ? kCrcHost.slice : kCrcHost.slice_sh, c ^ w[3]);
        }
        for (int p = 0; p < 8; ++p) raw ^= kCrcHost.comb[p][(c >> (4 * p)) & 15u][l];
    }
    return ~(raw ^ kCrcHost.init4096);
}

static uint32_t partial_block(const uint8_t *blk, uint32_t len)
{
    uint32_t raw = 0;
    for (uint32_t l = 0; l < 32; ++l) {
        const uint32_t start = 128u * l;
        const uint32_t seg = len > start ? (len - start < 128u ? len - start : 128u) : 0u;
        uint32_t c = 0;
        for (uint32_t k = 0; k < seg; ++k) c = step1(c, blk[start + k]);
        raw ^= host_shift(c, len > start + 128u ? len - start - 128u : 0u);
    }
    return ~(raw ^ host_shift(0xFFFFFFFFu, len));
}

int main()
{
    std::vector<uint8_t> data;
    int ch;
    while ((ch = getchar()) != EOF) data.push_back((uint8_t)ch);
    for (size_t off = 0; off < data.size(); off += 4096) {
        const size_t len = data.size() - off < 4096 ? data.size() - off : 4096;
        printf("%08x\n", len == 4096 ? full_block(&data[off]) : partial_block(&data[off], (uint32_t)len));
    }
    uint64_t s = 0x9E3779B97F4A7C15ull;
    bool ok = true;
    for (int i = 0; i < 2000; ++i) {
        s ^= s << 13; s ^= s >> 7; s ^= s << 17;
        const uint32_t c = (uint32_t)s, k = (uint32_t)(s >> 32) % (i < 1000 ? 4097u : 0xFFFFFFFFu);
        if (host_shift(c, k) != gf_mul(c, gf_xpow8(k))) ok = false;
    }
    printf(ok ? "shift ok\n" : "shift bad\n");
    return 0;
}
