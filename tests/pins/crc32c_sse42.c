/*
 * Independent CRC32C for the oracle's tests: the x86 SSE4.2 CRC32 instruction
 * computes the reflected Castagnoli CRC register update in hardware, so this
 * file shares nothing with the oracle's table or bit loop.  Initial value and
 * final XOR 0xFFFFFFFF as in the CRC32C definition (RFC 3720, Sec. 12.1).
 * Build: gcc -O2 -msse4.2 -fPIC -shared
 */
#include <nmmintrin.h>
#include <stdint.h>

uint32_t hw_crc32c(const uint8_t *p, uint64_t n)
{
    uint32_t c = 0xFFFFFFFFu;
    for (uint64_t i = 0; i < n; ++i)
        c = _mm_crc32_u8(c, p[i]);
    return c ^ 0xFFFFFFFFu;
}
