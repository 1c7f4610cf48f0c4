/*
 * ref_vote.c -- plain, slow, scalar CPU oracle for the heterogeneity-aware
 * majority voter and its per-block CRC32C digest.
 *
 * TEST INFRASTRUCTURE. Only the test suite, __graft_entry__.smoke() and the
 * CPU-baseline / reference leg of bench.py load this library. The product path
 * (the CUDA library under paper_1405_2912_b300/ and its Python binding) never
 * links, imports or calls it, and it shares no source with that path.
 *
 * What is computed, and where it comes from (Kicherer & Karl, "Heterogeneity-
 * aware Fault Tolerance using a Self-Organizing Runtime System"):
 *
 *   Sec. IV.D: redundant task results are compared by a majority voter that
 *   determines the presumable correct result.  Integer values compare bit by
 *   bit; floating-point values may differ by a programmer-chosen maximum and
 *   still count as equal, because CPU and GPU kernels order and round their
 *   arithmetic differently.
 *
 *   Readings taken where the paper is silent:
 *     eq(a,b), integers:  bit patterns equal.
 *     eq(a,b), floats, evaluated in the element's own precision with IEEE
 *       round-to-nearest, no fused multiply-add, no flush-to-zero:
 *         (i)   bit patterns equal                       -> equal
 *         (ii)  either value is NaN                      -> not equal
 *         (iii) either value is +-Inf                    -> not equal
 *         (iv)  d = |a - b| (one rounded subtraction),
 *               m = max(|a|, |b|),
 *               equal  iff  d <= abs_tol  or  d <= rel_tol * m
 *               (one rounded multiplication); both tolerances are the
 *               double-typed arguments rounded once to the element type.
 *     support s_r = number of replicas q (q = r included) with eq(x_r, x_q).
 *     winner  w   = the smallest r whose support is the maximum.
 *     voted value y = bit copy of x_w.
 *     majority    iff 2 * s_w > R; otherwise the element is counted in
 *                 no_majority (its value is still x_w).
 *     mismatch[r] = number of elements with not eq(x_r, y); first_mismatch[r]
 *                 is the smallest such index, -1 when there is none.
 *     block CRC   = CRC32C (Castagnoli polynomial 0x1EDC6F41, bit-reflected
 *                 form 0x82F63B78, initial value 0xFFFFFFFF, final XOR
 *                 0xFFFFFFFF) of each 4096-byte block of y's little-endian
 *                 bytes, blocks independent, the last block partial.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

enum { REF_I32 = 0, REF_U32 = 1, REF_I64 = 2, REF_U64 = 3, REF_U8 = 4,
       REF_F32 = 5, REF_F64 = 6 };

#define REF_MAX_R 8
#define REF_BLOCK 4096u

/* ------------------------------------------------------------------------ */
/* CRC32C, byte at a time, from the reflected polynomial                      */
/* ------------------------------------------------------------------------ */

static uint32_t crc_table[256];

/* The byte table: entry b is the register after shifting the 8 bits of b
 * through the reflected division by the polynomial, one bit at a time. */
__attribute__((constructor)) static void ref_make_table(void)
{
    for (uint32_t b = 0; b < 256; ++b) {
        uint32_t c = b;
        for (int k = 0; k < 8; ++k)
            c = (c & 1u) ? (c >> 1) ^ 0x82F63B78u : (c >> 1);
        crc_table[b] = c;
    }
}

/* CRC32C of n bytes, table form. */
uint32_t ref_crc32c(const uint8_t *p, uint64_t n)
{
    uint32_t c = 0xFFFFFFFFu;
    for (uint64_t i = 0; i < n; ++i)
        c = crc_table[(c ^ p[i]) & 0xFFu] ^ (c >> 8);
    return c ^ 0xFFFFFFFFu;
}

/* CRC32C of n bytes, one bit at a time (no table): a second form of the same
 * definition, used by the tests to check the table form. */
uint32_t ref_crc32c_bitwise(const uint8_t *p, uint64_t n)
{
    uint32_t c = 0xFFFFFFFFu;
    for (uint64_t i = 0; i < n; ++i) {
        c ^= p[i];
        for (int k = 0; k < 8; ++k)
            c = (c & 1u) ? (c >> 1) ^ 0x82F63B78u : (c >> 1);
    }
    return c ^ 0xFFFFFFFFu;
}

/* Independent CRC32C of every block_bytes-sized block of nbytes bytes; the
 * last block holds the remainder.  Writes ceil(nbytes / block_bytes) values. */
int ref_block_crc32c(const uint8_t *p, uint64_t nbytes, uint32_t block_bytes,
                     uint32_t *out)
{
    if (block_bytes == 0)
        return -1;
    uint64_t nblocks = (nbytes + block_bytes - 1) / block_bytes;
    for (uint64_t b = 0; b < nblocks; ++b) {
        uint64_t off = b * block_bytes;
        uint64_t len = nbytes - off < block_bytes ? nbytes - off : block_bytes;
        out[b] = ref_crc32c(p + off, len);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Typed comparison (Sec. IV.D)                                               */
/* ------------------------------------------------------------------------ */

static size_t ref_elem_size(int dtype)
{
    switch (dtype) {
    case REF_I32: case REF_U32: case REF_F32: return 4;
    case REF_I64: case REF_U64: case REF_F64: return 8;
    case REF_U8: return 1;
    default: return 0;
    }
}

static int eq_f32(float a, float b, float abs_t, float rel_t)
{
    uint32_t ia, ib;
    memcpy(&ia, &a, 4);
    memcpy(&ib, &b, 4);
    if (ia == ib)
        return 1;                               /* (i)   */
    if (isnan(a) || isnan(b))
        return 0;                               /* (ii)  */
    if (isinf(a) || isinf(b))
        return 0;                               /* (iii) */
    float d = fabsf(a - b);                     /* (iv)  */
    float m = fabsf(a) > fabsf(b) ? fabsf(a) : fabsf(b);
    float t = rel_t * m;
    return d <= abs_t || d <= t;
}

static int eq_f64(double a, double b, double abs_t, double rel_t)
{
    uint64_t ia, ib;
    memcpy(&ia, &a, 8);
    memcpy(&ib, &b, 8);
    if (ia == ib)
        return 1;                               /* (i)   */
    if (isnan(a) || isnan(b))
        return 0;                               /* (ii)  */
    if (isinf(a) || isinf(b))
        return 0;                               /* (iii) */
    double d = fabs(a - b);                     /* (iv)  */
    double m = fabs(a) > fabs(b) ? fabs(a) : fabs(b);
    double t = rel_t * m;
    return d <= abs_t || d <= t;
}

/* eq of two elements given by address. */
static int ref_eq_ptr(int dtype, const uint8_t *a, const uint8_t *b,
                      double abs_tol, double rel_tol)
{
    if (dtype == REF_F32) {
        float x, y;
        memcpy(&x, a, 4);
        memcpy(&y, b, 4);
        return eq_f32(x, y, (float)abs_tol, (float)rel_tol);
    }
    if (dtype == REF_F64) {
        double x, y;
        memcpy(&x, a, 8);
        memcpy(&y, b, 8);
        return eq_f64(x, y, abs_tol, rel_tol);
    }
    return memcmp(a, b, ref_elem_size(dtype)) == 0;
}

/* Exported single comparison, for the tests' tables of special values.
 * Returns 1 / 0, or -1 for an unknown dtype. */
int ref_eq(int dtype, const void *a, const void *b, double abs_tol,
           double rel_tol)
{
    if (ref_elem_size(dtype) == 0)
        return -1;
    return ref_eq_ptr(dtype, (const uint8_t *)a, (const uint8_t *)b, abs_tol,
                      rel_tol);
}

/* ------------------------------------------------------------------------ */
/* The voter                                                                  */
/* ------------------------------------------------------------------------ */

/*
 * Votes n elements of R replica buffers (host memory).  Outputs:
 *   out[n]                 voted values (bit copies of a replica's element)
 *   block_crc[ceil(n*size/4096)]  per-4096-byte-block CRC32C of out, or NULL
 *   mismatch[R], first_mismatch[R], *no_majority, *first_no_majority
 *   tie_flags[n] (or NULL): bit 0 set where another replica with the same,
 *     maximal support would have given a different mismatch pattern; bit 1
 *     set where it would have given different output bits.  These mark the
 *     elements that the lowest-index tie rule decides.
 * Returns 0, or -1 for invalid arguments.
 */
int ref_vote(const void *const *replicas, int R, uint64_t n, int dtype,
             double abs_tol, double rel_tol, void *out, uint32_t *block_crc,
             uint64_t *mismatch, int64_t *first_mismatch,
             uint64_t *no_majority, int64_t *first_no_majority,
             uint8_t *tie_flags)
{
    size_t sz = ref_elem_size(dtype);
    if (sz == 0 || R < 2 || R > REF_MAX_R)
        return -1;
    if (!(abs_tol >= 0.0) || !(rel_tol >= 0.0))   /* rejects NaN too */
        return -1;
    if (n > 0 && (replicas == NULL || out == NULL))
        return -1;

    const uint8_t *x[REF_MAX_R];
    for (int r = 0; r < R; ++r)
        x[r] = (const uint8_t *)replicas[r];
    uint8_t *y = (uint8_t *)out;

    for (int r = 0; r < R; ++r) {
        mismatch[r] = 0;
        first_mismatch[r] = -1;
    }
    *no_majority = 0;
    *first_no_majority = -1;

    for (uint64_t i = 0; i < n; ++i) {
        int e[REF_MAX_R][REF_MAX_R];
        int s[REF_MAX_R];
        for (int r = 0; r < R; ++r)
            for (int q = 0; q < R; ++q)
                e[r][q] = ref_eq_ptr(dtype, x[r] + i * sz, x[q] + i * sz,
                                     abs_tol, rel_tol);
        for (int r = 0; r < R; ++r) {
            s[r] = 0;
            for (int q = 0; q < R; ++q)
                s[r] += e[r][q];
        }
        int w = 0;
        for (int r = 1; r < R; ++r)
            if (s[r] > s[w])
                w = r;
        memcpy(y + i * sz, x[w] + i * sz, sz);

        for (int r = 0; r < R; ++r) {
            if (!e[r][w]) {
                mismatch[r] += 1;
                if (first_mismatch[r] < 0)
                    first_mismatch[r] = (int64_t)i;
            }
        }
        if (!(2 * s[w] > R)) {
            *no_majority += 1;
            if (*first_no_majority < 0)
                *first_no_majority = (int64_t)i;
        }
        if (tie_flags) {
            uint8_t f = 0;
            for (int v = 0; v < R; ++v) {
                if (v == w || s[v] != s[w])
                    continue;
                for (int r = 0; r < R; ++r)
                    if (e[r][v] != e[r][w])
                        f |= 1u;
                if (memcmp(x[v] + i * sz, x[w] + i * sz, sz) != 0)
                    f |= 2u;
            }
            tie_flags[i] = f;
        }
    }
    if (block_crc)
        ref_block_crc32c(y, n * sz, REF_BLOCK, block_crc);
    return 0;
}
