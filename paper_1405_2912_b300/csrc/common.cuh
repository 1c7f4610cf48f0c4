// common.cuh -- device building blocks of the voter: typed comparison, the
// R-way vote, per-replica statistics and the fused CRC32C of a 4 KiB block.
//
// Work decomposition (shared by the single-task and the batched kernels): one
// warp owns one 4096-byte block of the voted output at a time.  Lane l loads
// the 16-byte vectors l, l+32, ..., l+224 of the block from every replica
// (coalesced 128-bit loads), votes their elements in registers and stores the
// voted vectors (coalesced 128-bit stores).  It digests the same eight
// vectors in registers: its CRC32C register runs over them in order, and
// folded into the tables of each vector's last step is the jump over the 496
// bytes of other lanes' vectors up to its next one.  The 32 lane registers
// are then moved to their place in the block by a per-lane GF(2)
// multiplication and XOR-reduced across the warp.  Shared memory holds only
// the lookup tables.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ftvote.h"

namespace ftv {

// ---------------------------------------------------------------------------
// CRC32C arithmetic over GF(2), reflected representation.
// A 32-bit register value c stands for the polynomial whose x^(31-j)
// coefficient is bit j of c.  Processing a message M from register 0 yields
// M(x) * x^32 mod P(x); a zero byte multiplies the register by x^8.
// ---------------------------------------------------------------------------
constexpr uint32_t kPoly = 0x82F63B78u;          // reflected Castagnoli polynomial

__host__ __device__ constexpr uint32_t gf_mulx(uint32_t a)
{
    return (a >> 1) ^ ((a & 1u) ? kPoly : 0u);
}

// a(x) * b(x) mod P(x)
__host__ __device__ constexpr uint32_t gf_mul(uint32_t a, uint32_t b)
{
    uint32_t r = 0;
    for (int j = 0; j < 32; ++j) {
        if (b & (0x80000000u >> j)) r ^= a;
        a = gf_mulx(a);
    }
    return r;
}

// x^(8 * nbytes) mod P(x): the operator "append nbytes zero bytes".
__host__ __device__ constexpr uint32_t gf_xpow8(uint64_t nbytes)
{
    uint32_t result = 0x80000000u;   // x^0
    uint32_t base = 0x40000000u;     // x^1
    uint64_t e = nbytes * 8u;
    while (e) {
        if (e & 1u) result = gf_mul(result, base);
        base = gf_mul(base, base);
        e >>= 1;
    }
    return result;
}

struct CrcTables {
    uint32_t slice[4][256];     // slicing-by-4 byte tables
    uint32_t slice_sh[4][256];  // slice[k][b] * x^(8*496): a step, then 496 zero bytes
    uint32_t comb[8][16][32];   // comb[p][v][l] = (v << 4p) * x^(8*16*(31-l))
    uint32_t shift4096[8][16];  // shift4096[p][v] = (v << 4p) * x^(8*4096)
    uint32_t init4096;          // 0xFFFFFFFF * x^(8*4096): initial-value term of a full block
    uint32_t shift_pow[32][8][16];   // shift_pow[j][p][v] = (v << 4p) * x^(8 * 2^j)
    uint32_t shift1552[8][16];       // shift1552[p][v] = (v << 4p) * x^(8*1552): a lane's last four vectors
};

constexpr CrcTables make_crc_tables()
{
    CrcTables t{};
    for (uint32_t b = 0; b < 256; ++b) {
        uint32_t c = b;
        for (int k = 0; k < 8; ++k) c = gf_mulx(c);
        t.slice[0][b] = c;
    }
    for (int k = 1; k < 4; ++k)
        for (uint32_t b = 0; b < 256; ++b) {
            uint32_t prev = t.slice[k - 1][b];
            t.slice[k][b] = (prev >> 8) ^ t.slice[0][prev & 0xFFu];
        }
    {
        const uint32_t M = gf_xpow8(496);
        for (int k = 0; k < 4; ++k)
            for (uint32_t b = 0; b < 256; ++b) t.slice_sh[k][b] = gf_mul(t.slice[k][b], M);
    }
    for (int l = 0; l < 32; ++l) {
        uint32_t K = gf_xpow8(16ull * (31 - l));
        for (int p = 0; p < 8; ++p) {
            uint32_t bit[4] = {};
            for (int q = 0; q < 4; ++q) bit[q] = gf_mul(1u << (4 * p + q), K);
            for (uint32_t v = 0; v < 16; ++v) {
                uint32_t acc = 0;
                for (int q = 0; q < 4; ++q)
                    if (v & (1u << q)) acc ^= bit[q];
                t.comb[p][v][l] = acc;
            }
        }
    }
    {
        uint32_t K = gf_xpow8(4096);
        for (int p = 0; p < 8; ++p)
            for (uint32_t v = 0; v < 16; ++v) t.shift4096[p][v] = gf_mul(v << (4 * p), K);
        t.init4096 = gf_mul(0xFFFFFFFFu, K);
    }
    {
        const uint32_t K = gf_xpow8(16 + 3 * 512);
        for (int p = 0; p < 8; ++p)
            for (uint32_t v = 0; v < 16; ++v) t.shift1552[p][v] = gf_mul(v << (4 * p), K);
    }
    {
        uint32_t K = gf_xpow8(1);                   // x^8, then squared: x^(8 * 2^j)
        for (int j = 0; j < 32; ++j) {
            for (int p = 0; p < 8; ++p)
                for (uint32_t v = 0; v < 16; ++v) t.shift_pow[j][p][v] = gf_mul(v << (4 * p), K);
            K = gf_mul(K, K);
        }
    }
    return t;
}

constexpr CrcTables kCrcHost = make_crc_tables();
// Device copy, initialised at load time from the compile-time tables.
__device__ const CrcTables g_crc = kCrcHost;

constexpr int kBlockBytes = 4096;
constexpr int kCombWords = 8 * 16 * 32;
constexpr int kCrcRowWords = 64;    // one 256-byte row per byte value: 4 tables x 16 copies
constexpr int kCrcWords = 256 * kCrcRowWords;
// Shared-memory table image: slicing tables, shifted slicing tables, combine
// tables, in that order (word offsets).
constexpr int kCrcShOffset = kCrcWords;
constexpr int kCombOffset = 2 * kCrcWords;
constexpr int kTableWords = 2 * kCrcWords + kCombWords;
constexpr uint64_t kNone = ~0ull;   // "no index yet"; reads as -1 through int64

// The shared-memory image of the tables, built at compile time: the slicing
// tables (row e holds T_k[e] for k = 0..3, 16 copies each), the shifted
// slicing tables in the same layout, then the per-lane combine tables.  A CTA
// copies it with 16-byte loads.
struct alignas(16) CrcImage {
    uint32_t w[kTableWords];
};

constexpr CrcImage make_crc_image()
{
    CrcImage im{};
    for (int i = 0; i < kCrcWords; ++i) {
        im.w[i] = kCrcHost.slice[(i >> 4) & 3][i >> 6];
        im.w[kCrcShOffset + i] = kCrcHost.slice_sh[(i >> 4) & 3][i >> 6];
    }
    for (int p = 0; p < 8; ++p)
        for (int v = 0; v < 16; ++v)
            for (int l = 0; l < 32; ++l) im.w[kCombOffset + (p * 16 + v) * 32 + l] = kCrcHost.comb[p][v][l];
    return im;
}

__device__ const CrcImage g_crc_image = make_crc_image();

// Shared memory of a CTA: the table image, nothing else.  Every kernel
// digests from registers, so no data is staged in shared memory, and the
// footprint (144 KiB) leaves the SM's L1 its share for in-flight loads.
constexpr size_t kSmemBytes = sizeof(uint32_t) * kTableWords;

// Copies the table image to s_crc (kTableWords words) with the CTA's W * 32
// threads; the shifted tables and the combine tables then sit at
// s_crc + kCrcShOffset and s_crc + kCombOffset.  Each thread issues all of its
// 16-byte loads before its first store, so the copy costs about one L2 round
// trip (a few loads per round measured ~0.65 us a round on B300, which a
// 16 MiB vote pays in full).
template <int W>
__device__ __forceinline__ void load_crc_tables(uint32_t *s_crc)
{
    constexpr int kVecs = kTableWords / 4;
    constexpr int kThreads = W * 32;
    constexpr int kPer = (kVecs + kThreads - 1) / kThreads;
    const uint4 *src = reinterpret_cast<const uint4 *>(g_crc_image.w);
    uint4 *dst = reinterpret_cast<uint4 *>(s_crc);
    uint4 v[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int i = (int)threadIdx.x + k * kThreads;
        if (i < kVecs) v[k] = src[i];
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int i = (int)threadIdx.x + k * kThreads;
        if (i < kVecs) dst[i] = v[k];
    }
}

// Per-lane constants of the table lookups.  Lane l reads copy l % 16.  In
// lookup i of a slicing step, lanes 0-15 read table T_{3-i} at byte i of the
// register and lanes 16-31 read T_{3-(i^1)} at byte i^1: tables of even index
// sit in banks 0-15 and odd ones in banks 16-31, so the two half-warps never
// share a bank and each lookup is one wavefront.  Each address is built by one
// byte permute: byte 0 = the lane's offset within the row, byte 1 = the data
// byte (the row), bytes 2-3 = 0.
struct CrcLane {
    uint32_t off01, off23;   // offsets for lookups 0,1 (bytes 0,1) and 2,3
    uint32_t sel[4];         // byte-permute selectors
    __device__ __forceinline__ void init(int lane)
    {
        const int h = lane >> 4, c = lane & 15;
        uint32_t o[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int m = h ? (i ^ 1) : i;
            o[i] = (uint32_t)(((3 - m) * 16 + c) * 4);
            sel[i] = 0x6600u | ((uint32_t)m << 4) | (4u + (i & 1));
        }
        off01 = o[0] | (o[1] << 8);
        off23 = o[2] | (o[3] << 8);
    }
};

__device__ __forceinline__ uint32_t lds_at(const uint32_t *base, uint32_t byte_off)
{
    return *reinterpret_cast<const uint32_t *>(reinterpret_cast<const uint8_t *>(base) + byte_off);
}

// One slicing-by-4 step: the register after four more message bytes, given
// c = register XOR (next four bytes, little-endian).
__device__ __forceinline__ uint32_t crc_step4(const uint32_t *s_crc, const CrcLane &L, uint32_t c)
{
    const uint32_t a = lds_at(s_crc, __byte_perm(c, L.off01, L.sel[0]));
    const uint32_t b = lds_at(s_crc, __byte_perm(c, L.off01, L.sel[1]));
    const uint32_t d = lds_at(s_crc, __byte_perm(c, L.off23, L.sel[2]));
    const uint32_t e = lds_at(s_crc, __byte_perm(c, L.off23, L.sel[3]));
    return a ^ b ^ d ^ e;
}

// One byte step with table T_0 (slow paths only).
__device__ __forceinline__ uint32_t crc_step1(const uint32_t *s_crc, uint32_t c, uint32_t byte)
{
    return s_crc[((c ^ byte) & 0xFFu) * kCrcRowWords] ^ (c >> 8);
}

__device__ __forceinline__ uint32_t warp_xor(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v ^= __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// The digest of a full 4 KiB block is taken in the layout of coalesced loads:
// lane l holds the 16-byte vectors l + 32 t, t = 0..7, of the block.  The lane
// runs its register over its vectors in order, one slicing step per word; the
// last step of each vector except the final one uses the shifted tables, which
// also move the register over the 496 bytes up to the lane's next vector.  The
// lane's register then covers bytes [16 l, 16 (l + 225)) with the other lanes'
// vectors as zeros, and the combine step moves it over the 16 (31 - l) bytes
// that follow and XORs the lanes together (the raw register is linear in the
// data).  No vector leaves its lane, so no staging through shared memory.
__device__ __forceinline__ uint32_t crc_vec(const uint32_t *s_crc, const CrcLane &L, uint32_t c, const uint4 &v,
                                            bool last)
{
    c = crc_step4(s_crc, L, c ^ v.x);
    c = crc_step4(s_crc, L, c ^ v.y);
    c = crc_step4(s_crc, L, c ^ v.z);
    return crc_step4(last ? s_crc : s_crc + kCrcShOffset, L, c ^ v.w);
}

// The raw (zero-init) register of the whole block from the lanes' registers.
__device__ __forceinline__ uint32_t crc_combine(const uint32_t *s_crc, uint32_t c, int lane)
{
    const uint32_t *s_comb = s_crc + kCombOffset;
    uint32_t r = 0;
#pragma unroll
    for (int p = 0; p < 8; ++p) r ^= s_comb[(p * 16 + ((c >> (4 * p)) & 15u)) * 32 + lane];
    return warp_xor(r);
}

// c * x^(8k) mod P: the register after k more zero bytes (k < 2^32), one
// nibble-table multiplication by x^(8 * 2^j) per set bit j of k.
__device__ __forceinline__ uint32_t shift_bytes(uint32_t c, uint32_t k)
{
    for (int j = 0; k != 0u; ++j, k >>= 1) {
        if (!(k & 1u)) continue;
        uint32_t r = 0;
#pragma unroll
        for (int p = 0; p < 8; ++p) r ^= g_crc.shift_pow[j][p][(c >> (4 * p)) & 15u];
        c = r;
    }
    return c;
}

// Multiply by x^(8*1552), the span from the start of a lane's fifth vector to
// the end of its eighth (one vector and three jumps of 512 bytes): a lane's
// register over its first four vectors, moved to where the register over its
// last four ends.
__device__ __forceinline__ uint32_t shift_1552(uint32_t c)
{
    uint32_t r = 0;
#pragma unroll
    for (int p = 0; p < 8; ++p) r ^= g_crc.shift1552[p][(c >> (4 * p)) & 15u];
    return r;
}

// Multiply by x^(8*4096) with the shared nibble tables (uniform across the warp).
__device__ __forceinline__ uint32_t shift_4096(uint32_t c)
{
    uint32_t r = 0;
#pragma unroll
    for (int p = 0; p < 8; ++p) r ^= g_crc.shift4096[p][(c >> (4 * p)) & 15u];
    return r;
}

// Programmatic dependent launch (sm_90 and later).  A kernel launched with the
// programmatic-serialization attribute may start once the kernel before it in
// the stream has executed pdl_release(); its pdl_wait() then blocks until that
// kernel has completed and its writes are visible.  Without the attribute
// both are no-ops.
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Streaming 16-byte load of read-only data that bypasses L1 allocation.
__device__ __forceinline__ uint4 ld_stream(const uint4 *p)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Bulk prefetch of `bytes` (a multiple of 16, 16-byte aligned) into L2.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------------------
// Element kinds.  Integer types compare bits, so only their width matters.
// Each kind has a per-call context (its tolerances), a per-replica prepared
// value P and the exact comparison eq(P, P).
// ---------------------------------------------------------------------------
enum Kind { K_F32 = 0, K_F64 = 1, K_B1 = 2, K_B4 = 3, K_B8 = 4 };

template <int K> struct Elem;

// f32.  With rel_tol <= 1 and a finite abs_tol (both checked by the host),
//   eq(a,b) = bits(a) == bits(b)  or  |a-b| <= max(u_a, u_b),
//   u_x = min(max(abs_tol, rel_tol*|x|), FLT_MAX)
// equals the rule "equal bits; else NaN/Inf -> unequal; else |a-b| <= abs_tol
// or |a-b| <= rel_tol*max(|a|,|b|)": rounding is monotone, so
// max(rel*|a|, rel*|b|) = rel*max(|a|,|b|); a NaN or infinite operand makes
// |a-b| NaN or +Inf, which the clamp of u to FLT_MAX rejects; and for finite
// operands the clamp is inactive.
template <> struct Elem<K_F32> {
    using V = uint32_t;
    static constexpr int kSize = 4;
    static constexpr bool kBitsFirst = false;
    struct Ctx { float a, r; };
    struct P { uint32_t bits; float v, u; };
    static __device__ __forceinline__ Ctx ctx(double a, double r) { return {__double2float_rn(a), __double2float_rn(r)}; }
    static __device__ __forceinline__ P prep(V x, Ctx c)
    {
        const float v = __uint_as_float(x);
        return {x, v, fminf(fmaxf(c.a, __fmul_rn(c.r, fabsf(v))), 3.402823466e38f)};
    }
    static __device__ __forceinline__ bool eq(const P &x, const P &y, Ctx)
    {
        return (x.bits == y.bits) | (fabsf(__fsub_rn(x.v, y.v)) <= fmaxf(x.u, y.u));
    }
    static __device__ __forceinline__ V get(const uint4 &v, int e) { return (&v.x)[e]; }
    static __device__ __forceinline__ void set(uint4 &v, int e, V x) { (&v.x)[e] = x; }
};

// f64.  FP64 arithmetic is slow on this part, so the rule is evaluated in FP64
// only for operands whose bits differ.
template <> struct Elem<K_F64> {
    using V = unsigned long long;
    static constexpr int kSize = 8;
    static constexpr bool kBitsFirst = true;
    struct Ctx { double a, r; };
    struct P { V bits; };
    static __device__ __forceinline__ Ctx ctx(double a, double r) { return {a, r}; }
    static __device__ __forceinline__ P prep(V x, Ctx) { return {x}; }
    static __device__ __noinline__ bool eq_slow(V ia, V ib, double ta, double tr)
    {
        const bool fin = ((ia & 0x7FFFFFFFFFFFFFFFull) < 0x7FF0000000000000ull) &
                         ((ib & 0x7FFFFFFFFFFFFFFFull) < 0x7FF0000000000000ull);
        if (!fin) return false;
        const double a = __longlong_as_double((long long)ia), b = __longlong_as_double((long long)ib);
        const double d = fabs(__dsub_rn(a, b));
        const double m = fmax(fabs(a), fabs(b));
        return (d <= ta) | (d <= __dmul_rn(tr, m));
    }
    static __device__ __forceinline__ bool eq(const P &x, const P &y, Ctx c)
    {
        return x.bits == y.bits || eq_slow(x.bits, y.bits, c.a, c.r);
    }
    static __device__ __forceinline__ V get(const uint4 &v, int e)
    {
        return e == 0 ? ((V)v.y << 32 | v.x) : ((V)v.w << 32 | v.z);
    }
    static __device__ __forceinline__ void set(uint4 &v, int e, V x)
    {
        if (e == 0) { v.x = (uint32_t)x; v.y = (uint32_t)(x >> 32); }
        else        { v.z = (uint32_t)x; v.w = (uint32_t)(x >> 32); }
    }
};

template <typename VV, int S, int PER>
struct ElemBits {
    using V = VV;
    static constexpr int kSize = S;
    static constexpr bool kBitsFirst = false;
    struct Ctx {};
    struct P { V bits; };
    static __device__ __forceinline__ Ctx ctx(double, double) { return {}; }
    static __device__ __forceinline__ P prep(V x, Ctx) { return {x}; }
    static __device__ __forceinline__ bool eq(const P &x, const P &y, Ctx) { return x.bits == y.bits; }
};

template <> struct Elem<K_B4> : ElemBits<uint32_t, 4, 4> {
    static __device__ __forceinline__ V get(const uint4 &v, int e) { return (&v.x)[e]; }
    static __device__ __forceinline__ void set(uint4 &v, int e, V x) { (&v.x)[e] = x; }
};

template <> struct Elem<K_B8> : ElemBits<unsigned long long, 8, 2> {
    static __device__ __forceinline__ V get(const uint4 &v, int e) { return Elem<K_F64>::get(v, e); }
    static __device__ __forceinline__ void set(uint4 &v, int e, V x) { Elem<K_F64>::set(v, e, x); }
};

template <> struct Elem<K_B1> : ElemBits<uint32_t, 1, 16> {   // one byte, zero-extended
    static __device__ __forceinline__ V get(const uint4 &v, int e) { return ((&v.x)[e >> 2] >> (8 * (e & 3))) & 0xFFu; }
    static __device__ __forceinline__ void set(uint4 &v, int e, V x)
    {
        uint32_t &w = (&v.x)[e >> 2];
        const int s = 8 * (e & 3);
        w = (w & ~(0xFFu << s)) | (x << s);
    }
};

// ---------------------------------------------------------------------------
// The vote of one element, exact form.  E[r] is the set (bit mask) of
// replicas equal to x_r, self included, so the support is popc(E[r]); the
// first maximum wins.  Returns the winner's bits in y and in m the mismatch
// mask (bit r: x_r is not equal to the winner) with bit R set when there is no
// majority.
// ---------------------------------------------------------------------------
template <int K, int R>
__device__ __forceinline__ void vote_elem(const typename Elem<K>::V (&x)[R], typename Elem<K>::Ctx c,
                                          typename Elem<K>::V &y, uint32_t &m)
{
    using E = Elem<K>;
    typename E::P p[R];
#pragma unroll
    for (int r = 0; r < R; ++r) p[r] = E::prep(x[r], c);
    uint32_t Em[R];
#pragma unroll
    for (int r = 0; r < R; ++r) Em[r] = 1u << r;
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int q = r + 1; q < R; ++q) {
            const bool e = E::eq(p[r], p[q], c);
            Em[r] |= e ? (1u << q) : 0u;
            Em[q] |= e ? (1u << r) : 0u;
        }
    int best = __popc(Em[0]);
    uint32_t Ew = Em[0];
    y = x[0];
#pragma unroll
    for (int r = 1; r < R; ++r) {
        const int s = __popc(Em[r]);
        const bool better = s > best;
        best = better ? s : best;
        Ew = better ? Em[r] : Ew;
        y = better ? x[r] : y;
    }
    m = (~Ew & ((1u << R) - 1u)) | ((2 * best > R) ? 0u : (1u << R));
}

// Per-lane statistics: counts and first indices for the R replicas and, at
// index R, for elements without a majority.
template <int R>
struct LaneStats {
    unsigned long long cnt[R + 1];
    unsigned long long first[R + 1];
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int r = 0; r <= R; ++r) { cnt[r] = 0; first[r] = kNone; }
    }
    __device__ __forceinline__ void add_one(uint32_t m, unsigned long long idx)
    {
#pragma unroll
        for (int r = 0; r <= R; ++r)
            if ((m >> r) & 1u) {
                cnt[r] += 1;
                first[r] = first[r] < idx ? first[r] : idx;
            }
    }
    __device__ __forceinline__ void merge(const LaneStats &o)
    {
#pragma unroll
        for (int r = 0; r <= R; ++r) {
            cnt[r] += o.cnt[r];
            first[r] = o.first[r] < first[r] ? o.first[r] : first[r];
        }
    }
    // Warp-reduce and add into the task's ft_stats (one atomic per non-empty
    // quantity per warp).
    __device__ __forceinline__ void flush(ft_stats *s, int lane)
    {
#pragma unroll
        for (int r = 0; r <= R; ++r) {
            unsigned long long c = cnt[r], f = first[r];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
                const unsigned long long g = __shfl_xor_sync(0xFFFFFFFFu, f, o);
                f = g < f ? g : f;
            }
            if (lane == 0) {
                unsigned long long *pc = r < R ? reinterpret_cast<unsigned long long *>(&s->mismatch[r])
                                               : reinterpret_cast<unsigned long long *>(&s->no_majority);
                unsigned long long *pf = r < R ? reinterpret_cast<unsigned long long *>(&s->first_mismatch[r])
                                               : reinterpret_cast<unsigned long long *>(&s->first_no_majority);
                if (c) atomicAdd(pc, c);
                if (f != kNone) atomicMin(pf, f);
            }
        }
    }
};

// Statistics of one task are reset to (0, -1) before its vote.
__device__ __forceinline__ void reset_stats(ft_stats *s, int i)
{
    if (i < FT_MAX_R) { s->mismatch[i] = 0; s->first_mismatch[i] = -1; }
    if (i == FT_MAX_R) { s->no_majority = 0; s->first_no_majority = -1; }
}

// Arguments of one vote as the kernels see them.
struct TaskArgs {
    const uint8_t *rep[FT_MAX_R];
    uint8_t *out;
    uint32_t *crc;          // may be null
    ft_stats *stats;
    unsigned long long n;   // elements
    unsigned long long nfull;   // full 4 KiB blocks
    uint32_t tail_bytes;    // bytes of the partial last block (0 = none)
    int32_t R;
    int32_t kind;
    int32_t pad_;
    double abs_tol, rel_tol;
};

template <int K>
__device__ __forceinline__ typename Elem<K>::V load_elem(const uint8_t *p)
{
    if constexpr (Elem<K>::kSize == 8) return *reinterpret_cast<const unsigned long long *>(p);
    else if constexpr (Elem<K>::kSize == 4) return *reinterpret_cast<const uint32_t *>(p);
    else return *p;
}

template <int K>
__device__ __forceinline__ void store_elem(uint8_t *p, typename Elem<K>::V v)
{
    if constexpr (Elem<K>::kSize == 8) *reinterpret_cast<unsigned long long *>(p) = v;
    else if constexpr (Elem<K>::kSize == 4) *reinterpret_cast<uint32_t *>(p) = v;
    else *p = (uint8_t)v;
}

// 16-byte vectors per lane that a sub-batch loads from each replica.  (8 for
// R = 2 measured 1-2 % slower than 4 on every kind with 256 MB replicas; 4 for
// R = 5..6 of the kinds with the equal-bits fast path measured the same as 2
// on the 5 x 64M f64 / i32 workloads and spilled.)
template <int K, int R>
constexpr int kSubBatch = (R <= 4) ? 4 : 2;

// Launch shape of the voter kernels for one (kind, R), chosen by measurement
// on B300 (3 x 256M f32; 5 x 64M f64 and i32; 256 MB replicas of every kind
// for R = 2): warps per CTA (one CTA per SM) and whether a warp prefetches its
// next block into L2 while voting the current one.  The f32 R = 3 closed form
// is ALU-heavier per byte and gains from the prefetch with 12 warps (6.7 TB/s
// against 6.2 with 16); every other (kind, R) runs best with 16 warps and no
// prefetch, whose extra L2 footprint costs more than it hides there (f32 R = 2:
// 5.95 against 5.68 TB/s).
//
// kOverlapCrc: a lane digests each sub-batch's voted vectors while the next
// sub-batch's loads are in flight, instead of all eight after the block.
// Measured with 256 MB replicas: i32 R = 5 6.15 -> 6.29 TB/s, f32 R = 2
// 6.04 -> 6.12, f32 R = 5 6.32 -> 6.35; but f32 R = 3, which keeps DRAM busy
// with its L2 prefetch, 6.28 -> 6.05, and i32 R = 3 and u8 R = 5 lose 1-2 %.
template <int K, int R>
struct VotePolicy {
    static constexpr bool kPrefetch = (K == K_F32 && R == 3);
    static constexpr int kWarps = kPrefetch ? 12 : 16;
    static constexpr bool kOverlapCrc = (R == 2) || (R >= 4 && (K == K_F32 || K == K_B4));
};

// Which fast form a (kind, R) takes in the full blocks.
//   F_CLOSED2  R = 2, every kind: replica 0 always wins (equal supports tie
//              to the lower index); replica 1 mismatches, and there is no
//              majority, exactly where the pair is not equal.  One comparison
//              per element; the statistics come from a bit mask.
//   F_CLOSED3  R = 3, f32 and the bit-compared integers: the winner in closed
//              form from the three pairwise comparisons, branch-free; a
//              sub-batch where replica 0 disagrees with another replica is
//              read again for its statistics.
//   F_EQ0      f32, R >= 4: replica 0 equal to every other replica (support R)
//              wins with no mismatch, R - 1 comparisons per element; any
//              other sub-batch is read again and voted in the exact form.
//   F_BITS     integers with R >= 4 and f64 with R >= 3: equal bits in all
//              replicas give replica 0 at once; an element whose bits differ
//              takes the exact form out of line (FP64 arithmetic is slow on
//              this part, so it runs only there).
// ULP-level disagreements are common in float results, which is why the f32
// forms apply the tolerance rule to every element rather than bits first.
enum Form { F_CLOSED2, F_CLOSED3, F_EQ0, F_BITS };
template <int K, int R>
constexpr Form kForm = (R == 2) ? F_CLOSED2
                     : (R == 3 && !Elem<K>::kBitsFirst) ? F_CLOSED3
                     : (K == K_F32 ? F_EQ0 : F_BITS);

// Adds the elements of bit mask q (bit k: element idx0 + (k / P) * 32 * P +
// k % P, P elements per 16-byte vector, a lane's vectors 32 apart) to
// quantity r of the lane statistics.  The index grows with k, so the first
// index is that of the lowest set bit.
template <int P, int R>
__device__ __forceinline__ void add_mask(LaneStats<R> &st, int r, uint64_t q, unsigned long long idx0)
{
    if (!q) return;
    const int k = __ffsll((long long)q) - 1;
    const unsigned long long i = idx0 + (unsigned long long)(k / P) * (32ull * P) + (unsigned long long)(k % P);
    st.cnt[r] += (unsigned long long)__popcll(q);
    st.first[r] = st.first[r] < i ? st.first[r] : i;
}

// The rare paths are kept out of line so that they do not shape the fast
// path's register allocation.
template <int R>
__device__ __noinline__ void record_mask(LaneStats<R> &st, uint32_t m, unsigned long long idx)
{
    st.add_one(m, idx);
}

template <int K, int R>
__device__ __noinline__ void vote_elem_record(typename Elem<K>::V (&x)[R], typename Elem<K>::Ctx c,
                                              typename Elem<K>::V &y, LaneStats<R> &st, unsigned long long idx)
{
    uint32_t m;
    vote_elem<K, R>(x, c, y, m);
    if (m) st.add_one(m, idx);
}

// R = 2: bit k of n01 set where the pair of element k is not equal.
template <int P>
__device__ __noinline__ void closed2_stats(uint64_t n01, unsigned long long idx0, LaneStats<2> &st)
{
    add_mask<P, 2>(st, 1, n01, idx0);
    add_mask<P, 2>(st, 2, n01, idx0);
}

// Statistics of the R = 3 closed form for one sub-batch of a lane, from the
// pairwise comparisons as bit masks: bit k of n01, n02, n12 is set when the
// pair (0,1), (0,2), (1,2) of element k is NOT equal.  Element k is element
// idx0 + (k / P) * 32 * P + k % P of the task (P elements per 16-byte vector,
// a lane's vectors 32 apart), which grows with k, so a quantity's first index
// is that of its lowest set bit.  With e_rq the equalities, the supports are
// 1+e01+e02, 1+e01+e12, 1+e02+e12 and the first maximum wins: replica 1 iff
// e12 and not e02, replica 2 iff e02 and e12 and not e01, else replica 0.
// Replica r mismatches iff it is not equal to the winner; the winner's
// support is 1 (no majority) iff no pair is equal.
template <int P>
__device__ __forceinline__ void closed3_stats(uint64_t n01, uint64_t n02, uint64_t n12, unsigned long long idx0,
                                              LaneStats<3> &st)
{
    const uint64_t w1 = ~n12 & n02;
    const uint64_t w2 = ~n02 & ~n12 & n01;
    const uint64_t w0 = ~(w1 | w2);
    add_mask<P, 3>(st, 0, (w1 & n01) | (w2 & n02), idx0);
    add_mask<P, 3>(st, 1, (w0 & n01) | (w2 & n12), idx0);
    add_mask<P, 3>(st, 2, (w0 & n02) | (w1 & n12), idx0);
    add_mask<P, 3>(st, 3, n01 & n02 & n12, idx0);
}

// Rare path of the R = 3 closed form: the sub-batch (vectors j0 .. j0+JB-1 of
// the lane in the block at byte offset boff) had an element where replica 0
// disagrees with another replica.  The sub-batch is read again from the
// replicas (one round trip, all vectors in flight; the output never overlaps
// a replica) and its pairwise comparisons turned into statistics.
template <int K, int JB>
__device__ __noinline__ void closed3_rare(const TaskArgs &a, unsigned long long boff, int lane, int j0,
                                          unsigned long long idx0, LaneStats<3> &st)
{
    using E = Elem<K>;
    constexpr int P = 16 / E::kSize;
    const typename E::Ctx c = E::ctx(a.abs_tol, a.rel_tol);
    uint4 v[3][JB];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int jj = 0; jj < JB; ++jj)
            v[r][jj] = reinterpret_cast<const uint4 *>(a.rep[r] + boff)[lane + 32 * (j0 + jj)];
    uint64_t n01 = 0, n02 = 0, n12 = 0;
#pragma unroll
    for (int jj = 0; jj < JB; ++jj)
#pragma unroll
        for (int e = 0; e < P; ++e) {
            const uint64_t bit = 1ull << (jj * P + e);
            const typename E::P p0 = E::prep(E::get(v[0][jj], e), c), p1 = E::prep(E::get(v[1][jj], e), c),
                                p2 = E::prep(E::get(v[2][jj], e), c);
            n01 |= E::eq(p0, p1, c) ? 0ull : bit;
            n02 |= E::eq(p0, p2, c) ? 0ull : bit;
            n12 |= E::eq(p1, p2, c) ? 0ull : bit;
        }
    closed3_stats<P>(n01, n02, n12, idx0, st);
}

// Rare path of F_EQ0: in the sub-batch (vectors j0 .. j0+JB-1 of the lane in
// the block at byte offset boff) some element's replica 0 disagrees with
// another replica.  The sub-batch is read again (one round trip; the output
// never overlaps a replica) and voted in the exact form; its voted vectors
// replace the fast form's in the output, from where the lane reads them back.
template <int K, int R, int JB>
__device__ __noinline__ void eq0_rare(const TaskArgs &a, unsigned long long boff, int lane, int j0,
                                      unsigned long long idx0, LaneStats<R> &st)
{
    using E = Elem<K>;
    constexpr int P = 16 / E::kSize;
    const typename E::Ctx c = E::ctx(a.abs_tol, a.rel_tol);
    uint4 v[R][JB];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int jj = 0; jj < JB; ++jj)
            v[r][jj] = reinterpret_cast<const uint4 *>(a.rep[r] + boff)[lane + 32 * (j0 + jj)];
#pragma unroll
    for (int jj = 0; jj < JB; ++jj) {
        uint4 yv;
#pragma unroll
        for (int e = 0; e < P; ++e) {
            typename E::V x[R];
#pragma unroll
            for (int r = 0; r < R; ++r) x[r] = E::get(v[r][jj], e);
            typename E::V y;
            uint32_t m;
            vote_elem<K, R>(x, c, y, m);
            E::set(yv, e, y);
            if (m) st.add_one(m, idx0 + (unsigned long long)(jj * 32 * P + e));
        }
        const int vi = lane + 32 * (j0 + jj);
        reinterpret_cast<uint4 *>(a.out + boff)[vi] = yv;
    }
}

// u8, R = 3: the closed form on four bytes at a time.  __vcmpeq4 gives 0xFF
// in each byte where two words agree; the byte masks then select replica 1
// (e12 and not e02), replica 2 (e02 and e12 and not e01) or replica 0, as in
// the element form.  `flagged` is set when a byte of replica 0 disagrees with
// replica 1 or 2.
__device__ __forceinline__ uint4 vote_b1_closed3(const uint4 &a, const uint4 &b, const uint4 &c, uint64_t &flagged)
{
    uint4 y;
    uint32_t nf = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const uint32_t x0 = (&a.x)[w], x1 = (&b.x)[w], x2 = (&c.x)[w];
        const uint32_t e01 = __vcmpeq4(x0, x1), e02 = __vcmpeq4(x0, x2), e12 = __vcmpeq4(x1, x2);
        const uint32_t s1 = e12 & ~e02, s2 = e02 & e12 & ~e01;
        (&y.x)[w] = (x0 & ~(s1 | s2)) | (x1 & s1) | (x2 & s2);
        nf |= ~(e01 & e02);
    }
    flagged |= nf ? 1ull : 0ull;
    return y;
}

// Fast vote of element k of a lane's sub-batch (element idx of the task):
// the winner's bits in y, or replica 0's where the rare path of the form
// decides.  F_CLOSED2, F_CLOSED3 and F_EQ0 set bit k of `flagged` where the
// element may have a mismatch or lack a majority; F_BITS records a mismatch
// into st at once, out of line.
template <int K, int R>
__device__ __forceinline__ void vote_fast(const typename Elem<K>::V (&x)[R], typename Elem<K>::Ctx c,
                                          typename Elem<K>::V &y, int k, uint64_t &flagged, LaneStats<R> &st,
                                          unsigned long long idx)
{
    using E = Elem<K>;
    constexpr Form F = kForm<K, R>;
    if constexpr (F == F_CLOSED2) {
        y = x[0];
        flagged |= E::eq(E::prep(x[0], c), E::prep(x[1], c), c) ? 0ull : (1ull << k);
    } else if constexpr (F == F_CLOSED3) {
        const typename E::P p0 = E::prep(x[0], c), p1 = E::prep(x[1], c), p2 = E::prep(x[2], c);
        const bool e01 = E::eq(p0, p1, c), e02 = E::eq(p0, p2, c), e12 = E::eq(p1, p2, c);
        const bool w1 = e12 & !e02;
        const bool w2 = e02 & e12 & !e01;
        y = w2 ? x[2] : (w1 ? x[1] : x[0]);
        flagged |= (e01 & e02) ? 0ull : (1ull << k);
    } else if constexpr (F == F_EQ0) {
        const typename E::P p0 = E::prep(x[0], c);
        bool all = true;
#pragma unroll
        for (int r = 1; r < R; ++r) all &= E::eq(p0, E::prep(x[r], c), c);
        y = x[0];
        flagged |= all ? 0ull : (1ull << k);
    } else {
        bool same = true;
#pragma unroll
        for (int r = 1; r < R; ++r) same &= (x[r] == x[0]);
        if (same) {
            y = x[0];
        } else {
            // exactly one replica's bits differ (the usual single fault): the
            // other R - 1 >= 2 agree with replica 0, whose support is then the
            // maximum and a majority whatever that replica compares as, so
            // replica 0 wins and only that replica can mismatch
            uint32_t dm = 0;
            typename E::V xd = x[1];
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const bool d = x[r] != x[0];
                dm |= d ? (1u << r) : 0u;
                xd = d ? x[r] : xd;
            }
            if ((dm & (dm - 1u)) == 0u) {
                y = x[0];
                if (!E::eq(E::prep(x[0], c), E::prep(xd, c), c)) record_mask<R>(st, dm, idx);
            } else {
                typename E::V xc[R];
#pragma unroll
                for (int r = 0; r < R; ++r) xc[r] = x[r];
                vote_elem_record<K, R>(xc, c, y, st, idx);
            }
        }
    }
}

template <int R>
__device__ __forceinline__ const uint8_t *rep_for_lane(const TaskArgs &a, int lane)
{
    const uint8_t *p = a.rep[0];
#pragma unroll
    for (int r = 1; r < R; ++r) p = (lane == r) ? a.rep[r] : p;
    return p;
}

// ---------------------------------------------------------------------------
// One full 4 KiB block of one task, voted and digested by one warp.  Lanes
// 0..R-1 first prefetch the warp's next block (b_next, if any) into L2.  Each
// lane keeps its eight voted vectors in registers and digests them after the
// vote (crc_vec), or, where VotePolicy says so, each sub-batch's under the
// next sub-batch's loads.  Digesting each vector as soon as it is voted
// measured 9 % slower on 3 x 256M f32: the table lookups then sit between the
// vote and the next loads.
// ---------------------------------------------------------------------------
//
// SMALL (the shape of votes of at most one block per warp, where each warp's
// one block is the whole critical path): the lane's CRC runs as two
// independent chains, over vectors 0-3 while the loads of the later vectors
// are in flight and over vectors 4-7 at the end, joined by one multiplication
// (shift_1552); and the R = 3 closed form keeps its pairwise masks in
// registers instead of reading a flagged sub-batch again.
template <int K, int R, int JB = kSubBatch<K, R>, bool SMALL = false>
__device__ __forceinline__ void vote_full_block(const TaskArgs &a, unsigned long long b, unsigned long long b_next,
                                                const uint32_t *s_crc, const CrcLane &L, LaneStats<R> &st, int lane)
{
    using E = Elem<K>;
    using V = typename E::V;
    constexpr int kPerVec = 16 / E::kSize;
    static_assert(JB == 1 || JB == 2 || JB == 4 || JB == 8, "JB: vectors per lane per sub-batch");
    constexpr unsigned long long kEpb = kBlockBytes / E::kSize;
    constexpr Form F = kForm<K, R>;
    static_assert(F == F_BITS || JB * kPerVec <= 64, "`flagged` holds one bit per element of a sub-batch");
    const typename E::Ctx ctx = E::ctx(a.abs_tol, a.rel_tol);
    const unsigned long long boff = b * kBlockBytes;
    if (lane < R && b_next < a.nfull) prefetch_l2(rep_for_lane<R>(a, lane) + b_next * kBlockBytes, kBlockBytes);
    constexpr bool kOverlap = SMALL || VotePolicy<K, R>::kOverlapCrc;
    constexpr bool kInlineStats = SMALL && F == F_CLOSED3 && K != K_B1;
    uint4 yall[8];            // the lane's voted vectors l + 32 t, t = 0..7
    uint32_t cc = 0;          // the lane's CRC register (over vectors 0-3 when SMALL)
    uint32_t cc2 = 0;         // SMALL: the register over vectors 4-7
    auto digest = [&](int t) {
        if (!SMALL || t < 4) cc = crc_vec(s_crc, L, cc, yall[t], t == 7);
        else cc2 = crc_vec(s_crc, L, cc2, yall[t], t == 7);
    };

#pragma unroll
    for (int j0 = 0; j0 < 8; j0 += JB) {
        uint4 v[R][JB];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int jj = 0; jj < JB; ++jj)
                v[r][jj] = ld_stream(reinterpret_cast<const uint4 *>(a.rep[r] + boff) + lane + 32 * (j0 + jj));
        if constexpr (kOverlap) {
            // digest the previous sub-batch while these loads are in flight
            if (j0 > 0) {
#pragma unroll
                for (int jj = 0; jj < JB; ++jj) digest(j0 - JB + jj);
            }
        }
        uint64_t flagged = 0;
        uint64_t n01 = 0, n02 = 0, n12 = 0;   // kInlineStats: bit k set where a pair of element k differs
        const unsigned long long idx0 = b * kEpb + (unsigned long long)(lane + 32 * j0) * kPerVec;
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
            uint4 yv = v[0][jj];
            if constexpr (K == K_B1 && R == 3) {
                yv = vote_b1_closed3(v[0][jj], v[1][jj], v[2][jj], flagged);
            } else if constexpr (kInlineStats) {
#pragma unroll
                for (int e = 0; e < kPerVec; ++e) {
                    const typename E::P p0 = E::prep(E::get(v[0][jj], e), ctx), p1 = E::prep(E::get(v[1][jj], e), ctx),
                                        p2 = E::prep(E::get(v[2][jj], e), ctx);
                    const bool e01 = E::eq(p0, p1, ctx), e02 = E::eq(p0, p2, ctx), e12 = E::eq(p1, p2, ctx);
                    const bool w1 = e12 & !e02;
                    const bool w2 = e02 & e12 & !e01;
                    E::set(yv, e, w2 ? E::get(v[2][jj], e) : (w1 ? E::get(v[1][jj], e) : E::get(v[0][jj], e)));
                    const uint64_t bit = 1ull << (jj * kPerVec + e);
                    n01 |= e01 ? 0ull : bit;
                    n02 |= e02 ? 0ull : bit;
                    n12 |= e12 ? 0ull : bit;
                }
            } else {
                // kinds compared bits first (all but f32): a vector equal in
                // all replicas is replica 0's, with no mismatch
                constexpr bool kPre = (K != K_F32) && F != F_CLOSED3;
                bool differ = !kPre;
                if constexpr (kPre) {
#pragma unroll
                    for (int r = 1; r < R; ++r)
                        differ |= ((v[r][jj].x ^ v[0][jj].x) | (v[r][jj].y ^ v[0][jj].y) |
                                   (v[r][jj].z ^ v[0][jj].z) | (v[r][jj].w ^ v[0][jj].w)) != 0u;
                }
                if (differ) {
#pragma unroll
                    for (int e = 0; e < kPerVec; ++e) {
                        V x[R];
#pragma unroll
                        for (int r = 0; r < R; ++r) x[r] = E::get(v[r][jj], e);
                        V y;
                        vote_fast<K, R>(x, ctx, y, jj * kPerVec + e, flagged, st,
                                        idx0 + (unsigned long long)(jj * 32 * kPerVec + e));
                        E::set(yv, e, y);
                    }
                }
            }
            const int vi = lane + 32 * (j0 + jj);
            __stcs(reinterpret_cast<uint4 *>(a.out + boff) + vi, yv);
            yall[j0 + jj] = yv;
        }
        if constexpr (F == F_CLOSED2)
            if (flagged) closed2_stats<kPerVec>(flagged, idx0, st);
        if constexpr (kInlineStats) {
            if (n01 | n02 | n12) closed3_stats<kPerVec>(n01, n02, n12, idx0, st);
        } else if constexpr (F == F_CLOSED3) {
            if (flagged) closed3_rare<K, JB>(a, boff, lane, j0, idx0, st);
        }
        if constexpr (F == F_EQ0) {
            if (flagged) {
                // re-voted in the exact form and stored; the lane reads its
                // own stores back
                eq0_rare<K, R, JB>(a, boff, lane, j0, idx0, st);
#pragma unroll
                for (int jj = 0; jj < JB; ++jj)
                    yall[j0 + jj] = reinterpret_cast<const uint4 *>(a.out + boff)[lane + 32 * (j0 + jj)];
            }
        }
    }
    if constexpr (kOverlap) {
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) digest(8 - JB + jj);
    } else {
#pragma unroll
        for (int t = 0; t < 8; ++t) digest(t);
    }
    if constexpr (SMALL) cc = shift_1552(cc) ^ cc2;
    const uint32_t raw = crc_combine(s_crc, cc, lane);
    if (lane == 0 && a.crc) a.crc[b] = ~(raw ^ g_crc.init4096);
}

// One element of a partial block into a lane's register, in byte order:
// 4-byte kinds take one slicing step, 8-byte kinds two; bytes are gathered
// four at a time in `w` (n of them so far) and the leftover is flushed by
// crc_flush_bytes.
template <int K>
__device__ __forceinline__ uint32_t crc_elem(const uint32_t *s_crc, const CrcLane &L, uint32_t c,
                                             typename Elem<K>::V y, uint32_t &w, int &n)
{
    if constexpr (Elem<K>::kSize == 8) {
        c = crc_step4(s_crc, L, c ^ (uint32_t)y);
        return crc_step4(s_crc, L, c ^ (uint32_t)(y >> 32));
    } else if constexpr (Elem<K>::kSize == 4) {
        return crc_step4(s_crc, L, c ^ (uint32_t)y);
    } else {
        w |= (uint32_t)y << (8 * n);
        if (++n == 4) {
            c = crc_step4(s_crc, L, c ^ w);
            w = 0;
            n = 0;
        }
        return c;
    }
}

__device__ __forceinline__ uint32_t crc_flush_bytes(const uint32_t *s_crc, uint32_t c, uint32_t w, int n)
{
    for (int k = 0; k < n; ++k) c = crc_step1(s_crc, c, (w >> (8 * k)) & 0xFFu);
    return c;
}

// The partial last block (a.tail_bytes bytes), element by element.  Lane l
// takes the elements of bytes [128 l, 128 l + 128).  The loads of a chunk of
// C elements are issued together before any of its stores: the compiler
// cannot move a load above a store to the output, which may alias for all
// it knows, so one element at a time would pay one memory latency each.
template <int K, int R>
__device__ __noinline__ void vote_tail_block(const TaskArgs &a, unsigned long long b, const uint32_t *s_crc,
                                             const CrcLane &L, LaneStats<R> &st, int lane)
{
    using E = Elem<K>;
    using V = typename E::V;
    constexpr unsigned long long kEpb = kBlockBytes / E::kSize;
    constexpr int C = (R <= 4) ? 8 : 4;
    const typename E::Ctx c = E::ctx(a.abs_tol, a.rel_tol);
    const uint32_t len = a.tail_bytes;
    const unsigned long long boff = b * kBlockBytes;
    const uint32_t e0 = (128u * lane) / E::kSize;
    const uint32_t e1 = min(128u * (lane + 1), len) / E::kSize;
    uint32_t cr = 0, w = 0;   // the lane's CRC register over its bytes, and gathered bytes
    int nw = 0;
    for (uint32_t e = e0; e < e1; e += C) {
        V x[C][R];
#pragma unroll
        for (int j = 0; j < C; ++j)
#pragma unroll
            for (int r = 0; r < R; ++r)
                x[j][r] = (e + j < e1) ? load_elem<K>(a.rep[r] + boff + (unsigned long long)(e + j) * E::kSize)
                                       : V(0);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            if (e + j >= e1) break;
            V y;
            uint32_t m;
            vote_elem<K, R>(x[j], c, y, m);
            store_elem<K>(a.out + boff + (unsigned long long)(e + j) * E::kSize, y);
            cr = crc_elem<K>(s_crc, L, cr, y, w, nw);
            if (m) st.add_one(m, b * kEpb + e + j);
        }
    }
    cr = crc_flush_bytes(s_crc, cr, w, nw);
    // move the lane's register over the bytes after its segment, combine
    const uint32_t start = 128u * lane;
    cr = shift_bytes(cr, len > start + 128u ? len - start - 128u : 0u);
    const uint32_t raw = warp_xor(cr);
    if (lane == 0 && a.crc) a.crc[b] = ~(raw ^ shift_bytes(0xFFFFFFFFu, len));
}

}  // namespace ftv
