// body_hash.cuh -- the compute-bound hash kernels of Sec. 4.1 (SHA256,
// Blake256, Blake2B) as nonce scans of an 80-byte block header.
//
// Each thread takes items grid-stride; item i hashes the header with the
// nonce (first + i) mod 2^32 in bytes 76..79.  The part of the work that
// does not depend on the nonce -- the compression of the first 64-byte
// block for SHA-256 and BLAKE-256 (the "midstate") -- is done once per
// thread before the loop, as miners do; BLAKE2b's 128-byte block holds the
// whole header, so every item runs one full compression.
//
// All rounds are unrolled at compile time: round constants, message-word
// permutations and the constant padding words are constant expressions, so
// they fold into immediate operands and the message array stays in
// registers.  No shared memory, no barriers: these bodies occupy the
// integer ALU pipes only, which is what makes a pair of them the paper's
// negative case (two kernels that want the same resource, Sec. 4.2).
#pragma once
#include <utility>

#include "hf_device.cuh"

namespace hf {
namespace hash {

__device__ __forceinline__ uint32_t rotr32(uint32_t x, int n) { return __funnelshift_r(x, x, n); }
__device__ __forceinline__ uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0u, 0x0123); }

// 64-bit rotation on the two 32-bit halves (funnel shifts; n = 32 is a swap).
__device__ __forceinline__ uint64_t rotr64(uint64_t x, int n)
{
    const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
    uint32_t nlo, nhi;
    if (n == 32) {
        nlo = hi;
        nhi = lo;
    } else if (n < 32) {
        nlo = __funnelshift_r(lo, hi, n);
        nhi = __funnelshift_r(hi, lo, n);
    } else {
        nlo = __funnelshift_r(hi, lo, n - 32);
        nhi = __funnelshift_r(lo, hi, n - 32);
    }
    return ((uint64_t)nhi << 32) | nlo;
}

// FIPS 180-4 Sec. 4.2.2: the 64 SHA-256 round constants.
__host__ __device__ constexpr uint32_t sha256_k(int t)
{
    constexpr uint32_t k[64] = {
        0x428a2f98u, 0x71374491u, 0xb5c0fbcfu, 0xe9b5dba5u, 0x3956c25bu, 0x59f111f1u, 0x923f82a4u,
        0xab1c5ed5u, 0xd807aa98u, 0x12835b01u, 0x243185beu, 0x550c7dc3u, 0x72be5d74u, 0x80deb1feu,
        0x9bdc06a7u, 0xc19bf174u, 0xe49b69c1u, 0xefbe4786u, 0x0fc19dc6u, 0x240ca1ccu, 0x2de92c6fu,
        0x4a7484aau, 0x5cb0a9dcu, 0x76f988dau, 0x983e5152u, 0xa831c66du, 0xb00327c8u, 0xbf597fc7u,
        0xc6e00bf3u, 0xd5a79147u, 0x06ca6351u, 0x14292967u, 0x27b70a85u, 0x2e1b2138u, 0x4d2c6dfcu,
        0x53380d13u, 0x650a7354u, 0x766a0abbu, 0x81c2c92eu, 0x92722c85u, 0xa2bfe8a1u, 0xa81a664bu,
        0xc24b8b70u, 0xc76c51a3u, 0xd192e819u, 0xd6990624u, 0xf40e3585u, 0x106aa070u, 0x19a4c116u,
        0x1e376c08u, 0x2748774cu, 0x34b0bcb5u, 0x391c0cb3u, 0x4ed8aa4au, 0x5b9cca4fu, 0x682e6ff3u,
        0x748f82eeu, 0x78a5636fu, 0x84c87814u, 0x8cc70208u, 0x90befffau, 0xa4506cebu, 0xbef9a3f7u,
        0xc67178f2u};
    return k[t];
}

// FIPS 180-4 Sec. 5.3.3: SHA-256's initial hash value (also the IV of
// BLAKE-256 and BLAKE2s).
__host__ __device__ constexpr uint32_t sha256_h0(int i)
{
    constexpr uint32_t h[8] = {0x6a09e667u, 0xbb67ae85u, 0x3c6ef372u, 0xa54ff53au,
                               0x510e527fu, 0x9b05688cu, 0x1f83d9abu, 0x5be0cd19u};
    return h[i];
}

// BLAKE-256's sixteen constants: the leading 512 bits of the fractional part
// of pi.
__host__ __device__ constexpr uint32_t blake256_u(int k)
{
    constexpr uint32_t u[16] = {0x243f6a88u, 0x85a308d3u, 0x13198a2eu, 0x03707344u,
                                0xa4093822u, 0x299f31d0u, 0x082efa98u, 0xec4e6c89u,
                                0x452821e6u, 0x38d01377u, 0xbe5466cfu, 0x34e90c6cu,
                                0xc0ac29b7u, 0xc97c50ddu, 0x3f84d5b5u, 0xb5470917u};
    return u[k];
}

// RFC 7693 Sec. 2.6: BLAKE2b's IV (SHA-512's initial hash value).
__host__ __device__ constexpr uint64_t blake2b_iv(int i)
{
    constexpr uint64_t v[8] = {0x6a09e667f3bcc908ull, 0xbb67ae8584caa73bull, 0x3c6ef372fe94f82bull,
                               0xa54ff53a5f1d36f1ull, 0x510e527fade682d1ull, 0x9b05688c2b3e6c1full,
                               0x1f83d9abfb41bd6bull, 0x5be0cd19137e2179ull};
    return v[i];
}

// The ten message permutations of the BLAKE family (BLAKE-256 round r uses
// row r mod 10; RFC 7693 Sec. 2.7 gives the same rows for BLAKE2).
__host__ __device__ constexpr int sigma(int r, int k)
{
    constexpr unsigned char s[10][16] = {
        {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15},
        {14, 10, 4, 8, 9, 15, 13, 6, 1, 12, 0, 2, 11, 7, 5, 3},
        {11, 8, 12, 0, 5, 2, 15, 13, 10, 14, 3, 6, 7, 1, 9, 4},
        {7, 9, 3, 1, 13, 12, 11, 14, 2, 6, 5, 10, 4, 0, 15, 8},
        {9, 0, 5, 7, 2, 4, 10, 15, 14, 1, 11, 12, 6, 8, 3, 13},
        {2, 12, 6, 10, 0, 11, 8, 3, 4, 13, 7, 5, 15, 14, 1, 9},
        {12, 5, 1, 15, 14, 13, 4, 10, 0, 7, 6, 3, 9, 2, 8, 11},
        {13, 11, 7, 14, 12, 1, 3, 9, 5, 0, 15, 4, 8, 6, 2, 10},
        {6, 15, 14, 9, 11, 3, 0, 8, 12, 2, 13, 7, 1, 4, 10, 5},
        {10, 2, 8, 4, 7, 6, 1, 5, 15, 11, 9, 14, 3, 12, 13, 0}};
    return s[r % 10][k];
}

// State words of G number i of a round: columns 0..3, then diagonals 4..7.
__host__ __device__ constexpr int gidx(int i, int j)
{
    return i < 4 ? i + 4 * j : (j == 0 ? i - 4 : 4 * j + (i - 4 + j) % 4);
}

// ------------------------------------------------------------------ SHA-256
// Round T of Sec. 6.2.2 with the eight working variables kept in place:
// variable r (a = 0 .. h = 7) of round T lives in s[(r - T) mod 8], so the
// end-of-round renaming costs nothing.  The schedule word W_T replaces
// W_{T-16} in a 16-word ring.
template <int T>
__device__ __forceinline__ void sha256_round(uint32_t (&s)[8], uint32_t (&w)[16])
{
    if constexpr (T >= 16) {
        const uint32_t x = w[(T - 15) & 15], y = w[(T - 2) & 15];
        const uint32_t s0 = rotr32(x, 7) ^ rotr32(x, 18) ^ (x >> 3);
        const uint32_t s1 = rotr32(y, 17) ^ rotr32(y, 19) ^ (y >> 10);
        w[T & 15] = s1 + w[(T - 7) & 15] + s0 + w[T & 15];
    }
    constexpr uint32_t kt = sha256_k(T);
    uint32_t &a = s[(64 - T) & 7], &b = s[(65 - T) & 7], &c = s[(66 - T) & 7];
    uint32_t &d = s[(67 - T) & 7], &e = s[(68 - T) & 7], &f = s[(69 - T) & 7];
    uint32_t &g = s[(70 - T) & 7], &h = s[(71 - T) & 7];
    const uint32_t S1 = rotr32(e, 6) ^ rotr32(e, 11) ^ rotr32(e, 25);
    const uint32_t ch = (e & f) ^ (~e & g);
    const uint32_t t1 = h + S1 + ch + kt + w[T & 15];
    const uint32_t S0 = rotr32(a, 2) ^ rotr32(a, 13) ^ rotr32(a, 22);
    const uint32_t maj = (a & b) ^ (a & c) ^ (b & c);
    d += t1;
    h = t1 + S0 + maj;
}

template <int... T>
__device__ __forceinline__ void sha256_rounds(uint32_t (&s)[8], uint32_t (&w)[16],
                                              std::integer_sequence<int, T...>)
{
    (sha256_round<T>(s, w), ...);
}

// One compression: st += rounds(st, w).  w is consumed (schedule in place).
__device__ __forceinline__ void sha256_compress(uint32_t (&st)[8], uint32_t (&w)[16])
{
    uint32_t s[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) s[i] = st[i];
    sha256_rounds(s, w, std::make_integer_sequence<int, 64>{});
#pragma unroll
    for (int i = 0; i < 8; ++i) st[i] += s[i];
}

// ------------------------------------------------------------------ BLAKE-256
template <int R, int I>
__device__ __forceinline__ void blake256_g(uint32_t (&v)[16], const uint32_t (&m)[16])
{
    constexpr int a = gidx(I, 0), b = gidx(I, 1), c = gidx(I, 2), d = gidx(I, 3);
    constexpr int x = sigma(R, 2 * I), y = sigma(R, 2 * I + 1);
    constexpr uint32_t ux = blake256_u(x), uy = blake256_u(y);
    v[a] = v[a] + v[b] + (m[x] ^ uy);
    v[d] = rotr32(v[d] ^ v[a], 16);
    v[c] = v[c] + v[d];
    v[b] = rotr32(v[b] ^ v[c], 12);
    v[a] = v[a] + v[b] + (m[y] ^ ux);
    v[d] = rotr32(v[d] ^ v[a], 8);
    v[c] = v[c] + v[d];
    v[b] = rotr32(v[b] ^ v[c], 7);
}

template <int R>
__device__ __forceinline__ void blake256_round(uint32_t (&v)[16], const uint32_t (&m)[16])
{
    blake256_g<R, 0>(v, m);
    blake256_g<R, 1>(v, m);
    blake256_g<R, 2>(v, m);
    blake256_g<R, 3>(v, m);
    blake256_g<R, 4>(v, m);
    blake256_g<R, 5>(v, m);
    blake256_g<R, 6>(v, m);
    blake256_g<R, 7>(v, m);
}

template <int... R>
__device__ __forceinline__ void blake256_rounds(uint32_t (&v)[16], const uint32_t (&m)[16],
                                                std::integer_sequence<int, R...>)
{
    (blake256_round<R>(v, m), ...);
}

// Compression with salt 0 and bit counter (t1:t0): 14 rounds, then
// h ^= v[0..7] ^ v[8..15].
__device__ __forceinline__ void blake256_compress(uint32_t (&h)[8], const uint32_t (&m)[16],
                                                  uint32_t t0, uint32_t t1)
{
    uint32_t v[16];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = h[i];
    v[8] = blake256_u(0);
    v[9] = blake256_u(1);
    v[10] = blake256_u(2);
    v[11] = blake256_u(3);
    v[12] = t0 ^ blake256_u(4);
    v[13] = t0 ^ blake256_u(5);
    v[14] = t1 ^ blake256_u(6);
    v[15] = t1 ^ blake256_u(7);
    blake256_rounds(v, m, std::make_integer_sequence<int, 14>{});
#pragma unroll
    for (int i = 0; i < 8; ++i) h[i] ^= v[i] ^ v[i + 8];
}

// ------------------------------------------------------------------ BLAKE2b
template <int R, int I>
__device__ __forceinline__ void blake2b_g(uint64_t (&v)[16], const uint64_t (&m)[16])
{
    constexpr int a = gidx(I, 0), b = gidx(I, 1), c = gidx(I, 2), d = gidx(I, 3);
    constexpr int x = sigma(R, 2 * I), y = sigma(R, 2 * I + 1);
    v[a] = v[a] + v[b] + m[x];
    v[d] = rotr64(v[d] ^ v[a], 32);
    v[c] = v[c] + v[d];
    v[b] = rotr64(v[b] ^ v[c], 24);
    v[a] = v[a] + v[b] + m[y];
    v[d] = rotr64(v[d] ^ v[a], 16);
    v[c] = v[c] + v[d];
    v[b] = rotr64(v[b] ^ v[c], 63);
}

template <int R>
__device__ __forceinline__ void blake2b_round(uint64_t (&v)[16], const uint64_t (&m)[16])
{
    blake2b_g<R, 0>(v, m);
    blake2b_g<R, 1>(v, m);
    blake2b_g<R, 2>(v, m);
    blake2b_g<R, 3>(v, m);
    blake2b_g<R, 4>(v, m);
    blake2b_g<R, 5>(v, m);
    blake2b_g<R, 6>(v, m);
    blake2b_g<R, 7>(v, m);
}

template <int... R>
__device__ __forceinline__ void blake2b_rounds(uint64_t (&v)[16], const uint64_t (&m)[16],
                                               std::integer_sequence<int, R...>)
{
    (blake2b_round<R>(v, m), ...);
}

// ------------------------------------------------------------------ scan
// Header word k (bytes 4k..4k+3) as the little-endian uint32 it is in memory.
__device__ __forceinline__ uint32_t header_word(const hf_hash_scan_args &a, int k)
{
    return reinterpret_cast<const uint32_t *>(a.header)[k];
}

// Store one digest (8 words, in the order they sit in memory) and apply the
// acceptance test to word 7 (digest bytes 28..31 as a little-endian uint32).
__device__ __forceinline__ void emit(const hf_hash_scan_args &a, int64_t i, uint32_t nonce,
                                     const uint32_t (&d)[8])
{
    if (a.digests) {
        uint4 *o = reinterpret_cast<uint4 *>(a.digests + 32 * i);
        o[0] = make_uint4(d[0], d[1], d[2], d[3]);
        o[1] = make_uint4(d[4], d[5], d[6], d[7]);
    }
    if (d[7] <= a.target && a.hit_count) {
        const uint32_t slot = atomicAdd(a.hit_count, 1u);
        if ((int64_t)slot < (int64_t)a.hit_cap) a.hits[slot] = nonce;
    }
}

__host__ inline hf_status validate_scan(const hf_hash_scan_args &a)
{
    if (a.n < 0 || a.n > ((int64_t)1 << 32)) return HF_ERR_INVALID;
    if (a.digests && !aligned16(a.digests)) return HF_ERR_INVALID;
    if (a.hit_cap < 0) return HF_ERR_INVALID;
    if (a.hit_cap > 0 && (!a.hits || !a.hit_count)) return HF_ERR_INVALID;
    return HF_OK;
}

} // namespace hash

// SHA-256(SHA-256(header)): midstate of block 1 once per thread; per item
// block 2 (header words 16..18, the nonce, then the padding of an 80-byte
// message) and the 32-byte second hash (one padded block).
struct BodySha256d {
    using Args = hf_hash_scan_args;
    static constexpr int kId = HF_BODY_SHA256D;
    static constexpr int kBarriers = 0;

    static __host__ size_t workspace_bytes(const Args &) { return 0; }
    static __host__ size_t smem_bytes(int, const Args &) { return 0; }
    static __host__ hf_status validate(const Args &a) { return hash::validate_scan(a); }

    static __device__ void run(const Args &a, const Ctx &cx)
    {
        using namespace hash;
        uint32_t mid[8];
        {
            uint32_t w[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) w[k] = bswap32(header_word(a, k));
#pragma unroll
            for (int k = 0; k < 8; ++k) mid[k] = sha256_h0(k);
            sha256_compress(mid, w);
        }
        const uint32_t w16 = bswap32(header_word(a, 16)), w17 = bswap32(header_word(a, 17));
        const uint32_t w18 = bswap32(header_word(a, 18));
        const int64_t stride = (int64_t)cx.grid * cx.nthreads;
        for (int64_t i = (int64_t)cx.block * cx.nthreads + cx.tid; i < a.n; i += stride) {
            const uint32_t nonce = a.first + (uint32_t)i;
            uint32_t s1[8], w[16] = {w16, w17, w18, bswap32(nonce), 0x80000000u, 0, 0, 0,
                                     0, 0, 0, 0, 0, 0, 0, 640u};
#pragma unroll
            for (int k = 0; k < 8; ++k) s1[k] = mid[k];
            sha256_compress(s1, w);
            uint32_t s2[8], w2[16] = {s1[0], s1[1], s1[2], s1[3], s1[4], s1[5], s1[6], s1[7],
                                      0x80000000u, 0, 0, 0, 0, 0, 0, 256u};
#pragma unroll
            for (int k = 0; k < 8; ++k) s2[k] = sha256_h0(k);
            sha256_compress(s2, w2);
            uint32_t d[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) d[k] = bswap32(s2[k]);
            emit(a, i, nonce, d);
        }
    }
};

// BLAKE-256 of the 80-byte header: block 1 (counter 512) once per thread;
// per item block 2 = header words 16..18, the nonce, a 1 bit, zeros, the
// final 1 bit and the 64-bit length 640, with counter 640.
struct BodyBlake256 {
    using Args = hf_hash_scan_args;
    static constexpr int kId = HF_BODY_BLAKE256;
    static constexpr int kBarriers = 0;

    static __host__ size_t workspace_bytes(const Args &) { return 0; }
    static __host__ size_t smem_bytes(int, const Args &) { return 0; }
    static __host__ hf_status validate(const Args &a) { return hash::validate_scan(a); }

    static __device__ void run(const Args &a, const Ctx &cx)
    {
        using namespace hash;
        uint32_t mid[8];
        {
            uint32_t m[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) m[k] = bswap32(header_word(a, k));
#pragma unroll
            for (int k = 0; k < 8; ++k) mid[k] = sha256_h0(k);
            blake256_compress(mid, m, 512u, 0u);
        }
        const uint32_t m0 = bswap32(header_word(a, 16)), m1 = bswap32(header_word(a, 17));
        const uint32_t m2 = bswap32(header_word(a, 18));
        const int64_t stride = (int64_t)cx.grid * cx.nthreads;
        for (int64_t i = (int64_t)cx.block * cx.nthreads + cx.tid; i < a.n; i += stride) {
            const uint32_t nonce = a.first + (uint32_t)i;
            const uint32_t m[16] = {m0, m1, m2, bswap32(nonce), 0x80000000u, 0, 0, 0,
                                    0,  0,  0,  0,             0,           1u, 0, 640u};
            uint32_t h[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) h[k] = mid[k];
            blake256_compress(h, m, 640u, 0u);
            uint32_t d[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) d[k] = bswap32(h[k]);
            emit(a, i, nonce, d);
        }
    }
};

// Unkeyed BLAKE2b with a 32-byte digest of the 80-byte header: one final
// block (byte counter 80) per item; message words 10..15 are zero.
struct BodyBlake2b {
    using Args = hf_hash_scan_args;
    static constexpr int kId = HF_BODY_BLAKE2B;
    static constexpr int kBarriers = 0;

    static __host__ size_t workspace_bytes(const Args &) { return 0; }
    static __host__ size_t smem_bytes(int, const Args &) { return 0; }
    static __host__ hf_status validate(const Args &a) { return hash::validate_scan(a); }

    static __device__ void run(const Args &a, const Ctx &cx)
    {
        using namespace hash;
        uint64_t hw[9];
#pragma unroll
        for (int k = 0; k < 9; ++k)
            hw[k] = (uint64_t)header_word(a, 2 * k) | ((uint64_t)header_word(a, 2 * k + 1) << 32);
        const uint32_t w18 = header_word(a, 18);
        // parameter block: digest length 32, no key, fanout 1, depth 1
        const uint64_t h0 = blake2b_iv(0) ^ 0x01010020ull;
        const int64_t stride = (int64_t)cx.grid * cx.nthreads;
        for (int64_t i = (int64_t)cx.block * cx.nthreads + cx.tid; i < a.n; i += stride) {
            const uint32_t nonce = a.first + (uint32_t)i;
            const uint64_t m[16] = {hw[0], hw[1], hw[2], hw[3], hw[4], hw[5], hw[6], hw[7], hw[8],
                                    (uint64_t)w18 | ((uint64_t)nonce << 32), 0, 0, 0, 0, 0, 0};
            uint64_t v[16] = {h0,
                              blake2b_iv(1),
                              blake2b_iv(2),
                              blake2b_iv(3),
                              blake2b_iv(4),
                              blake2b_iv(5),
                              blake2b_iv(6),
                              blake2b_iv(7),
                              blake2b_iv(0),
                              blake2b_iv(1),
                              blake2b_iv(2),
                              blake2b_iv(3),
                              blake2b_iv(4) ^ 80ull,
                              blake2b_iv(5),
                              ~blake2b_iv(6),
                              blake2b_iv(7)};
            blake2b_rounds(v, m, std::make_integer_sequence<int, 12>{});
            const uint64_t d0 = h0 ^ v[0] ^ v[8], d1 = blake2b_iv(1) ^ v[1] ^ v[9];
            const uint64_t d2 = blake2b_iv(2) ^ v[2] ^ v[10], d3 = blake2b_iv(3) ^ v[3] ^ v[11];
            const uint32_t d[8] = {(uint32_t)d0, (uint32_t)(d0 >> 32), (uint32_t)d1,
                                   (uint32_t)(d1 >> 32), (uint32_t)d2, (uint32_t)(d2 >> 32),
                                   (uint32_t)d3, (uint32_t)(d3 >> 32)};
            emit(a, i, nonce, d);
        }
    }
};

} // namespace hf
