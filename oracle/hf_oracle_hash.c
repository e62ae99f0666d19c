/*
 * hf_oracle_hash.c -- plain CPU oracle of the hash kernels.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this code.  The product path
 * never calls it and shares no code, header, table or constant with it.
 *
 * Sec. 4.1 names three compute-intensive hash functions among the fused
 * kernels (SHA256, Blake256 and Blake2B, taken from a cryptocurrency miner).
 * A miner hashes an 80-byte block header again and again with a different
 * 32-bit nonce in its last four bytes; these scans reproduce that work:
 *
 *   or_sha256d_scan   SHA-256 applied twice (FIPS 180-4, Sec. 5.1.1 padding,
 *                     Sec. 6.2 computation), the Bitcoin proof of work
 *   or_blake256_scan  BLAKE-256 with 14 rounds (Aumasson, Henzen, Meier,
 *                     Phan: "SHA-3 proposal BLAKE")
 *   or_blake2b_scan   BLAKE2b with a 32-byte digest (RFC 7693)
 *
 * Header layout: 80 bytes; bytes 76..79 hold the nonce as a little-endian
 * uint32.  Digests are 32 bytes in each function's own byte order.
 *
 * The round constants and initial values are arguments: the Python side
 * derives them from their definitions (fractional parts of square and cube
 * roots of primes, hexadecimal digits of pi).  The sigma permutations are
 * the one table of the BLAKE family written out by hand; BLAKE2b and BLAKE2s
 * use the same ten rows, so the library pins of those two pin the table.
 *
 * or_blake2s exists only to pin the 32-bit round function that BLAKE-256
 * shares with it (same G, same rotations, same column/diagonal order); the
 * BLAKE-256-specific framing (the constant XOR in G, the counter words, the
 * padding with its final 1 bit) has no published vector in reach and is
 * pinned by reading only.
 */
#include <stdint.h>
#include <string.h>

static uint32_t rotr32(uint32_t x, int n) { return (x >> n) | (x << (32 - n)); }
static uint64_t rotr64(uint64_t x, int n) { return (x >> n) | (x << (64 - n)); }

static uint32_t get_be32(const uint8_t *p)
{
    return ((uint32_t)p[0] << 24) | ((uint32_t)p[1] << 16) | ((uint32_t)p[2] << 8) | p[3];
}
static void put_be32(uint8_t *p, uint32_t v)
{
    p[0] = (uint8_t)(v >> 24);
    p[1] = (uint8_t)(v >> 16);
    p[2] = (uint8_t)(v >> 8);
    p[3] = (uint8_t)v;
}
static uint32_t get_le32(const uint8_t *p)
{
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static void put_le32(uint8_t *p, uint32_t v)
{
    p[0] = (uint8_t)v;
    p[1] = (uint8_t)(v >> 8);
    p[2] = (uint8_t)(v >> 16);
    p[3] = (uint8_t)(v >> 24);
}
static uint64_t get_le64(const uint8_t *p)
{
    return (uint64_t)get_le32(p) | ((uint64_t)get_le32(p + 4) << 32);
}

/* ------------------------------------------------------------------ SHA-256 */
/* One compression (FIPS 180-4 Sec. 6.2.2): message schedule W_0..W_63 from
 * the 16 big-endian words M, 64 rounds on a..h, then H += a..h.            */
void or_sha256_compress(uint32_t H[8], const uint32_t M[16], const uint32_t K[64])
{
    uint32_t W[64];
    for (int t = 0; t < 16; ++t) W[t] = M[t];
    for (int t = 16; t < 64; ++t) {
        uint32_t s0 = rotr32(W[t - 15], 7) ^ rotr32(W[t - 15], 18) ^ (W[t - 15] >> 3);
        uint32_t s1 = rotr32(W[t - 2], 17) ^ rotr32(W[t - 2], 19) ^ (W[t - 2] >> 10);
        W[t] = s1 + W[t - 7] + s0 + W[t - 16];
    }
    uint32_t a = H[0], b = H[1], c = H[2], d = H[3], e = H[4], f = H[5], g = H[6], h = H[7];
    for (int t = 0; t < 64; ++t) {
        uint32_t S1 = rotr32(e, 6) ^ rotr32(e, 11) ^ rotr32(e, 25);
        uint32_t ch = (e & f) ^ (~e & g);
        uint32_t T1 = h + S1 + ch + K[t] + W[t];
        uint32_t S0 = rotr32(a, 2) ^ rotr32(a, 13) ^ rotr32(a, 22);
        uint32_t maj = (a & b) ^ (a & c) ^ (b & c);
        uint32_t T2 = S0 + maj;
        h = g;
        g = f;
        f = e;
        e = d + T1;
        d = c;
        c = b;
        b = a;
        a = T1 + T2;
    }
    H[0] += a;
    H[1] += b;
    H[2] += c;
    H[3] += d;
    H[4] += e;
    H[5] += f;
    H[6] += g;
    H[7] += h;
}

/* Byte b of the padded message of length len (Sec. 5.1.1): the message, one
 * 0x80 byte, zeros, and the 64-bit big-endian bit length in the last eight
 * bytes of the last 64-byte block.  total = padded length in bytes.        */
static uint8_t sha_pad_byte(const uint8_t *msg, uint64_t len, uint64_t total, uint64_t b)
{
    if (b < len) return msg[b];
    if (b == len) return 0x80;
    if (b >= total - 8) {
        const uint64_t bits = len * 8;
        return (uint8_t)(bits >> (8 * (total - 1 - b)));
    }
    return 0;
}

void or_sha256(const uint8_t *msg, uint64_t len, const uint32_t K[64], const uint32_t H0[8],
               uint8_t out[32])
{
    uint32_t H[8];
    memcpy(H, H0, sizeof H);
    const uint64_t total = (len + 9 + 63) / 64 * 64;
    for (uint64_t blk = 0; blk < total; blk += 64) {
        uint8_t B[64];
        uint32_t M[16];
        for (int i = 0; i < 64; ++i) B[i] = sha_pad_byte(msg, len, total, blk + i);
        for (int i = 0; i < 16; ++i) M[i] = get_be32(B + 4 * i);
        or_sha256_compress(H, M, K);
    }
    for (int i = 0; i < 8; ++i) put_be32(out + 4 * i, H[i]);
}

/* digests[i] = SHA-256(SHA-256(header with nonce first + i)). */
void or_sha256d_scan(const uint8_t header[80], uint32_t first, long n, const uint32_t K[64],
                     const uint32_t H0[8], uint8_t *digests)
{
    uint8_t h[80], d1[32];
    memcpy(h, header, 80);
    for (long i = 0; i < n; ++i) {
        put_le32(h + 76, first + (uint32_t)i);
        or_sha256(h, 80, K, H0, d1);
        or_sha256(d1, 32, K, H0, digests + 32 * i);
    }
}

/* ------------------------------------------------- the BLAKE family rounds */
static const uint8_t OR_SIGMA[10][16] = {
    {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15},
    {14, 10, 4, 8, 9, 15, 13, 6, 1, 12, 0, 2, 11, 7, 5, 3},
    {11, 8, 12, 0, 5, 2, 15, 13, 10, 14, 3, 6, 7, 1, 9, 4},
    {7, 9, 3, 1, 13, 12, 11, 14, 2, 6, 5, 10, 4, 0, 15, 8},
    {9, 0, 5, 7, 2, 4, 10, 15, 14, 1, 11, 12, 6, 8, 3, 13},
    {2, 12, 6, 10, 0, 11, 8, 3, 4, 13, 7, 5, 15, 14, 1, 9},
    {12, 5, 1, 15, 14, 13, 4, 10, 0, 7, 6, 3, 9, 2, 8, 11},
    {13, 11, 7, 14, 12, 1, 3, 9, 5, 0, 15, 4, 8, 6, 2, 10},
    {6, 15, 14, 9, 11, 3, 0, 8, 12, 2, 13, 7, 1, 4, 10, 5},
    {10, 2, 8, 4, 7, 6, 1, 5, 15, 11, 9, 14, 3, 12, 13, 0},
};

/* The state words each G of a round touches: four columns, then four
 * diagonals. */
static const int OR_GIDX[8][4] = {{0, 4, 8, 12}, {1, 5, 9, 13}, {2, 6, 10, 14}, {3, 7, 11, 15},
                                  {0, 5, 10, 15}, {1, 6, 11, 12}, {2, 7, 8, 13}, {3, 4, 9, 14}};

/* G of the 32-bit family (BLAKE-256 and BLAKE2s): rotations 16, 12, 8, 7. */
static void or_g32(uint32_t v[16], const int *q, uint32_t x, uint32_t y)
{
    const int a = q[0], b = q[1], c = q[2], d = q[3];
    v[a] = v[a] + v[b] + x;
    v[d] = rotr32(v[d] ^ v[a], 16);
    v[c] = v[c] + v[d];
    v[b] = rotr32(v[b] ^ v[c], 12);
    v[a] = v[a] + v[b] + y;
    v[d] = rotr32(v[d] ^ v[a], 8);
    v[c] = v[c] + v[d];
    v[b] = rotr32(v[b] ^ v[c], 7);
}

/* `rounds` rounds of the 32-bit family.  Round r permutes the message by
 * sigma[r mod 10]; G number i takes words s[2i] and s[2i+1].  BLAKE-256
 * (U != NULL) XORs each with the constant of the other index of the pair;
 * BLAKE2s (U == NULL) uses the words as they are.                          */
static void or_rounds32(uint32_t v[16], const uint32_t m[16], const uint32_t *U, int rounds)
{
    for (int r = 0; r < rounds; ++r) {
        const uint8_t *s = OR_SIGMA[r % 10];
        for (int i = 0; i < 8; ++i) {
            uint32_t x = m[s[2 * i]], y = m[s[2 * i + 1]];
            if (U) {
                x ^= U[s[2 * i + 1]];
                y ^= U[s[2 * i]];
            }
            or_g32(v, OR_GIDX[i], x, y);
        }
    }
}

/* ---------------------------------------------------------------- BLAKE-256 */
/* Compression with salt 0: v = h, U[0..3], t0^U[4], t0^U[5], t1^U[6], t1^U[7];
 * 14 rounds; h'[i] = h[i] ^ v[i] ^ v[i+8].                                 */
void or_blake256_compress(uint32_t h[8], const uint32_t m[16], uint64_t t, const uint32_t U[16])
{
    uint32_t v[16];
    const uint32_t t0 = (uint32_t)t, t1 = (uint32_t)(t >> 32);
    for (int i = 0; i < 8; ++i) v[i] = h[i];
    for (int i = 0; i < 4; ++i) v[8 + i] = U[i];
    v[12] = t0 ^ U[4];
    v[13] = t0 ^ U[5];
    v[14] = t1 ^ U[6];
    v[15] = t1 ^ U[7];
    or_rounds32(v, m, U, 14);
    for (int i = 0; i < 8; ++i) h[i] ^= v[i] ^ v[i + 8];
}

/* BLAKE-256 of len bytes.  Padding: a 1 bit, zeros up to bit 447 of the
 * last block, a 1 bit there, then the 64-bit big-endian bit length; for a
 * byte message that is 0x80 after the message, 0x01 OR-ed into byte 55 of
 * the last block (the two meet as 0x81 when len mod 64 = 55) and the length
 * in bytes 56..63.  The counter of a block is the number of message bits up
 * to its end, or 0 for a block that holds no message bit.  Words are
 * big-endian.                                                              */
void or_blake256(const uint8_t *msg, uint64_t len, const uint32_t IV[8], const uint32_t U[16],
                 uint8_t out[32])
{
    uint32_t h[8];
    memcpy(h, IV, sizeof h);
    const uint64_t total = (len + 9 + 63) / 64 * 64;
    for (uint64_t blk = 0; blk < total; blk += 64) {
        uint8_t B[64];
        uint32_t m[16];
        for (int i = 0; i < 64; ++i) {
            const uint64_t b = blk + i;
            B[i] = b < len ? msg[b] : (b == len ? 0x80 : 0);
        }
        if (blk + 64 == total) {
            B[55] |= 0x01;
            const uint64_t bits = len * 8;
            for (int i = 0; i < 8; ++i) B[56 + i] = (uint8_t)(bits >> (8 * (7 - i)));
        }
        for (int i = 0; i < 16; ++i) m[i] = get_be32(B + 4 * i);
        const uint64_t t = blk < len ? 8 * (len < blk + 64 ? len : blk + 64) : 0;
        or_blake256_compress(h, m, t, U);
    }
    for (int i = 0; i < 8; ++i) put_be32(out + 4 * i, h[i]);
}

void or_blake256_scan(const uint8_t header[80], uint32_t first, long n, const uint32_t IV[8],
                      const uint32_t U[16], uint8_t *digests)
{
    uint8_t h[80];
    memcpy(h, header, 80);
    for (long i = 0; i < n; ++i) {
        put_le32(h + 76, first + (uint32_t)i);
        or_blake256(h, 80, IV, U, digests + 32 * i);
    }
}

/* ------------------------------------------------------------------ BLAKE2s */
/* RFC 7693 unkeyed BLAKE2s with an nn-byte digest (1 <= nn <= 32): used to
 * pin the 32-bit rounds above.                                             */
void or_blake2s(const uint8_t *msg, uint64_t len, int nn, const uint32_t IV[8], uint8_t *out)
{
    uint32_t h[8];
    for (int i = 0; i < 8; ++i) h[i] = IV[i];
    h[0] ^= 0x01010000u ^ (uint32_t)nn;
    const uint64_t nblk = len ? (len + 63) / 64 : 1;
    for (uint64_t k = 0; k < nblk; ++k) {
        uint8_t B[64];
        uint32_t m[16], v[16];
        for (int i = 0; i < 64; ++i) {
            const uint64_t b = 64 * k + i;
            B[i] = b < len ? msg[b] : 0;
        }
        for (int i = 0; i < 16; ++i) m[i] = get_le32(B + 4 * i);
        const int last = k + 1 == nblk;
        const uint64_t t = last ? len : 64 * (k + 1);
        for (int i = 0; i < 8; ++i) {
            v[i] = h[i];
            v[8 + i] = IV[i];
        }
        v[12] ^= (uint32_t)t;
        v[13] ^= (uint32_t)(t >> 32);
        if (last) v[14] = ~v[14];
        or_rounds32(v, m, NULL, 10);
        for (int i = 0; i < 8; ++i) h[i] ^= v[i] ^ v[i + 8];
    }
    uint8_t full[32];
    for (int i = 0; i < 8; ++i) put_le32(full + 4 * i, h[i]);
    memcpy(out, full, (size_t)nn);
}

/* ------------------------------------------------------------------ BLAKE2b */
/* G of the 64-bit family: rotations 32, 24, 16, 63. */
static void or_g64(uint64_t v[16], const int *q, uint64_t x, uint64_t y)
{
    const int a = q[0], b = q[1], c = q[2], d = q[3];
    v[a] = v[a] + v[b] + x;
    v[d] = rotr64(v[d] ^ v[a], 32);
    v[c] = v[c] + v[d];
    v[b] = rotr64(v[b] ^ v[c], 24);
    v[a] = v[a] + v[b] + y;
    v[d] = rotr64(v[d] ^ v[a], 16);
    v[c] = v[c] + v[d];
    v[b] = rotr64(v[b] ^ v[c], 63);
}

/* RFC 7693 Sec. 3.2 compression F with a byte counter t < 2^64. */
void or_blake2b_compress(uint64_t h[8], const uint64_t m[16], uint64_t t, int last,
                         const uint64_t IV[8])
{
    uint64_t v[16];
    for (int i = 0; i < 8; ++i) {
        v[i] = h[i];
        v[8 + i] = IV[i];
    }
    v[12] ^= t;
    if (last) v[14] = ~v[14];
    for (int r = 0; r < 12; ++r) {
        const uint8_t *s = OR_SIGMA[r % 10];
        for (int i = 0; i < 8; ++i) or_g64(v, OR_GIDX[i], m[s[2 * i]], m[s[2 * i + 1]]);
    }
    for (int i = 0; i < 8; ++i) h[i] ^= v[i] ^ v[i + 8];
}

/* Unkeyed BLAKE2b with an nn-byte digest (1 <= nn <= 64), little-endian. */
void or_blake2b(const uint8_t *msg, uint64_t len, int nn, const uint64_t IV[8], uint8_t *out)
{
    uint64_t h[8];
    for (int i = 0; i < 8; ++i) h[i] = IV[i];
    h[0] ^= 0x01010000u ^ (uint64_t)nn;
    const uint64_t nblk = len ? (len + 127) / 128 : 1;
    for (uint64_t k = 0; k < nblk; ++k) {
        uint8_t B[128];
        uint64_t m[16];
        for (int i = 0; i < 128; ++i) {
            const uint64_t b = 128 * k + i;
            B[i] = b < len ? msg[b] : 0;
        }
        for (int i = 0; i < 16; ++i) m[i] = get_le64(B + 8 * i);
        const int last = k + 1 == nblk;
        or_blake2b_compress(h, m, last ? len : 128 * (k + 1), last, IV);
    }
    uint8_t full[64];
    for (int i = 0; i < 8; ++i) {
        put_le32(full + 8 * i, (uint32_t)h[i]);
        put_le32(full + 8 * i + 4, (uint32_t)(h[i] >> 32));
    }
    memcpy(out, full, (size_t)nn);
}

void or_blake2b_scan(const uint8_t header[80], uint32_t first, long n, const uint64_t IV[8],
                     uint8_t *digests)
{
    uint8_t h[80];
    memcpy(h, header, 80);
    for (long i = 0; i < n; ++i) {
        put_le32(h + 76, first + (uint32_t)i);
        or_blake2b(h, 80, 32, IV, digests + 32 * i);
    }
}
