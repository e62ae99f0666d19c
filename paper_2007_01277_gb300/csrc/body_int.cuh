// body_int.cuh -- the integer bodies: the 256-bin byte histogram (the
// kernelHistogram1D kernel of Sec. 2.3, shared-memory atomics between two
// block barriers) and the Philox4x32-10 counter-based generator (Salmon,
// Moraes, Dror & Shaw, SC'11).
#pragma once
#include "hf_device.cuh"

namespace hf {

// ------------------------------------------------------------------------
// Histogram.  Each warp of the interval owns a private 256-counter copy in
// shared memory (1 KB), which keeps same-bin conflicts inside one warp.  The
// three phases of Sec. 2.3 are kept: zero the copies, barrier, count every
// byte with a shared atomic, barrier, merge the copies into the global bins
// with one atomic per non-empty bin.  Bytes stream in as 128-bit loads, four
// in flight per thread.
struct BodyHist {
    using Args = hf_hist256_args;
    static constexpr int kId = HF_BODY_HIST256;
    static constexpr int kBarriers = 2;

    // whole tiles of bytes stream through a bulk-copy ring
    static __host__ bool uses_ring(const Args &a) { return a.n >= 512 && aligned16(a.x); }

    static __host__ size_t workspace_bytes(const Args &) { return 0; }
    static __host__ size_t smem_bytes(int nthreads, const Args &)
    {
        return (size_t)(nthreads / 32) * 256 * sizeof(unsigned);
    }
    static __host__ hf_status validate(const Args &a)
    {
        if (a.n < 0) return HF_ERR_INVALID;
        if (a.n > 0 && (!a.x || !a.bins)) return HF_ERR_INVALID;
        return HF_OK;
    }

    static __device__ __forceinline__ void count_word(unsigned *h, unsigned w)
    {
        atomicAdd(h + (w & 0xffu), 1u);
        atomicAdd(h + ((w >> 8) & 0xffu), 1u);
        atomicAdd(h + ((w >> 16) & 0xffu), 1u);
        atomicAdd(h + (w >> 24), 1u);
    }
    static __device__ __forceinline__ void count16(unsigned *h, uint4 v)
    {
        count_word(h, v.x);
        count_word(h, v.y);
        count_word(h, v.z);
        count_word(h, v.w);
    }

    static __device__ void run(const Args &a, const Ctx &cx)
    {
        const int nw = cx.nthreads >> 5;
        if (!smem_fits(cx, (size_t)nw * 256 * sizeof(unsigned))) {
            // no room for the counter copies: count straight into the bins
            for (int64_t i = (int64_t)cx.block * cx.nthreads + cx.tid; i < a.n;
                 i += (int64_t)cx.grid * cx.nthreads)
                atomicAdd(a.bins + a.x[i], 1u);
            return;
        }
        unsigned *sh = reinterpret_cast<unsigned *>(cx.smem);
        for (int i = cx.tid; i < nw * 256; i += cx.nthreads) sh[i] = 0u;
        interval_sync(cx);

        unsigned *mine = sh + (cx.tid >> 5) * 256;
        const int64_t gt = (int64_t)cx.block * cx.nthreads + cx.tid;
        const int64_t stride = (int64_t)cx.grid * cx.nthreads;
        int64_t done = 0;   // bytes handled by the vector loop
        if (aligned16(a.x)) {
            const int64_t n16 = a.n >> 4;
            const uint8_t *x = a.x;
            int64_t first = 0;   // 16-byte groups handled by the ring
            const int64_t B = cx.ring_stage;   // bytes per tile
            const int64_t tiles = B ? a.n / B : 0;
            const size_t counters = (size_t)nw * 256 * sizeof(unsigned);   // a multiple of 128
            if (tiles > 0 && WarpRing::available(cx, counters)) {
                // whole tiles through the bulk-copy ring placed after the
                // counter copies, one warp per tile
                WarpRing r;
                r.init(cx, counters);
                const int64_t gw = (int64_t)cx.block * nw + (cx.tid >> 5), W = (int64_t)cx.grid * nw;
                ring_stream(
                    r, gw, W, tiles,
                    [&](int st, int64_t t) {
                        r.expect(st, r.bytes);
                        r.copy(st, 0, x + B * t, r.bytes);
                    },
                    [&](const unsigned char *p, int64_t) {
                        const uint4 *q = reinterpret_cast<const uint4 *>(p);
                        for (int k = r.lane; k < B / 16; k += 32) count16(mine, q[k]);
                    });
                r.finish();
                first = tiles * (B / 16);
            }
            int64_t i = first + gt;
            for (; i + 3 * stride < n16; i += 4 * stride) {
                uint4 v0 = ldcs4u(x + 16 * i);
                uint4 v1 = ldcs4u(x + 16 * (i + stride));
                uint4 v2 = ldcs4u(x + 16 * (i + 2 * stride));
                uint4 v3 = ldcs4u(x + 16 * (i + 3 * stride));
                count16(mine, v0);
                count16(mine, v1);
                count16(mine, v2);
                count16(mine, v3);
            }
            for (; i < n16; i += stride) count16(mine, ldcs4u(x + 16 * i));
            done = n16 << 4;
        }
        for (int64_t i = done + gt; i < a.n; i += stride) atomicAdd(mine + a.x[i], 1u);
        interval_sync(cx);

        for (int b = cx.tid; b < 256; b += cx.nthreads) {
            unsigned s = 0;
            for (int w = 0; w < nw; ++w) s += sh[w * 256 + b];
            if (s) atomicAdd(a.bins + b, s);
        }
    }
};

// ------------------------------------------------------------------------
// Philox4x32-10.  Output i is the block for counter (lo32(first+i),
// hi32(first+i), 0, 0) under key (lo32(seed), hi32(seed)); each of the ten
// rounds multiplies two counter words by the Philox multipliers, mixes the
// high halves with the other words and the round key, and the key advances
// by the Weyl increments between rounds.  The ten round keys are computed
// once per thread; each multiply is a high-half and a low-half 32-bit
// multiply (cheaper on the integer multiply pipe than one 64-bit product).
// Blocks leave as 128-bit streaming stores.
struct BodyPhilox {
    using Args = hf_philox_args;
    static constexpr int kId = HF_BODY_PHILOX;
    static constexpr int kBarriers = 0;
    static constexpr unsigned kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
    static constexpr unsigned kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;

    static __host__ size_t workspace_bytes(const Args &) { return 0; }
    static __host__ size_t smem_bytes(int, const Args &) { return 0; }
    static __host__ hf_status validate(const Args &a)
    {
        if (a.n < 0) return HF_ERR_INVALID;
        if (a.n > 0 && !a.out) return HF_ERR_INVALID;
        if (a.n > 0 && !aligned16(a.out)) return HF_ERR_INVALID;
        return HF_OK;
    }

    static __device__ __forceinline__ uint4 block(uint64_t ctr, const unsigned (&K0)[10],
                                                 const unsigned (&K1)[10])
    {
        unsigned c0 = (unsigned)ctr, c1 = (unsigned)(ctr >> 32), c2 = 0u, c3 = 0u;
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            const unsigned h0 = __umulhi(kM0, c0), l0 = kM0 * c0;
            const unsigned h1 = __umulhi(kM1, c2), l1 = kM1 * c2;
            c0 = h1 ^ c1 ^ K0[r];
            c2 = h0 ^ c3 ^ K1[r];
            c1 = l1;
            c3 = l0;
        }
        return make_uint4(c0, c1, c2, c3);
    }

    static __device__ void run(const Args &a, const Ctx &cx)
    {
        unsigned K0[10], K1[10];
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            K0[r] = (unsigned)a.seed + (unsigned)r * kW0;
            K1[r] = (unsigned)(a.seed >> 32) + (unsigned)r * kW1;
        }
        const int64_t stride = (int64_t)cx.grid * cx.nthreads;
        uint4 *out = reinterpret_cast<uint4 *>(a.out);
        for (int64_t i = (int64_t)cx.block * cx.nthreads + cx.tid; i < a.n; i += stride)
            __stcs(out + i, block(a.first + (uint64_t)i, K0, K1));
    }
};

} // namespace hf
