// body_fp.cuh -- floating-point bodies: the FMA-chain polynomial, bf16
// scale+add, and the parametric stream template used to generate the
// cost-model corpus.
#pragma once
#include "hf_device.cuh"

namespace hf {

// ------------------------------------------------------------------------
// Polynomial chain: acc <- acc * x^33 + p(x), evaluated as one 33-step
// Horner pass per iteration, `iters` iterations.
//
// The work is compute-bound and comes in long, equal units, so its balance
// across SMs decides the tail.  A unit is 64 consecutive elements (two per
// lane, advanced together by one packed FMA chain); warps take units in an
// order that interleaves blocks (warp w of block b has rank w * grid + b),
// so when the units do not divide evenly the extra ones land on every SM
// alike instead of on the first blocks.  A warp runs four units at a time
// (four independent chains per lane) while it has four left, then two,
// then one: in a fused block the polynomial has few warps per scheduler, and
// independent chains are what covers the FMA latency while the other
// bodies' warps take issue slots.
struct BodyPoly {
    using Args = hf_poly_args;
    static constexpr int kId = HF_BODY_POLY;
    static constexpr int kBarriers = 0;
    static constexpr int kUnit = 64;   // elements per warp unit

    static __host__ size_t workspace_bytes(const Args &) { return 0; }
    static __host__ size_t smem_bytes(int, const Args &) { return 0; }
    static __host__ hf_status validate(const Args &a)
    {
        if (a.n < 0 || a.iters < 0) return HF_ERR_INVALID;
        if (a.n > 0 && (!a.x || !a.y)) return HF_ERR_INVALID;
        return HF_OK;
    }

    // One packed FMA (fma.rn.f32x2) performs two independent correctly
    // rounded FMAs, so each packed chain equals two scalar chains bit for
    // bit with half the instructions -- issue slots are what the polynomial
    // shares with the other bodies of a fused block.  NC chains advance
    // together (NC independent packed FMAs per Horner step).
    template <int NC>
    static __device__ __forceinline__ void chains(unsigned long long (&acc)[NC],
                                                  const unsigned long long (&x)[NC],
                                                  const float (&c)[HF_POLY_NCOEF], int iters)
    {
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[j] = f2pack(0.f, 0.f);
#pragma unroll 1
        for (int t = 0; t < iters; ++t) {
#pragma unroll
            for (int k = HF_POLY_NCOEF - 1; k >= 0; --k) {
                const unsigned long long ck = f2pack(c[k], c[k]);
#pragma unroll
                for (int j = 0; j < NC; ++j) acc[j] = f2fma(acc[j], x[j], ck);
            }
        }
    }

    // lane's two elements of unit u (zero past the end; never stored)
    static __device__ __forceinline__ unsigned long long load2(const Args &a, int64_t e)
    {
        const float v0 = e < a.n ? __ldcs(a.x + e) : 0.f;
        const float v1 = e + 1 < a.n ? __ldcs(a.x + e + 1) : 0.f;
        return f2pack(v0, v1);
    }
    static __device__ __forceinline__ void store2(const Args &a, int64_t e, unsigned long long r)
    {
        float v0, v1;
        f2unpack(r, v0, v1);
        if (e < a.n) __stcs(a.y + e, v0);
        if (e + 1 < a.n) __stcs(a.y + e + 1, v1);
    }

    static __device__ void run(const Args &a, const Ctx &cx)
    {
        float c[HF_POLY_NCOEF];
#pragma unroll
        for (int k = 0; k < HF_POLY_NCOEF; ++k) c[k] = a.coef[k];
        const int64_t units = (a.n + kUnit - 1) / kUnit;
        const int64_t nwt = (int64_t)cx.grid * (cx.nthreads >> 5);
        const int64_t lane2 = 2 * lane_id();
        int64_t u = (int64_t)(cx.tid >> 5) * cx.grid + cx.block;
        for (; u + 3 * nwt < units; u += 4 * nwt) {
            int64_t e[4];
            unsigned long long x[4], r[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                e[j] = (u + j * nwt) * kUnit + lane2;
                x[j] = load2(a, e[j]);
            }
            chains<4>(r, x, c, a.iters);
#pragma unroll
            for (int j = 0; j < 4; ++j) store2(a, e[j], r[j]);
        }
        for (; u + nwt < units; u += 2 * nwt) {
            const int64_t e0 = u * kUnit + lane2, e1 = (u + nwt) * kUnit + lane2;
            const unsigned long long x[2] = {load2(a, e0), load2(a, e1)};
            unsigned long long r[2];
            chains<2>(r, x, c, a.iters);
            store2(a, e0, r[0]);
            store2(a, e1, r[1]);
        }
        if (u < units) {
            const int64_t e0 = u * kUnit + lane2;
            const unsigned long long x[1] = {load2(a, e0)};
            unsigned long long r[1];
            chains<1>(r, x, c, a.iters);
            store2(a, e0, r[0]);
        }
    }
};

// ------------------------------------------------------------------------
// bf16 scale+add: out = bf16_rne(alpha * x + y), one FP32 fused multiply-add
// then one rounding to bf16 (ties to even).  Eight elements per 128-bit
// load.
struct BodyBf16Axpy {
    using Args = hf_bf16_axpy_args;
    static constexpr int kId = HF_BODY_BF16_AXPY;
    static constexpr int kBarriers = 0;

    // whole tiles of x and y stream through a bulk-copy ring
    static __host__ bool uses_ring(const Args &a)
    {
        return a.n >= 8 * 32 && aligned16(a.x) && aligned16(a.y) && aligned16(a.out);
    }

    static __host__ size_t workspace_bytes(const Args &) { return 0; }
    static __host__ size_t smem_bytes(int, const Args &) { return 0; }
    static __host__ hf_status validate(const Args &a)
    {
        if (a.n < 0) return HF_ERR_INVALID;
        if (a.n > 0 && (!a.x || !a.y || !a.out)) return HF_ERR_INVALID;
        return HF_OK;
    }

    static __device__ __forceinline__ float lo(unsigned w) { return __uint_as_float(w << 16); }
    static __device__ __forceinline__ float hi(unsigned w) { return __uint_as_float(w & 0xffff0000u); }
    static __device__ __forceinline__ unsigned pack(float u, float v)
    {
        __nv_bfloat162 h = __floats2bfloat162_rn(u, v);   // .x = u (low half)
        return *reinterpret_cast<unsigned *>(&h);
    }
    // the two elements of a 32-bit word in one packed FMA
    static __device__ __forceinline__ unsigned axpy2(float al, unsigned x, unsigned y)
    {
        float r0, r1;
        f2unpack(f2fma(f2pack(al, al), f2pack(lo(x), hi(x)), f2pack(lo(y), hi(y))), r0, r1);
        return pack(r0, r1);
    }

    static __device__ __forceinline__ uint4 axpy8(float al, uint4 x, uint4 y)
    {
        return make_uint4(axpy2(al, x.x, y.x), axpy2(al, x.y, y.y), axpy2(al, x.z, y.z), axpy2(al, x.w, y.w));
    }

    static __device__ void run(const Args &a, const Ctx &cx)
    {
        const float al = a.alpha;
        const int64_t gt = (int64_t)cx.block * cx.nthreads + cx.tid;
        const int64_t stride = (int64_t)cx.grid * cx.nthreads;
        int64_t done = 0;
        if (aligned16(a.x) && aligned16(a.y) && aligned16(a.out)) {
            const int64_t n8 = a.n >> 3;
            int64_t first = 0;   // groups handled by the ring
            // a tile is half a stage of x groups and half of y groups
            const int64_t G = cx.ring_stage / 32;   // groups per tensor per tile
            const int64_t tiles = G ? n8 / G : 0;
            if (tiles > 0 && WarpRing::available(cx, 0)) {
                // whole tiles through the bulk-copy ring, one warp per tile
                WarpRing r;
                r.init(cx, 0);
                const int nw = cx.nthreads >> 5;
                const int64_t gw = (int64_t)cx.block * nw + (cx.tid >> 5), W = (int64_t)cx.grid * nw;
                const unsigned half = r.bytes / 2;
                uint4 *out = reinterpret_cast<uint4 *>(a.out);
                ring_stream(
                    r, gw, W, tiles,
                    [&](int st, int64_t t) {
                        r.expect(st, r.bytes);
                        r.copy(st, 0, a.x + 8 * G * t, half);
                        r.copy(st, half, a.y + 8 * G * t, half);
                    },
                    [&](const unsigned char *p, int64_t t) {
                        const uint4 *px = reinterpret_cast<const uint4 *>(p), *py = px + G;
                        for (int g = r.lane; g < G; g += 32) __stcs(out + G * t + g, axpy8(al, px[g], py[g]));
                    });
                r.finish();
                first = tiles * G;
            }
            int64_t i = first + gt;
            for (; i + stride < n8; i += 2 * stride) {
                const uint4 x0 = ldcs4u(a.x + 8 * i), y0 = ldcs4u(a.y + 8 * i);
                const uint4 x1 = ldcs4u(a.x + 8 * (i + stride)), y1 = ldcs4u(a.y + 8 * (i + stride));
                stcs4u(a.out + 8 * i, make_uint4(axpy2(al, x0.x, y0.x), axpy2(al, x0.y, y0.y),
                                                 axpy2(al, x0.z, y0.z), axpy2(al, x0.w, y0.w)));
                stcs4u(a.out + 8 * (i + stride),
                       make_uint4(axpy2(al, x1.x, y1.x), axpy2(al, x1.y, y1.y),
                                  axpy2(al, x1.z, y1.z), axpy2(al, x1.w, y1.w)));
            }
            if (i < n8) {
                const uint4 x0 = ldcs4u(a.x + 8 * i), y0 = ldcs4u(a.y + 8 * i);
                stcs4u(a.out + 8 * i, make_uint4(axpy2(al, x0.x, y0.x), axpy2(al, x0.y, y0.y),
                                                 axpy2(al, x0.z, y0.z), axpy2(al, x0.w, y0.w)));
            }
            done = n8 << 3;
        }
        for (int64_t i = done + gt; i < a.n; i += stride) {
            const float r = __fmaf_rn(al, __uint_as_float((unsigned)a.x[i] << 16),
                                      __uint_as_float((unsigned)a.y[i] << 16));
            __nv_bfloat16 h = __float2bfloat16_rn(r);
            a.out[i] = *reinterpret_cast<unsigned short *>(&h);
        }
    }
};

// ------------------------------------------------------------------------
// Parametric stream template.  Each loop tile, a thread loads one 16-byte
// group, round-trips it through its own slot of the interval's shared
// buffer, applies k multiply-adds (k/4 rounds over all four components,
// then k%4 more on the leading components) and stores it.  The first
// barrier follows the staging, the others split the FMA rounds evenly.  All
// threads run the same number of tiles so every barrier is uniform.
struct BodyStreamTmpl {
    using Args = hf_stream_tmpl_args;
    static constexpr int kId = HF_BODY_STREAM_TMPL;
    static constexpr int kBarriers = 4;   // at most

    static __host__ size_t workspace_bytes(const Args &) { return 0; }
    static __host__ size_t smem_bytes(int, const Args &a) { return (size_t)a.smem_bytes; }
    static __host__ hf_status validate(const Args &a)
    {
        if (a.n < 0 || (a.n & 3) || a.k < 0 || a.k > 4096) return HF_ERR_INVALID;
        if (a.n_barriers < 0 || a.n_barriers > 4) return HF_ERR_INVALID;
        if (a.smem_bytes < 0 || a.smem_bytes > 49152 || (a.smem_bytes & 15)) return HF_ERR_INVALID;
        if (a.n > 0 && (!a.x || !a.y || !aligned16(a.x) || !aligned16(a.y))) return HF_ERR_INVALID;
        return HF_OK;
    }

    static __device__ __forceinline__ void round4(float4 &v, float m, float b)
    {
        v.x = __fmaf_rn(v.x, m, b);
        v.y = __fmaf_rn(v.y, m, b);
        v.z = __fmaf_rn(v.z, m, b);
        v.w = __fmaf_rn(v.w, m, b);
    }

    static __device__ void run(const Args &a, const Ctx &cx)
    {
        const int64_t n4 = a.n >> 2;
        const int64_t stride = (int64_t)cx.grid * cx.nthreads;
        const int64_t tiles = (n4 + stride - 1) / stride;
        const int nslots = smem_fits(cx, (size_t)a.smem_bytes) ? a.smem_bytes >> 4 : 0;
        const bool staged = cx.tid < nslots;
        const unsigned slot = (unsigned)__cvta_generic_to_shared(cx.smem) + 16u * cx.tid;
        const int k4 = a.k >> 2, kr = a.k & 3, nb = a.n_barriers;
        const float m = a.a, b = a.b;
        for (int64_t t = 0; t < tiles; ++t) {
            const int64_t i = (int64_t)cx.block * cx.nthreads + cx.tid + t * stride;
            const bool ok = i < n4;
            float4 v = ok ? ldcs4(a.x + 4 * i) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (staged)
                asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(slot), "f"(v.x),
                             "f"(v.y), "f"(v.z), "f"(v.w)
                             : "memory");
            if (nb >= 1) interval_sync(cx);
            if (staged)
                asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                             : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                             : "r"(slot)
                             : "memory");
            int done = 0;
            for (int s = 1; s < nb; ++s) {
                const int upto = (int)((int64_t)k4 * s / nb);
#pragma unroll 4
                for (; done < upto; ++done) round4(v, m, b);
                interval_sync(cx);
            }
#pragma unroll 4
            for (; done < k4; ++done) round4(v, m, b);
            if (kr > 0) v.x = __fmaf_rn(v.x, m, b);
            if (kr > 1) v.y = __fmaf_rn(v.y, m, b);
            if (kr > 2) v.z = __fmaf_rn(v.z, m, b);
            if (ok) stcs4(a.y + 4 * i, v);
        }
    }
};

} // namespace hf
