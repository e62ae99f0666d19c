// body_resample.cuh -- the three image-rearranging bodies of Sec. 4.1:
// bilinear x2 upsampling, 3x3/s2/p1 max pooling and 3x3/s1/p1 im2col.
//
// All three are HBM-bound.  The vector paths give each warp a strip of rows
// of one plane: lane l holds input columns 4l..4l+3 of a 128-column band as
// one 128-bit load, the one-column halo comes from the neighbouring lane by
// shuffle, rows slide through registers so each input row is loaded once per
// strip, the next rows are loaded before the current one is used, and
// outputs leave as 128-bit (or 64-bit) streaming stores.  Shapes the vector
// path does not cover use a thread-per-output scalar path with the same
// arithmetic.
#pragma once
#include "hf_device.cuh"

namespace hf {

// (plane, strip) of a warp's ring work items -- items it, it + step, ...
// with it = plane * ns + strip -- advanced without divisions.
struct ItemCursor {
    unsigned p, s;
    __device__ void init(int64_t it, unsigned ns)
    {
        p = (unsigned)(it / ns);
        s = (unsigned)(it - (int64_t)p * ns);
    }
    __device__ void step(unsigned dq, unsigned dr, unsigned ns)   // step = dq * ns + dr
    {
        s += dr;
        p += dq;
        if (s >= ns) s -= ns, ++p;
    }
};

// ------------------------------------------------------------------------
// Bilinear x2, half-pixel centres.  Along one axis of length L, output 2i
// blends input i-1 and i with weights 1/4, 3/4 (output 0 is input 0) and
// output 2i+1 blends i and i+1 with 3/4, 1/4 (output 2L-1 is input L-1).
// Each blend is one fused multiply-add of an exactly scaled quarter, so it
// is correctly rounded; rows are blended horizontally first, then
// vertically, the order of the two-level formula.
struct BodyUpsample {
    using Args = hf_upsample2x_args;
    static constexpr int kId = HF_BODY_UPSAMPLE2X;
    static constexpr int kRows = 8;    // input rows per warp strip
    static constexpr int kBarriers = 0;
    // ring path: a stage holds the 6 input rows of an item and its two halo
    // rows (rows of up to 128 floats)
    static constexpr int kRingRows = 6;
    static constexpr bool kRingItem = true;
    static constexpr unsigned kRingMinBytes = 4096;   // the stage: one item

    // strips of whole rows (W <= 128, 16-byte rows) arrive as one bulk copy
    static __host__ bool uses_ring(const Args &a)
    {
        return (int64_t)a.P * a.H * a.W > 0 && (a.W & 3) == 0 && a.W <= 128 && aligned16(a.x) &&
               aligned16(a.y);
    }

    static __host__ size_t workspace_bytes(const Args &) { return 0; }
    static __host__ size_t smem_bytes(int, const Args &) { return 0; }
    static __host__ hf_status validate(const Args &a)
    {
        if (a.P < 0 || a.H < 0 || a.W < 0) return HF_ERR_INVALID;
        if ((int64_t)a.P * a.H * a.W == 0) return HF_OK;
        if (!a.x || !a.y) return HF_ERR_INVALID;
        if ((int64_t)a.P * a.H * a.W * 4 >= (int64_t)1 << 40) return HF_ERR_INVALID;
        return HF_OK;
    }

    static __device__ __forceinline__ float blend(float near, float far)
    {
        return __fmaf_rn(0.75f, near, __fmul_rn(0.25f, far));
    }

    struct Raw {
        float4 q;
        float left, right;   // halo columns fetched only at band edges
    };

    static __device__ __forceinline__ Raw load_row(const float *row, int c0, int W, bool act)
    {
        Raw r;
        r.q = act ? ldg4(row + c0) : make_float4(0.f, 0.f, 0.f, 0.f);
        const int lane = lane_id();
        r.left = 0.f;
        r.right = 0.f;
        if (act && lane == 0 && c0 > 0) r.left = __ldg(row + c0 - 1);
        if (act && lane == 31 && c0 + 4 < W) r.right = __ldg(row + c0 + 4);
        return r;
    }

    // Horizontal pass of one row: out[0..7] = outputs 2c0 .. 2c0+7.
    static __device__ __forceinline__ void hpass(const Raw &r, int c0, int W, float h[8])
    {
        const int lane = lane_id();
        float L = __shfl_up_sync(0xffffffffu, r.q.w, 1);
        float R = __shfl_down_sync(0xffffffffu, r.q.x, 1);
        if (lane == 0) L = r.left;
        if (lane == 31) R = r.right;
        const float C[4] = {r.q.x, r.q.y, r.q.z, r.q.w};
        const float Lf[4] = {L, r.q.x, r.q.y, r.q.z};
        const float Rt[4] = {r.q.y, r.q.z, r.q.w, R};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int col = c0 + i;
            h[2 * i] = col == 0 ? C[i] : blend(C[i], Lf[i]);
            h[2 * i + 1] = col == W - 1 ? C[i] : blend(C[i], Rt[i]);
        }
    }

    static __device__ void run_vec(const Args &a, const Ctx &cx)
    {
        const int H = a.H, W = a.W, Wo = 2 * W;
        const int nb = (W + 127) / 128;
        const int ns = (H + kRows - 1) / kRows;
        const int64_t items = (int64_t)a.P * ns * nb;
        const int nw = cx.nthreads >> 5;
        const int lane = lane_id();
        for (int64_t it = (int64_t)cx.block * nw + (cx.tid >> 5); it < items;
             it += (int64_t)cx.grid * nw) {
            const int b = (int)(it % nb);
            const int64_t ps = it / nb;
            const int s = (int)(ps % ns);
            const int64_t p = ps / ns;
            const int c0 = b * 128 + 4 * lane;
            const bool act = c0 < W;
            const float *xp = a.x + p * H * W;
            float *yp = a.y + p * (int64_t)(2 * H) * Wo;
            const int r0 = s * kRows;
            const int r1 = min(r0 + kRows, H);
            float hp[8], hc[8], hn[8];
            Raw rn = load_row(xp + (int64_t)min(r0 + 1, H - 1) * W, c0, W, act);
            if (r0 > 0) {
                Raw rp = load_row(xp + (int64_t)(r0 - 1) * W, c0, W, act);
                hpass(rp, c0, W, hp);
            }
            {
                Raw rc = load_row(xp + (int64_t)r0 * W, c0, W, act);
                hpass(rc, c0, W, hc);
            }
#pragma unroll 2
            for (int r = r0; r < r1; ++r) {
                // prefetch row r+2 while row r+1 is blended
                Raw rf = load_row(xp + (int64_t)min(r + 2, H - 1) * W, c0, W, act);
                hpass(rn, c0, W, hn);
                float e[8], o[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    e[i] = r == 0 ? hc[i] : blend(hc[i], hp[i]);
                    o[i] = r == H - 1 ? hc[i] : blend(hc[i], hn[i]);
                }
                if (act) {
                    float *ye = yp + (int64_t)(2 * r) * Wo + 2 * c0;
                    stcs4(ye, make_float4(e[0], e[1], e[2], e[3]));
                    stcs4(ye + 4, make_float4(e[4], e[5], e[6], e[7]));
                    float *yo = ye + Wo;
                    stcs4(yo, make_float4(o[0], o[1], o[2], o[3]));
                    stcs4(yo + 4, make_float4(o[4], o[5], o[6], o[7]));
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) hp[i] = hc[i], hc[i] = hn[i];
                rn = rf;
            }
        }
    }

    // Ring path.  Work item = (plane, strip of R = 6 input rows); the strip
    // and its halo rows, [max(r0-1, 0), min(r0+R+1, H)), are contiguous and
    // arrive in one bulk copy in a stage of the warp's ring while the next
    // items' copies are in flight.  Lane l takes input columns 4l..4l+3 of
    // each row from shared memory (the halo columns from lanes l-1 and l+1
    // by shuffle; a band is the whole row, so lane 0's left and the last
    // lane's right column are outside the image and never blended) and
    // slides the horizontal passes of rows r-1, r, r+1 down the strip; each
    // output is the register path's blend of the same values, so the two
    // paths give the same bits.
    static __device__ bool run_ring(const Args &a, const Ctx &cx)
    {
        constexpr int R = kRingRows;
        const int H = a.H, W = a.W, Wo = 2 * W;
        const unsigned row_bytes = 4u * (unsigned)W;
        if (cx.ring_stage < (R + 2) * row_bytes || (int64_t)a.P * H >= ((int64_t)1 << 32)) return false;
        const unsigned ns = (unsigned)((H + R - 1) / R);
        const int64_t items = (int64_t)a.P * ns;
        WarpRing r;
        r.init(cx, 0);
        const int nw = cx.nthreads >> 5;
        const int64_t gw = (int64_t)cx.block * nw + (cx.tid >> 5), GW = (int64_t)cx.grid * nw;
        const unsigned dq = (unsigned)(GW / ns), dr = (unsigned)(GW % ns);
        const int lane = lane_id();
        const int c0 = 4 * lane;
        const bool act = c0 < W;
        ItemCursor fc, uc;   // the fill cursor runs S items ahead of the use cursor
        fc.init(gw, ns);
        uc = fc;
        ring_stream(
            r, gw, GW, items,
            [&](int st, int64_t) {
                const int r0 = (int)fc.s * R;
                const int ylo = max(r0 - 1, 0), yhi = min(r0 + R + 1, H);
                const unsigned bytes = (unsigned)(yhi - ylo) * row_bytes;   // rows are 16-byte multiples
                r.expect(st, bytes);
                r.copy(st, 0, a.x + ((uint64_t)fc.p * (unsigned)H + (unsigned)ylo) * W, bytes);
                fc.step(dq, dr, ns);
            },
            [&](const unsigned char *stage, int64_t) {
                const int r0 = (int)uc.s * R, r1 = min(r0 + R, H);
                const int ylo = max(r0 - 1, 0), yhi = min(r0 + R + 1, H);
                const unsigned char *base = stage + (act ? 4 * c0 : 0);
                auto hrow = [&](int y, float h[8]) {
                    y = min(max(y, ylo), yhi - 1);   // rows outside are never blended
                    Raw q;
                    q.q = *reinterpret_cast<const float4 *>(base + (unsigned)(y - ylo) * row_bytes);
                    q.left = 0.f;
                    q.right = 0.f;
                    hpass(q, c0, W, h);
                };
                float *yp = a.y + ((int64_t)uc.p * (2 * H) + 2 * r0) * Wo + 2 * c0;
                float hp[8], hc[8], hn[8];
                hrow(r0 - 1, hp);
                hrow(r0, hc);
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const int rr = r0 + i;
                    hrow(rr + 1, hn);
                    if (rr < r1) {
                        float e[8], o[8];
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            e[k] = rr == 0 ? hc[k] : blend(hc[k], hp[k]);
                            o[k] = rr == H - 1 ? hc[k] : blend(hc[k], hn[k]);
                        }
                        if (act) {
                            float *ye = yp + (int64_t)(2 * i) * Wo;
                            stcs4(ye, make_float4(e[0], e[1], e[2], e[3]));
                            stcs4(ye + 4, make_float4(e[4], e[5], e[6], e[7]));
                            stcs4(ye + Wo, make_float4(o[0], o[1], o[2], o[3]));
                            stcs4(ye + Wo + 4, make_float4(o[4], o[5], o[6], o[7]));
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k) hp[k] = hc[k], hc[k] = hn[k];
                }
                uc.step(dq, dr, ns);
            });
        r.finish();
        return true;
    }

    static __device__ void run_scalar(const Args &a, const Ctx &cx)
    {
        const int H = a.H, W = a.W, Ho = 2 * H, Wo = 2 * W;
        const int64_t total = (int64_t)a.P * Ho * Wo;
        for (int64_t i = (int64_t)cx.block * cx.nthreads + cx.tid; i < total;
             i += (int64_t)cx.grid * cx.nthreads) {
            const int ox = (int)(i % Wo);
            const int oy = (int)((i / Wo) % Ho);
            const int64_t p = i / ((int64_t)Wo * Ho);
            const float *xp = a.x + p * H * W;
            auto hrow = [&](int y) {
                const int c = ox >> 1;
                const float C = __ldg(xp + (int64_t)y * W + c);
                if (ox & 1)
                    return c == W - 1 ? C : blend(C, __ldg(xp + (int64_t)y * W + c + 1));
                return c == 0 ? C : blend(C, __ldg(xp + (int64_t)y * W + c - 1));
            };
            const int r = oy >> 1;
            const float hc = hrow(r);
            float v;
            if (oy & 1)
                v = r == H - 1 ? hc : blend(hc, hrow(r + 1));
            else
                v = r == 0 ? hc : blend(hc, hrow(r - 1));
            a.y[i] = v;
        }
    }

    static __device__ void run(const Args &a, const Ctx &cx)
    {
        if ((int64_t)a.P * a.H * a.W == 0) return;
        if ((a.W & 3) == 0 && aligned16(a.x) && aligned16(a.y)) {
            if (a.W <= 128 && WarpRing::available(cx, 0) && run_ring(a, cx)) return;
            run_vec(a, cx);
        } else {
            run_scalar(a, cx);
        }
    }
};

// ------------------------------------------------------------------------
// 3x3 max pooling, stride 2, padding 1 (padding never wins).
struct BodyMaxpool {
    using Args = hf_maxpool3s2_args;
    static constexpr int kId = HF_BODY_MAXPOOL3S2;
    static constexpr int kRows = 8;    // output rows per warp strip
    static constexpr int kBarriers = 0;
    // ring path: a stage must hold the 9 input rows of a strip of 4 output
    // rows (rows of up to 128 floats)
    static constexpr bool kRingItem = true;
    static constexpr unsigned kRingMinBytes = 4096;   // the stage: one item

    // strips of whole rows (W <= 128, 16-byte rows) arrive as one bulk copy
    static __host__ bool uses_ring(const Args &a)
    {
        return (int64_t)a.P * a.H * a.W > 0 && (a.W & 3) == 0 && a.W <= 128 && a.H >= 2 &&
               aligned16(a.x) && aligned16(a.y);
    }

    static __host__ size_t workspace_bytes(const Args &) { return 0; }
    static __host__ size_t smem_bytes(int, const Args &) { return 0; }
    static __host__ hf_status validate(const Args &a)
    {
        if (a.P < 0 || a.H < 0 || a.W < 0) return HF_ERR_INVALID;
        if ((int64_t)a.P * a.H * a.W == 0) return HF_OK;
        if (!a.x || !a.y) return HF_ERR_INVALID;
        if ((int64_t)a.P * a.H * a.W >= (int64_t)1 << 40) return HF_ERR_INVALID;
        return HF_OK;
    }

    static __device__ __forceinline__ float mx(float u, float v) { return v > u ? v : u; }

    struct Raw {
        float4 q;
        float left;
    };
    static __device__ __forceinline__ Raw load_row(const float *row, int c0, bool act, bool valid)
    {
        const float ninf = -__int_as_float(0x7f800000);
        Raw r;
        r.q = (act && valid) ? ldg4(row + c0) : make_float4(ninf, ninf, ninf, ninf);
        r.left = ninf;
        if (act && valid && lane_id() == 0 && c0 > 0) r.left = __ldg(row + c0 - 1);
        return r;
    }
    // Horizontal 3-wide maxima centred on input columns c0 and c0+2.
    static __device__ __forceinline__ float2 hmax(const Raw &r)
    {
        float L = __shfl_up_sync(0xffffffffu, r.q.w, 1);
        if (lane_id() == 0) L = r.left;
        return make_float2(mx(mx(L, r.q.x), r.q.y), mx(mx(r.q.y, r.q.z), r.q.w));
    }

    static __device__ void run_vec(const Args &a, const Ctx &cx)
    {
        const int H = a.H, W = a.W, Ho = (H - 1) / 2 + 1, Wo = (W - 1) / 2 + 1;
        const int nb = (W + 127) / 128;
        const int ns = (Ho + kRows - 1) / kRows;
        const int64_t items = (int64_t)a.P * ns * nb;
        const int nw = cx.nthreads >> 5;
        const int lane = lane_id();
        for (int64_t it = (int64_t)cx.block * nw + (cx.tid >> 5); it < items;
             it += (int64_t)cx.grid * nw) {
            const int b = (int)(it % nb);
            const int64_t ps = it / nb;
            const int s = (int)(ps % ns);
            const int64_t p = ps / ns;
            const int c0 = b * 128 + 4 * lane;
            const bool act = c0 < W;
            const float *xp = a.x + p * H * W;
            float *yp = a.y + p * (int64_t)Ho * Wo;
            const int o0 = s * kRows, o1 = min(o0 + kRows, Ho);
            // carried: horizontal maxima of input row 2*oy - 1
            float2 top = hmax(load_row(xp + (int64_t)(2 * o0 - 1) * W, c0, act, o0 > 0));
            Raw ra = load_row(xp + (int64_t)(2 * o0) * W, c0, act, 2 * o0 < H);
            Raw rb = load_row(xp + (int64_t)(2 * o0 + 1) * W, c0, act, 2 * o0 + 1 < H);
#pragma unroll 2
            for (int oy = o0; oy < o1; ++oy) {
                const int n0 = 2 * oy + 2, n1 = 2 * oy + 3;
                Raw na = load_row(xp + (int64_t)n0 * W, c0, act, oy + 1 < o1 && n0 < H);
                Raw nbr = load_row(xp + (int64_t)n1 * W, c0, act, oy + 1 < o1 && n1 < H);
                const float2 m0 = hmax(ra), m1 = hmax(rb);
                const float2 v = make_float2(mx(mx(top.x, m0.x), m1.x), mx(mx(top.y, m0.y), m1.y));
                if (act) stcs2(yp + (int64_t)oy * Wo + (c0 >> 1), v);
                top = m1;
                ra = na;
                rb = nbr;
            }
        }
    }

    // Ring path.  Work item = (plane, strip of R = 4 output rows); its
    // input rows [max(2*o0-1, 0), min(2*o1, H)) are contiguous and arrive
    // in one bulk copy in a stage of the warp's ring, the next items' copies
    // in flight meanwhile.  Lane l takes input columns 4l..4l+3 (output
    // columns 2l, 2l+1) of each of the strip's nine rows from shared memory
    // (nine independent loads); the left halo column comes from lane l-1 by
    // shuffle.  No loads are held in registers, so bytes in flight do not
    // depend on registers or warps.
    static constexpr int kRingRows = 4;   // output rows per ring work item

    static __device__ bool run_ring(const Args &a, const Ctx &cx)
    {
        constexpr int R = kRingRows, NR = 2 * R + 1;
        const int H = a.H, W = a.W, Ho = (H - 1) / 2 + 1, Wo = (W - 1) / 2 + 1;
        const unsigned row_bytes = 4u * (unsigned)W;
        if (cx.ring_stage < NR * row_bytes || (int64_t)a.P * H >= ((int64_t)1 << 32)) return false;
        const unsigned ns = (unsigned)((Ho + R - 1) / R);
        const int64_t items = (int64_t)a.P * ns;
        WarpRing r;
        r.init(cx, 0);
        const int nw = cx.nthreads >> 5;
        const int64_t gw = (int64_t)cx.block * nw + (cx.tid >> 5), GW = (int64_t)cx.grid * nw;
        const unsigned dq = (unsigned)(GW / ns), dr = (unsigned)(GW % ns);
        const int lane = lane_id();
        const int c0 = 4 * lane;
        const bool act = c0 < W;
        const float ninf = -__int_as_float(0x7f800000);
        ItemCursor fc, uc;   // the fill cursor runs S items ahead of the use cursor
        fc.init(gw, ns);
        uc = fc;
        ring_stream(
            r, gw, GW, items,
            [&](int st, int64_t) {
                const int o0 = (int)fc.s * R, o1 = min(o0 + R, Ho);
                const int ylo = max(2 * o0 - 1, 0), yhi = min(2 * o1, H);
                const unsigned first_row = fc.p * (unsigned)H + (unsigned)ylo;
                const unsigned bytes = (unsigned)(yhi - ylo) * row_bytes;   // rows are 16-byte multiples
                r.expect(st, bytes);
                r.copy(st, 0, a.x + (uint64_t)first_row * W, bytes);
                fc.step(dq, dr, ns);
            },
            [&](const unsigned char *stage, int64_t) {
                const int o0 = (int)uc.s * R, o1 = min(o0 + R, Ho);
                const int ylo = max(2 * o0 - 1, 0), yhi = min(2 * o1, H);
                // rows 2*o0-1 .. 2*o0+2R-1 at clamped (in-stage) offsets,
                // lanes past W reading column 0; row 2*o0-1 is padding in
                // the first strip and rows at or past H (odd H) in the last
                const unsigned char *base = stage + (act ? 4 * c0 : 0);
                float2 h[NR];
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    const int y = min(max(2 * o0 - 1 + k, ylo), yhi - 1);
                    const float4 q = *reinterpret_cast<const float4 *>(base + (unsigned)(y - ylo) * row_bytes);
                    float L = __shfl_up_sync(0xffffffffu, q.w, 1);
                    if (lane == 0) L = ninf;
                    h[k] = make_float2(mx(mx(L, q.x), q.y), mx(mx(q.y, q.z), q.w));
                }
                if (o0 == 0) h[0] = make_float2(ninf, ninf);
#pragma unroll
                for (int k = 1; k < NR; ++k)
                    if (2 * o0 - 1 + k >= yhi) h[k] = make_float2(ninf, ninf);
                float *yp = a.y + ((int64_t)uc.p * Ho + o0) * Wo + (c0 >> 1);
#pragma unroll
                for (int j = 0; j < R; ++j)
                    if (act && o0 + j < o1)
                        stcs2(yp + j * Wo, make_float2(mx(mx(h[2 * j].x, h[2 * j + 1].x), h[2 * j + 2].x),
                                                       mx(mx(h[2 * j].y, h[2 * j + 1].y), h[2 * j + 2].y)));
                uc.step(dq, dr, ns);
            });
        r.finish();
        return true;
    }

    static __device__ void run_scalar(const Args &a, const Ctx &cx)
    {
        const int H = a.H, W = a.W, Ho = (H - 1) / 2 + 1, Wo = (W - 1) / 2 + 1;
        const int64_t total = (int64_t)a.P * Ho * Wo;
        const float ninf = -__int_as_float(0x7f800000);
        for (int64_t i = (int64_t)cx.block * cx.nthreads + cx.tid; i < total;
             i += (int64_t)cx.grid * cx.nthreads) {
            const int ox = (int)(i % Wo);
            const int oy = (int)((i / Wo) % Ho);
            const int64_t p = i / ((int64_t)Wo * Ho);
            const float *xp = a.x + p * H * W;
            float m = ninf;
            for (int ky = 0; ky < 3; ++ky) {
                const int iy = 2 * oy - 1 + ky;
                if (iy < 0 || iy >= H) continue;
                for (int kx = 0; kx < 3; ++kx) {
                    const int ix = 2 * ox - 1 + kx;
                    if (ix < 0 || ix >= W) continue;
                    m = mx(m, __ldg(xp + (int64_t)iy * W + ix));
                }
            }
            a.y[i] = m;
        }
    }

    static __device__ void run(const Args &a, const Ctx &cx)
    {
        if ((int64_t)a.P * a.H * a.W == 0) return;
        if ((a.W & 3) == 0 && aligned16(a.x) && aligned16(a.y)) {
            if (a.W <= 128 && a.H >= 2 && WarpRing::available(cx, 0) && run_ring(a, cx)) return;
            run_vec(a, cx);
        } else {
            run_scalar(a, cx);
        }
    }
};

// ------------------------------------------------------------------------
// im2col, 3x3 window, stride 1, padding 1.  Vector path (W % 4 == 0,
// W <= 64): a warp takes a chunk of rows of one (n, c) plane, each half-warp
// half of the chunk; lane holds 4 columns of three consecutive input rows
// and writes the nine shifted copies (ky, kx) of its columns for each row.
struct BodyIm2col {
    using Args = hf_im2col3_args;
    static constexpr int kId = HF_BODY_IM2COL3;
    static constexpr int kBarriers = 0;
    // ring path: a stage holds an item's 14 rows and its two halo rows
    // (rows of up to 64 floats)
    static constexpr int kRingRows = 14;
    static constexpr bool kRingItem = true;
    static constexpr unsigned kRingMinBytes = 4096;   // the stage: one item

    // chunks of whole rows (W <= 64, 16-byte rows) arrive as one bulk copy
    static __host__ bool uses_ring(const Args &a)
    {
        return (int64_t)a.N * a.C * a.H * a.W > 0 && (a.W & 3) == 0 && a.W <= 64 && aligned16(a.x) &&
               aligned16(a.col);
    }

    static __host__ size_t workspace_bytes(const Args &) { return 0; }
    static __host__ size_t smem_bytes(int, const Args &) { return 0; }
    static __host__ hf_status validate(const Args &a)
    {
        if (a.N < 0 || a.C < 0 || a.H < 0 || a.W < 0) return HF_ERR_INVALID;
        if ((int64_t)a.N * a.C * a.H * a.W == 0) return HF_OK;
        if (!a.x || !a.col) return HF_ERR_INVALID;
        if ((int64_t)a.N * a.C * a.H * a.W * 9 >= (int64_t)1 << 40) return HF_ERR_INVALID;
        return HF_OK;
    }

    struct Row {
        float4 q;
        float L, R;   // columns c0-1 and c0+4 (0 outside the image)
    };

    static __device__ __forceinline__ float4 load(const float *xp, int iy, int H, int W, int c0,
                                                  bool act)
    {
        const bool ok = act && iy >= 0 && iy < H;
        return ok ? ldg4(xp + (int64_t)iy * W + c0) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    static __device__ __forceinline__ Row halo(float4 q, int c0, int W)
    {
        Row r;
        r.q = q;
        const int sub = lane_id() & 15;
        r.L = __shfl_up_sync(0xffffffffu, q.w, 1);
        r.R = __shfl_down_sync(0xffffffffu, q.x, 1);
        if (sub == 0) r.L = 0.f;
        if (c0 + 4 >= W) r.R = 0.f;
        return r;
    }

    // The three kx-shifted copies of one input row (rows ky*3 + 0..2).
    static __device__ __forceinline__ void emit(const Row &r, float *base, int64_t HW)
    {
        stcs4(base, make_float4(r.L, r.q.x, r.q.y, r.q.z));
        stcs4(base + HW, r.q);
        stcs4(base + 2 * HW, make_float4(r.q.y, r.q.z, r.q.w, r.R));
    }

    // Work items are (plane, chunk of rows); each half-warp takes half of a
    // chunk.  A plane is cut into as many chunks as give the interval's
    // warps about three items each (whole planes when there are enough of
    // them): with one item per plane, 2048 planes kept only 2048 of a
    // GB300's 9728 warp slots busy.  Every chunk re-reads its two halo rows
    // (from L2 in practice).
    static __device__ void run_vec(const Args &a, const Ctx &cx)
    {
        const int H = a.H, W = a.W;
        const int64_t HW = (int64_t)H * W;
        const int64_t planes = (int64_t)a.N * a.C;
        const int nw = cx.nthreads >> 5;
        const int64_t nwt = (int64_t)cx.grid * nw;
        const int lane = lane_id();
        const int half = lane >> 4;
        const int c0 = 4 * (lane & 15);
        const bool act = c0 < W;
        const int want = (int)min((3 * nwt + planes - 1) / planes, (int64_t)(H + 1) / 2);
        const int hh = ((H + max(want, 1) - 1) / max(want, 1) + 1) / 2;   // rows per half-warp
        const int nchunk = (H + 2 * hh - 1) / (2 * hh);
        const int64_t items = planes * nchunk;
        for (int64_t it = (int64_t)cx.block * nw + (cx.tid >> 5); it < items; it += nwt) {
            const int64_t pl = it / nchunk;
            const int ch = (int)(it - pl * nchunk);
            const int64_t n = pl / a.C;
            const int c = (int)(pl - n * a.C);
            const float *xp = a.x + pl * HW;
            float *cp = a.col + (n * a.C * 9 + (int64_t)c * 9) * HW;
            const int oyb = ch * 2 * hh + half * hh;
            const int oye = min(oyb + hh, H);
            Row up = halo(load(xp, oyb - 1, H, W, c0, act), c0, W);
            Row mid = halo(load(xp, oyb, H, W, c0, act), c0, W);
            float4 nq = load(xp, oyb + 1, H, W, c0, act);
#pragma unroll 2
            for (int i = 0; i < hh; ++i) {
                const int oy = oyb + i;
                const bool valid = act && oy < oye;
                float4 fq = load(xp, oy + 2, H, W, c0, act && oy + 1 < oye);
                Row dn = halo(nq, c0, W);
                if (valid) {
                    float *base = cp + (int64_t)oy * W + c0;
                    emit(up, base, HW);
                    emit(mid, base + 3 * HW, HW);
                    emit(dn, base + 6 * HW, HW);
                }
                up = mid;
                mid = dn;
                nq = fq;
            }
        }
    }

    // Ring path.  Work item = (plane, chunk of R = 14 rows); the chunk and
    // its halo rows, [max(r0-1, 0), min(r0+R+1, H)), are contiguous and
    // arrive in one bulk copy in a stage of the warp's ring.  As in the
    // register path each half-warp takes half of the chunk and lane l of a
    // half the columns 4l..4l+3, sliding three rows (from shared memory,
    // zero outside the image) and writing the nine shifted copies per row.
    static __device__ bool run_ring(const Args &a, const Ctx &cx)
    {
        constexpr int R = kRingRows, RH = R / 2;
        const int H = a.H, W = a.W;
        const int64_t HW = (int64_t)H * W;
        const unsigned row_bytes = 4u * (unsigned)W;
        const int64_t planes = (int64_t)a.N * a.C;
        if (cx.ring_stage < (R + 2) * row_bytes || planes * H >= ((int64_t)1 << 32)) return false;
        const unsigned ns = (unsigned)((H + R - 1) / R);
        const int64_t items = planes * ns;
        WarpRing r;
        r.init(cx, 0);
        const int nw = cx.nthreads >> 5;
        const int64_t gw = (int64_t)cx.block * nw + (cx.tid >> 5), GW = (int64_t)cx.grid * nw;
        const unsigned dq = (unsigned)(GW / ns), dr = (unsigned)(GW % ns);
        const int lane = lane_id();
        const int half = lane >> 4;
        const int c0 = 4 * (lane & 15);
        const bool act = c0 < W;
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        ItemCursor fc, uc;   // the fill cursor runs S items ahead of the use cursor
        fc.init(gw, ns);
        uc = fc;
        ring_stream(
            r, gw, GW, items,
            [&](int st, int64_t) {
                const int r0 = (int)fc.s * R;
                const int ylo = max(r0 - 1, 0), yhi = min(r0 + R + 1, H);
                const unsigned bytes = (unsigned)(yhi - ylo) * row_bytes;   // rows are 16-byte multiples
                r.expect(st, bytes);
                r.copy(st, 0, a.x + ((uint64_t)fc.p * (unsigned)H + (unsigned)ylo) * W, bytes);
                fc.step(dq, dr, ns);
            },
            [&](const unsigned char *stage, int64_t) {
                const int r0 = (int)uc.s * R;
                const int ylo = max(r0 - 1, 0), yhi = min(r0 + R + 1, H);
                const unsigned char *base = stage + (act ? 4 * c0 : 0);
                auto ld = [&](int y) {
                    const int yc = min(max(y, ylo), yhi - 1);   // an in-stage row
                    const float4 q = *reinterpret_cast<const float4 *>(base + (unsigned)(yc - ylo) * row_bytes);
                    return (act && y >= 0 && y < H) ? q : zero;
                };
                const unsigned n = uc.p / (unsigned)a.C, c = uc.p - n * (unsigned)a.C;
                float *cp = a.col + ((int64_t)n * a.C * 9 + (int64_t)c * 9) * HW;
                const int oyb = r0 + half * RH, oye = min(oyb + RH, H);
                Row up = halo(ld(oyb - 1), c0, W);
                Row mid = halo(ld(oyb), c0, W);
#pragma unroll
                for (int i = 0; i < RH; ++i) {
                    const int oy = oyb + i;
                    Row dn = halo(ld(oy + 1), c0, W);
                    if (act && oy < oye) {
                        float *o = cp + (int64_t)oy * W + c0;
                        emit(up, o, HW);
                        emit(mid, o + 3 * HW, HW);
                        emit(dn, o + 6 * HW, HW);
                    }
                    up = mid;
                    mid = dn;
                }
                uc.step(dq, dr, ns);
            });
        r.finish();
        return true;
    }

    static __device__ void run_scalar(const Args &a, const Ctx &cx)
    {
        const int H = a.H, W = a.W;
        const int64_t HW = (int64_t)H * W;
        const int64_t total = (int64_t)a.N * a.C * 9 * HW;
        for (int64_t i = (int64_t)cx.block * cx.nthreads + cx.tid; i < total;
             i += (int64_t)cx.grid * cx.nthreads) {
            const int64_t pix = i % HW;
            const int64_t row = i / HW;            // n*C*9 + c*9 + ky*3 + kx
            const int k = (int)(row % 9);
            const int64_t plane = row / 9;         // n*C + c
            const int oy = (int)(pix / W), ox = (int)(pix % W);
            const int iy = oy + k / 3 - 1, ix = ox + k % 3 - 1;
            float v = 0.f;
            if (iy >= 0 && iy < H && ix >= 0 && ix < W) v = __ldg(a.x + plane * HW + (int64_t)iy * W + ix);
            a.col[i] = v;
        }
    }

    static __device__ void run(const Args &a, const Ctx &cx)
    {
        if ((int64_t)a.N * a.C * a.H * a.W == 0) return;
        if ((a.W & 3) == 0 && a.W <= 64 && aligned16(a.x) && aligned16(a.col)) {
            if (WarpRing::available(cx, 0) && run_ring(a, cx)) return;
            run_vec(a, cx);
        } else {
            run_scalar(a, cx);
        }
    }
};

} // namespace hf
