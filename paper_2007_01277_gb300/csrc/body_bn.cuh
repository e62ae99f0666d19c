// body_bn.cuh -- batch-norm statistics body (the batch_norm_collect_statistics
// kernel of Sec. 2.3 / Sec. 4.1): per-channel mean and biased variance of an
// NCHW float32 tensor.
//
// GB300 layout.  Channel c is the sequence of its M = N*HW values (N runs of
// HW contiguous floats).  It is cut into tiles of TILE values; one warp
// reduces one tile at a time (warps stride over all C*T tiles of the grid),
// streaming it with 128-bit loads, 16 per lane with 8 in flight.  Each tile
// yields FP32 sums of d = x - K_c and d*d, where the shift K_c = x[0][c][0]
// keeps the variance free of cancellation (the shifted-data algorithm,
// Chan, Golub & LeVeque 1983).  A warp writes the tile's pair to the
// workspace; after its last tile it fences and bumps a per-channel counter
// once per tile, and the warp that brings channel c's counter to T combines
// that channel's T pairs in FP64 in tile order, writes mean/var and resets
// the counter.  There is no block barrier in the streaming loop; the
// reduction order depends only on (tile size, warp), so a fused interval and
// a standalone launch with the same grid give identical bits.
#pragma once
#include "hf_device.cuh"

namespace hf {

struct BodyBn {
    using Args = hf_bn_stats_args;
    static constexpr int kId = HF_BODY_BN_STATS;
    static constexpr int kTile = 2048;   // values per tile (multiple of 128)
    static constexpr int kBarriers = 0;

    static __host__ __device__ int64_t tiles_per_channel(const Args &a)
    {
        int64_t M = (int64_t)a.N * a.HW;
        return (M + kTile - 1) / kTile;
    }
    static __host__ size_t counters_bytes(const Args &a)
    {
        return ((size_t)a.C * sizeof(unsigned) + 255) / 256 * 256;
    }
    static __host__ size_t workspace_bytes(const Args &a)
    {
        if (a.C <= 0) return 0;
        return counters_bytes(a) + (size_t)a.C * tiles_per_channel(a) * sizeof(float2);
    }
    static __host__ size_t smem_bytes(int /*nthreads*/, const Args &) { return 0; }
    static __host__ hf_status validate(const Args &a)
    {
        if (a.N < 0 || a.C < 0 || a.HW < 0) return HF_ERR_INVALID;
        if (a.C == 0) return HF_OK;
        if (a.N == 0 || a.HW == 0) return HF_ERR_INVALID;
        if (!a.x || !a.mean || !a.var || !a.workspace) return HF_ERR_INVALID;
        if (!aligned16(a.workspace)) return HF_ERR_INVALID;
        if ((int64_t)a.N * a.C * a.HW >= (int64_t)1 << 40) return HF_ERR_INVALID;
        return HF_OK;
    }

    template <int VEC>
    static __device__ __forceinline__ void tile_sums(const Args &a, int c, int64_t t, float K,
                                                     float &s1, float &s2)
    {
        const int64_t M = (int64_t)a.N * a.HW;
        const int lane = lane_id();
        const int64_t j0 = t * kTile + (int64_t)VEC * lane;
        // (n, hw) of this lane's first value; later values advance by 32*VEC.
        int n = (int)(j0 / a.HW);
        int hw = (int)(j0 - (int64_t)n * a.HW);
        const int64_t jend = (t + 1) * kTile < M ? (t + 1) * kTile : M;
        float p1[VEC], p2[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) p1[v] = 0.f, p2[v] = 0.f;
        // VEC == 4: the four per-lane sums as two packed pairs (same
        // operations per value, half the instructions)
        unsigned long long P1a = f2pack(0.f, 0.f), P1b = P1a, P2a = P1a, P2b = P1a;
        const unsigned long long KK = f2pack(K, K);
        constexpr int kSteps = kTile / (32 * VEC);
        constexpr int kBatch = 8;
        int64_t j = j0;
#pragma unroll 1
        for (int s = 0; s < kSteps; s += kBatch) {
            float vals[kBatch][VEC];
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
                const bool ok = (s + b < kSteps) && (j < jend);
                const float *p = a.x + ((int64_t)n * a.C + c) * a.HW + hw;
                if (VEC == 4) {
                    float4 q = ok ? ldcs4(p) : make_float4(K, K, K, K);
                    vals[b][0] = q.x;
                    if (VEC > 1) vals[b][1 % VEC] = q.y;
                    if (VEC > 2) vals[b][2 % VEC] = q.z;
                    if (VEC > 3) vals[b][3 % VEC] = q.w;
                } else {
                    vals[b][0] = ok ? __ldcs(p) : K;
                }
                j += 32 * VEC;
                hw += 32 * VEC;
                while (hw >= a.HW) {
                    hw -= a.HW;
                    ++n;
                }
            }
            if (VEC == 4) {
#pragma unroll
                for (int b = 0; b < kBatch; ++b) {
                    const unsigned long long Da = f2sub(f2pack(vals[b][0], vals[b][1 % VEC]), KK);
                    const unsigned long long Db = f2sub(f2pack(vals[b][2 % VEC], vals[b][3 % VEC]), KK);
                    P1a = f2add(P1a, Da);
                    P1b = f2add(P1b, Db);
                    P2a = f2fma(Da, Da, P2a);
                    P2b = f2fma(Db, Db, P2b);
                }
            } else {
#pragma unroll
                for (int b = 0; b < kBatch; ++b)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        float d = __fsub_rn(vals[b][v], K);
                        p1[v] = __fadd_rn(p1[v], d);
                        p2[v] = __fmaf_rn(d, d, p2[v]);
                    }
            }
        }
        if (VEC == 4) {
            f2unpack(P1a, p1[0], p1[1 % VEC]);
            f2unpack(P1b, p1[2 % VEC], p1[3 % VEC]);
            f2unpack(P2a, p2[0], p2[1 % VEC]);
            f2unpack(P2b, p2[2 % VEC], p2[3 % VEC]);
        }
        s1 = p1[0];
        s2 = p2[0];
#pragma unroll
        for (int v = 1; v < VEC; ++v) {
            s1 = __fadd_rn(s1, p1[v]);
            s2 = __fadd_rn(s2, p2[v]);
        }
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
            s1 = __fadd_rn(s1, __shfl_xor_sync(0xffffffffu, s1, m));
            s2 = __fadd_rn(s2, __shfl_xor_sync(0xffffffffu, s2, m));
        }
    }

    // Combine the T tile pairs of channel c (FP64, tile order per lane, then
    // a butterfly whose result is identical on every lane) and write it out.
    static __device__ __forceinline__ void finalize(const Args &a, int c, int64_t T,
                                                    const float2 *part, unsigned *cnt)
    {
        const int lane = lane_id();
        double s1 = 0.0, s2 = 0.0;
        for (int64_t t = lane; t < T; t += 32) {
            float2 q = __ldcg(part + (int64_t)c * T + t);
            s1 += (double)q.x;
            s2 += (double)q.y;
        }
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, m);
            s2 += __shfl_xor_sync(0xffffffffu, s2, m);
        }
        if (lane == 0) {
            const double M = (double)a.N * (double)a.HW;
            const double K = (double)__ldg(a.x + (int64_t)c * a.HW);
            const double m1 = s1 / M;
            double var = s2 / M - m1 * m1;
            a.mean[c] = (float)(K + m1);
            a.var[c] = (float)(var > 0.0 ? var : 0.0);
            cnt[c] = 0u;
        }
    }

    template <int VEC>
    static __device__ __forceinline__ void run_vec(const Args &a, const Ctx &cx)
    {
        const int64_t T = tiles_per_channel(a);
        const int64_t ntiles = (int64_t)a.C * T;
        unsigned *cnt = reinterpret_cast<unsigned *>(a.workspace);
        float2 *part = reinterpret_cast<float2 *>(
            reinterpret_cast<unsigned char *>(a.workspace) +
            ((size_t)a.C * sizeof(unsigned) + 255) / 256 * 256);
        const int nw = cx.nthreads >> 5;
        const int64_t gw = (int64_t)cx.block * nw + (cx.tid >> 5);
        const int64_t TW = (int64_t)cx.grid * nw;
        const int lane = lane_id();
        int k = 0;
        for (int64_t tile = gw; tile < ntiles; tile += TW, ++k) {
            const int c = (int)(tile / T);
            const int64_t t = tile - (int64_t)c * T;
            const float K = __ldg(a.x + (int64_t)c * a.HW);
            float s1, s2;
            tile_sums<VEC>(a, c, t, K, s1, s2);
            if ((k & 31) == lane) part[tile] = make_float2(s1, s2);
        }
        // Release this warp's tile pairs, then count them (lane k%32 wrote
        // and counts the warp's k-th tile: store -> fence -> atomic in one
        // thread).
        __threadfence();
        k = 0;
        for (int64_t base = gw; base < ntiles; base += 32 * TW, k += 32) {
            const int64_t tile = base + (int64_t)lane * TW;
            bool last = false;
            int c = 0;
            if (tile < ntiles) {
                c = (int)(tile / T);
                last = atomicAdd(cnt + c, 1u) == (unsigned)(T - 1);
            }
            unsigned mask = __ballot_sync(0xffffffffu, last);
            if (mask) __threadfence();
            while (mask) {
                const int src = __ffs(mask) - 1;
                mask &= mask - 1;
                const int cc = __shfl_sync(0xffffffffu, c, src);
                finalize(a, cc, T, part, cnt);
            }
        }
    }

    static __device__ void run(const Args &a, const Ctx &cx)
    {
        if (a.C <= 0) return;
        if ((a.HW & 3) == 0 && aligned16(a.x))
            run_vec<4>(a, cx);
        else
            run_vec<1>(a, cx);
    }
};

} // namespace hf
