// body_bn.cuh -- batch-norm statistics body (the batch_norm_collect_statistics
// kernel of Sec. 2.3 / Sec. 4.1): per-channel mean and biased variance of an
// NCHW float32 tensor.
//
// GB300 layout.  Channel c is the sequence of its M = N*HW values (N runs of
// HW contiguous floats).  It is cut into tiles of TILE values; one warp
// reduces one tile at a time (each block's warps share its contiguous range
// of tiles through a counter in shared memory).  A tile arrives either
// through the warp's bulk-copy ring (its one to three runs copied into one
// stage, the next tiles' copies in flight) or, without a ring, as 128-bit
// loads, 16 per lane with 8 in flight.  Each tile yields FP32 sums of
// d = x - K_c and d*d, where the shift K_c = x[0][c][0] keeps the variance
// free of cancellation (the shifted-data algorithm, Chan, Golub & LeVeque
// 1983), in the same order on both paths.  A warp writes the tile's pair to
// the workspace and counts the tile -- in the block's shared-memory counter
// of channel c, the block's share then added to the global counter in one
// acquire-release atomic; the warp that brings channel c's global counter to
// T combines that channel's T pairs in tile order (double-float sums),
// writes mean/var and resets the counter.  The only block-level barrier is
// the one after the pool and the counters are set; the reduction order
// depends only on the tile size, so a fused interval and a standalone launch
// give identical bits whatever their threads, grid and path.
#pragma once
#include "hf_device.cuh"

namespace hf {

struct BodyBn {
    using Args = hf_bn_stats_args;
    static constexpr int kId = HF_BODY_BN_STATS;
    static constexpr int kTile = 2048;   // values per tile (multiple of 128)
    static constexpr int kBarriers = 1;   // once, after the tile pool is set up

    static __host__ __device__ int64_t tiles_per_channel(const Args &a)
    {
        int64_t M = (int64_t)a.N * a.HW;
        return (M + kTile - 1) / kTile;
    }
    // Workspace: C per-channel tile counters, then the C*T tile pairs.
    static __host__ __device__ size_t counters_bytes(const Args &a)
    {
        return ((size_t)a.C * sizeof(unsigned) + 255) / 256 * 256;
    }
    static __host__ size_t workspace_bytes(const Args &a)
    {
        if (a.C <= 0) return 0;
        return counters_bytes(a) + (size_t)a.C * tiles_per_channel(a) * sizeof(float2);
    }
    static constexpr size_t kPoolBytes = 16;   // the block's tile pool counter
    // then kSlots per-channel tile counters of the block (block counting)
    static constexpr int kSlots = 24;
    static constexpr size_t kCountBytes = kPoolBytes + kSlots * sizeof(unsigned);
    static constexpr size_t kRingOffset = 128;   // the ring follows the counters
    // ring path: one stage per tile (its <= 3 contiguous runs, HW >= 1024)
    static constexpr bool kRingItem = true;
    static constexpr unsigned kRingMinBytes = kTile * sizeof(float);
    static __host__ bool uses_ring(const Args &a)
    {
        return a.C > 0 && a.N > 0 && a.HW >= 1024 && (a.HW & 3) == 0 && aligned16(a.x);
    }
    static __host__ size_t smem_bytes(int /*nthreads*/, const Args &) { return kRingOffset; }
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

    // The tile's FP32 sums of d = x - K and d*d, in the one order every
    // path uses: lane l takes the VEC values at tile offsets VEC*l + 32*VEC*k
    // for k = 0, 1, ... (values past the channel's end read as K, so d = 0),
    // in batches of 8 steps whose values get(k) returns -- the batch's
    // loads are all issued before its arithmetic; four per-lane sums (two
    // packed pairs for VEC = 4), then their sum and a warp butterfly.
    template <int VEC, class Get>
    static __device__ __forceinline__ void accumulate(Get get, float K, float &s1, float &s2)
    {
        float p1[VEC], p2[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) p1[v] = 0.f, p2[v] = 0.f;
        // VEC == 4: the four per-lane sums as two packed pairs (same
        // operations per value, half the instructions)
        unsigned long long P1a = f2pack(0.f, 0.f), P1b = P1a, P2a = P1a, P2b = P1a;
        const unsigned long long KK = f2pack(K, K);
        constexpr int kSteps = kTile / (32 * VEC);
        constexpr int kBatch = 8;
#pragma unroll 1
        for (int s = 0; s < kSteps; s += kBatch) {
            float vals[kBatch][VEC];
#pragma unroll
            for (int b = 0; b < kBatch; ++b) get(s + b, vals[b]);
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

    // Register path: the values straight from global memory (streaming
    // loads), the lane's (n, hw) position advanced step by step.
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
        int64_t j = j0;
        accumulate<VEC>(
            [&](int, float(&v)[VEC]) {
                const bool ok = j < jend;
                const float *p = a.x + ((int64_t)n * a.C + c) * a.HW + hw;
                if (VEC == 4) {
                    const float4 q = ok ? ldcs4(p) : make_float4(K, K, K, K);
                    v[0] = q.x;
                    v[1 % VEC] = q.y;
                    v[2 % VEC] = q.z;
                    v[3 % VEC] = q.w;
                } else {
                    v[0] = ok ? __ldcs(p) : K;
                }
                j += 32 * VEC;
                hw += 32 * VEC;
                while (hw >= a.HW) {
                    hw -= a.HW;
                    ++n;
                }
            },
            K, s1, s2);
    }

    // Double-float sums: hi + lo, |lo| <= ulp(hi)/2, about 48 significant
    // bits.  FP64 arithmetic is a narrow, long-latency pipe on this part
    // (the five-level FP64 butterfly of this combine took 0.45 us, about
    // 90 ns a level); FP32 adds take a few cycles.  The addition is Knuth's
    // TwoSum of the high parts (the exact rounding error, whatever the
    // operand order) plus the low parts, then renormalised; it is
    // commutative bit for bit, so a butterfly leaves the same value on
    // every lane.
    struct DF {
        float hi, lo;
    };
    static __device__ __forceinline__ DF df_add(DF a, DF b)
    {
        const float s = __fadd_rn(a.hi, b.hi);
        const float bb = __fsub_rn(s, a.hi);
        float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
        e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
        const float hi = __fadd_rn(s, e);
        return DF{hi, __fsub_rn(e, __fsub_rn(hi, s))};
    }
    static __device__ __forceinline__ DF df_shfl_xor(DF a, int m)
    {
        return DF{__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m)};
    }

    // Combine the T tile pairs of channel c (double-float sums, tile order
    // per lane, then a butterfly whose result is identical on every lane)
    // and write mean and variance, formed in FP64 by lane 0.  K is the
    // channel's shift; each lane issues its loads four at a time.
    static __device__ __forceinline__ void finalize(const Args &a, int c, int64_t T, float K,
                                                    const float2 *part, unsigned *cnt)
    {
        const int lane = lane_id();
        const double inv_m = 1.0 / ((double)a.N * (double)a.HW);   // overlaps the loads
        const float2 *pc = part + (int64_t)c * T;
        DF s1{0.f, 0.f}, s2{0.f, 0.f};
        for (int64_t t0 = 0; t0 < T; t0 += 128) {
            float2 q[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t t = t0 + 32 * j + lane;
                q[j] = t < T ? __ldcg(pc + t) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                s1 = df_add(s1, DF{q[j].x, 0.f});
                s2 = df_add(s2, DF{q[j].y, 0.f});
            }
        }
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
            s1 = df_add(s1, df_shfl_xor(s1, m));
            s2 = df_add(s2, df_shfl_xor(s2, m));
        }
        if (lane == 0) {
            const double m1 = ((double)s1.hi + (double)s1.lo) * inv_m;
            const double var = fma(-m1, m1, ((double)s2.hi + (double)s2.lo) * inv_m);
            a.mean[c] = (float)((double)K + m1);
            a.var[c] = (float)(var > 0.0 ? var : 0.0);
            cnt[c] = 0u;
        }
    }

    // Counting finished tiles.  A channel is complete when all its T tiles
    // are counted; the warp whose count completes it runs the combine.
    // Per tile, a GPU-scope acquire-release atomic (its fence waits for the
    // warp's memory operations, the top stall of a warp that has no other
    // warps to hide it behind) -- unless the block counts first: its range
    // of tiles covers channels c_lo..c_lo+k (k < kSlots), each warp adds
    // its finished tile to the channel's counter in shared memory
    // (acquire-release at CTA scope) and the warp that completes the
    // block's share of a channel adds that share to the global counter in
    // one GPU-scope atomic.  The pairs stored by the block's other warps are
    // ordered before that atomic through the CTA-scope counter (release
    // sequences compose), so the combine sees them all.
    struct Counter {
        unsigned *slots;          // shared counters, or nullptr: count each tile globally
        unsigned bstart, bend, T, c_lo;   // 32-bit: block counting needs C*T < 2^31
        // lane 0: counts the finished tile of channel c; true when that
        // completes channel c
        __device__ bool count(unsigned *cnt, int c) const
        {
            if (!slots) return atom_add_acq_rel_gpu(cnt + c, 1u) == T - 1u;
            const unsigned lo = max(bstart, (unsigned)c * T), hi = min(bend, (unsigned)(c + 1) * T);
            const unsigned mine = hi - lo;   // the block's tiles of c
            if (atom_add_acq_rel_cta_shared(slots + (c - c_lo), 1u) + 1u != mine) return false;
            return atom_add_acq_rel_gpu(cnt + c, mine) + mine == T;
        }
    };
    // Block counting when the block's range [bstart, bend) spans at most
    // kSlots channels (slots zeroed by the caller before the interval
    // barrier) and every tile index fits in 31 bits.
    static __device__ __forceinline__ Counter make_counter(unsigned *slots, unsigned long long bstart,
                                                           unsigned long long bend, unsigned long long T,
                                                           unsigned long long ntiles)
    {
        Counter k;
        const bool fits = slots && ntiles < (1ull << 31) && bend > bstart &&
                          (bend - 1) / T - bstart / T < (unsigned long long)kSlots;
        k.slots = fits ? slots : nullptr;
        k.bstart = (unsigned)bstart;
        k.bend = (unsigned)bend;
        k.T = (unsigned)T;
        k.c_lo = fits ? (unsigned)(bstart / T) : 0u;
        return k;
    }

    // Tile assignment.  With the pool (a counter in the interval's shared
    // memory) block b owns a contiguous range of about C*T/grid tiles and
    // its warps take them in order one at a time, asking for the next one a
    // tile ahead: a warp slowed by a combine, or by the other bodies of a
    // fused block, simply takes fewer of its block's tiles.  A channel's
    // tiles then belong to a few neighbouring blocks, completed one after
    // another (64x256x56x56: 40.9 us against 44.9 with tiles b, b + grid,
    // ..., which spread each channel over 98 blocks finishing together).
    // One dispenser for the whole grid in global memory serialised every
    // request on one address.  Without shared memory, warp w takes tiles
    // w, w + W, ... of the W warps.
    template <int VEC>
    static __device__ __forceinline__ void run_vec(const Args &a, const Ctx &cx, unsigned *pool)
    {
        const int64_t T = tiles_per_channel(a);
        const unsigned long long ntiles = (unsigned long long)a.C * T;
        unsigned *cnt = reinterpret_cast<unsigned *>(a.workspace);
        float2 *part = reinterpret_cast<float2 *>(reinterpret_cast<unsigned char *>(a.workspace) +
                                                  counters_bytes(a));
        const int lane = lane_id();
        const unsigned long long stride = (unsigned long long)cx.grid * (unsigned long long)(cx.nthreads >> 5);
        // block b's range [bstart, bend): the first ntiles % grid blocks get
        // one tile more
        const unsigned long long G = (unsigned long long)cx.grid, b = (unsigned long long)cx.block;
        const unsigned long long q = ntiles / G, rem = ntiles % G;
        const unsigned long long bstart = b * q + (b < rem ? b : rem);
        const unsigned long long bend = bstart + q + (b < rem ? 1ull : 0ull);
        const Counter counter = make_counter(pool ? pool + kPoolBytes / sizeof(unsigned) : nullptr, bstart, bend,
                                             (unsigned long long)T, ntiles);
        unsigned long long tile;
        if (pool) {
            unsigned i = 0;
            if (lane == 0) i = atomicAdd(pool, 1u);
            tile = bstart + __shfl_sync(0xffffffffu, i, 0);
            if (tile >= bend) tile = ntiles;
        } else {
            tile = (unsigned long long)cx.block * (cx.nthreads >> 5) + (cx.tid >> 5);
        }
        while (tile < ntiles) {
            unsigned inext = 0;
            if (pool && lane == 0) inext = atomicAdd(pool, 1u);
            const int c = (int)(tile / (unsigned long long)T);
            const int64_t t = (int64_t)tile - (int64_t)c * T;
            const float K = __ldg(a.x + (int64_t)c * a.HW);
            float s1, s2;
            tile_sums<VEC>(a, c, t, K, s1, s2);
            // Lane 0 publishes the tile's pair and counts it with an
            // acquire-release atomic at GPU scope: the release orders the
            // pair before the count, and the lane whose increment completes
            // channel c acquires every other warp's pairs of c; the warp
            // barrier then orders the whole warp's reads after that acquire.
            bool last = false;
            if (lane == 0) {
                part[tile] = make_float2(s1, s2);
                last = counter.count(cnt, c);
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __syncwarp();
                finalize(a, c, T, K, part, cnt);
            }
            if (pool) {
                tile = bstart + __shfl_sync(0xffffffffu, inext, 0);
                if (tile >= bend) tile = ntiles;
            } else {
                tile += stride;
            }
        }
    }

    // Ring path.  The same tiles, taken from the block's pool two ahead:
    // lane 0 copies each tile's runs of the channel (a tile crosses at most
    // two image boundaries when HW >= 1024) into a stage of the warp's ring,
    // contiguous in the tile's order, and the lanes read their values from
    // shared memory in the order of accumulate(), so the sums -- and with
    // them the results -- are those of the register path, bit for bit.
    // Returns false (nothing done) when the launch's ring does not fit.
    static __device__ bool run_ring(const Args &a, const Ctx &cx, unsigned *pool)
    {
        const int64_t T64 = tiles_per_channel(a);
        const int64_t M = (int64_t)a.N * a.HW;
        // 32-bit tile arithmetic (fewer registers); larger tensors take the
        // register path
        if (!pool || cx.ring_stages != 2 || cx.ring_stage < kRingMinBytes || (int64_t)a.C * T64 >= ((int64_t)1 << 31) ||
            M >= ((int64_t)1 << 31) || !WarpRing::available(cx, kRingOffset))
            return false;
        const unsigned T = (unsigned)T64;
        const unsigned ntiles = (unsigned)a.C * T;
        unsigned *cnt = reinterpret_cast<unsigned *>(a.workspace);
        float2 *part = reinterpret_cast<float2 *>(reinterpret_cast<unsigned char *>(a.workspace) +
                                                  counters_bytes(a));
        const int lane = lane_id();
        const unsigned G = (unsigned)cx.grid, b = (unsigned)cx.block;
        const unsigned q = ntiles / G, rem = ntiles % G;
        const unsigned bstart = b * q + (b < rem ? b : rem);
        const unsigned bend = bstart + q + (b < rem ? 1u : 0u);
        WarpRing r;
        r.init(cx, kRingOffset);
        // lane 0: the next tile of the block's range (ntiles when done)
        auto grab = [&]() -> unsigned {
            const unsigned tl = bstart + atomicAdd(pool, 1u);
            return tl < bend ? tl : ntiles;
        };
        // lane 0: the tile's runs into stage st
        auto fill = [&](int st, unsigned tile) {
            const unsigned c = tile / T, t = tile - c * T;
            int j = (int)(t * kTile);
            const int jend = min(j + kTile, (int)M);
            r.expect(st, (unsigned)(4 * (jend - j)));
            int n = j / a.HW;
            int hw = j - n * a.HW;
            const int j0 = j;
            while (j < jend) {
                const int len = min(a.HW - hw, jend - j);
                r.copy(st, (unsigned)(4 * (j - j0)), a.x + ((int64_t)n * a.C + c) * a.HW + hw, (unsigned)(4 * len));
                j += len;
                hw = 0;
                ++n;
            }
        };
        unsigned tl0 = ntiles, tl1 = ntiles;   // the stages' tiles (lane 0)
        if (lane == 0) {
            tl0 = grab();
            if (tl0 < ntiles) fill(0, tl0);
            tl1 = grab();
            if (tl1 < ntiles) fill(1, tl1);
        }
        const Counter counter = make_counter(pool + kPoolBytes / sizeof(unsigned), bstart, bend, T, ntiles);
        int s = 0;
        unsigned ph = 0;
        for (;;) {
            // tiles are grabbed in increasing order: once one is past the
            // range, so is every later one, and no copy is in flight
            const unsigned tile = __shfl_sync(0xffffffffu, s ? tl1 : tl0, 0);
            if (tile >= ntiles) break;
            if (!r.wait(s, ph)) {
                if (lane == 0 && cx.err) atomicOr(cx.err, kErrWaitExpired);
                const unsigned other = __shfl_sync(0xffffffffu, s ? tl0 : tl1, 0);
                if (other < ntiles) r.wait(s ^ 1, s ? ph ^ 1u : ph);
                break;
            }
            const int c = (int)(tile / T);
            const int tt = (int)(tile - (unsigned)c * T);
            const float K = __ldg(a.x + (int64_t)c * a.HW);
            const int valid = min(kTile, (int)M - tt * kTile);   // values of this tile
            const float4 *st4 = reinterpret_cast<const float4 *>(r.stage(s));
            float s1, s2;
            accumulate<4>(
                [&](int k, float(&v)[4]) {
                    const int off = 4 * lane + 128 * k;   // value offset within the tile
                    const float4 x4 = off < valid ? st4[off >> 2] : make_float4(K, K, K, K);
                    v[0] = x4.x;
                    v[1] = x4.y;
                    v[2] = x4.z;
                    v[3] = x4.w;
                },
                K, s1, s2);
            __syncwarp();
            if (lane == 0) {
                r.refill_fence();
                const unsigned nx = grab();
                if (nx < ntiles) fill(s, nx);
                if (s) tl1 = nx;
                else tl0 = nx;
            }
            bool last = false;
            if (lane == 0) {
                part[tile] = make_float2(s1, s2);
                last = counter.count(cnt, c);
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __syncwarp();
                finalize(a, c, (int64_t)T, K, part, cnt);
            }
            s ^= 1;
            if (s == 0) ph ^= 1u;
        }
        r.finish();
        return true;
    }

    static __device__ void run(const Args &a, const Ctx &cx)
    {
        if (a.C <= 0) return;
        unsigned *pool = nullptr;
        if (smem_fits(cx, kCountBytes)) {
            pool = reinterpret_cast<unsigned *>(cx.smem);
            for (int i = cx.tid; i < (int)(kCountBytes / sizeof(unsigned)); i += cx.nthreads) pool[i] = 0u;
            interval_sync(cx);
        }
        if ((a.HW & 3) == 0 && aligned16(a.x)) {
            if (a.HW >= 1024 && run_ring(a, cx, pool)) return;
            run_vec<4>(a, cx, pool);
        } else {
            run_vec<1>(a, cx, pool);
        }
    }
};

} // namespace hf
