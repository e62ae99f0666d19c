// hf_device.cuh -- interval context, named barriers and memory helpers shared
// by every constituent body.
//
// A body never reads threadIdx / blockDim and never calls __syncthreads():
// the prologue of a fused kernel (Algorithm 1, Sec. 3.1) hands it an
// interval context instead -- its thread index tid_k, its interval size
// size_k = d_k, and the named barrier id that replaces the block barrier
// ("bar.sync id, d_k", Sec. 3.1 "Replace Synchronization Barriers").  The
// block index and grid size pass through unchanged, so bodies stride over
// the grid and compute the full result for any grid.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "../../include/hfuse.h"

namespace hf {

struct Ctx {
    int tid;             // thread index within the interval, [0, nthreads)
    int nthreads;        // interval size d_k, a multiple of 32
    int bar;             // named barrier id of the interval (0 = block barrier)
    int block;           // blockIdx.x
    int grid;            // gridDim.x
    unsigned char *smem; // this interval's slice of dynamic shared memory
    unsigned smem_end;   // shared-space address one past the slice
    unsigned *err;       // the device's error word (bits below), or NULL
    unsigned ring_stage; // bulk-copy ring of this interval: stage bytes per warp
    int ring_stages;     //   and stages per warp (0: no ring, use register loads)
#ifdef HF_CHECKED_BARRIERS
    unsigned *chk_bar;   // checked build: the interval's two software-barrier words
#endif
};

// Bits of the device error word read by hf_check_device_error().
constexpr unsigned kErrWaitExpired = 1u;      // a bounded wait on a bulk copy gave up
constexpr unsigned kErrBarrierExpired = 2u;   // a bounded software barrier gave up

// Shared-space address of the start of dynamic shared memory plus its size
// as launched (the %dynamic_smem_size register).
__device__ __forceinline__ unsigned dynamic_smem_end(const unsigned char *dyn_base)
{
    unsigned sz;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(sz));
    return (unsigned)__cvta_generic_to_shared(dyn_base) + sz;
}

// True when `bytes` from the start of the interval's slice were provided by
// the launch.  Bodies that stage through shared memory check this and take
// a path without shared memory otherwise, so an under-sized launch can never
// touch memory outside its allocation.
__device__ __forceinline__ bool smem_fits(const Ctx &c, size_t bytes)
{
    return (size_t)(unsigned)__cvta_generic_to_shared(c.smem) + bytes <= (size_t)c.smem_end;
}

#ifndef HF_CHECKED_BARRIERS
// The partial barrier of Sec. 3.1: only the d_k threads of this interval
// arrive.  Intervals are whole warps, so every warp either executes it with
// all its threads or not at all, as bar.sync requires.
__device__ __forceinline__ void interval_sync(const Ctx &c)
{
    asm volatile("bar.sync %0, %1;" ::"r"(c.bar), "r"(c.nthreads) : "memory");
}
#endif

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ unsigned long long timer_ns();

// A software barrier over `nwarps` warps with a bounded wait, for checking a
// barrier schedule without the risk of a hang: where a hardware barrier
// whose count is never reached would stall its warps for good, this one
// gives up after limit_ns of the global timer, sets kErrBarrierExpired in
// the error word and returns false.  bar points to two shared words
// (arrivals, generation), zero before first use; lane 0 of each warp
// arrives once, the last arrival resets the count and advances the
// generation, the others wait for the generation to change.
__device__ __forceinline__ bool soft_barrier(unsigned *bar, int nwarps, unsigned *err,
                                             unsigned long long limit_ns)
{
    volatile unsigned *vb = bar;
    bool ok = true;
    __syncwarp();
    if (lane_id() == 0) {
        const unsigned gen = vb[1];
        __threadfence_block();
        if (atomicAdd(&bar[0], 1u) + 1u == (unsigned)nwarps) {
            vb[0] = 0u;
            __threadfence_block();
            atomicAdd(&bar[1], 1u);
        } else {
            const unsigned long long t0 = timer_ns();
            while (vb[1] == gen) {
                if (timer_ns() - t0 > limit_ns) {
                    if (err) atomicOr(err, kErrBarrierExpired);
                    ok = false;
                    break;
                }
                __nanosleep(64);
            }
            __threadfence_block();
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok;
}

#ifdef HF_CHECKED_BARRIERS
// Checked build: the partial barrier of Sec. 3.1 becomes the bounded
// software barrier above over the interval's warps, so a barrier schedule
// whose count is never reached ends in kErrBarrierExpired after one second
// instead of a hang.  The fused kernel's prologue zeroes the interval's two
// words before any body runs.
constexpr unsigned long long kCheckedBarrierLimitNs = 1000000000ull;
__device__ __forceinline__ void interval_sync(const Ctx &c)
{
    soft_barrier(c.chk_bar, c.nthreads >> 5, c.err, kCheckedBarrierLimitNs);
}
#endif

// Packed FP32 pairs: two floats in one 64-bit register and the f32x2
// operations of sm_100 and later.  Each half is an ordinary correctly
// rounded operation, so a packed computation equals the scalar one bit for
// bit; it takes half the instructions (issue slots are what a body shares
// with the other bodies of a fused block).
__device__ __forceinline__ unsigned long long f2pack(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2unpack(unsigned long long r, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long f2fma(unsigned long long a, unsigned long long b,
                                                    unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long f2add(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2sub(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Read-only global loads through the non-coherent path.
__device__ __forceinline__ float4 ldg4(const float *p)
{
    return __ldg(reinterpret_cast<const float4 *>(p));
}
__device__ __forceinline__ uint4 ldg4u(const void *p)
{
    return __ldg(reinterpret_cast<const uint4 *>(p));
}
// Streaming (evict-first) loads and stores for data touched once.
__device__ __forceinline__ float4 ldcs4(const float *p)
{
    return __ldcs(reinterpret_cast<const float4 *>(p));
}
__device__ __forceinline__ uint4 ldcs4u(const void *p)
{
    return __ldcs(reinterpret_cast<const uint4 *>(p));
}
__device__ __forceinline__ void stcs4(float *p, float4 v)
{
    __stcs(reinterpret_cast<float4 *>(p), v);
}
__device__ __forceinline__ void stcs4u(void *p, uint4 v)
{
    __stcs(reinterpret_cast<uint4 *>(p), v);
}
__device__ __forceinline__ void stcs2(float *p, float2 v)
{
    __stcs(reinterpret_cast<float2 *>(p), v);
}

// Atomic add with acquire-release semantics at GPU scope; returns the old
// value.
__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
                 : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Atomic add on shared memory with acquire-release semantics at CTA scope;
// returns the old value.
__device__ __forceinline__ unsigned atom_add_acq_rel_cta_shared(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;"
                 : "=r"(old) : "r"((unsigned)__cvta_generic_to_shared(p)), "r"(v) : "memory");
    return old;
}

__host__ __device__ __forceinline__ bool aligned16(const void *p)
{
    return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

} // namespace hf

namespace hf {

// ------------------------------------------------------------------ bulk rings
// A per-warp ring of S stages in the interval's shared slice, each filled by
// bulk asynchronous copies (cp.async.bulk, the untiled TMA copy) that signal
// completion on the stage's mbarrier.  Lane 0 issues the copies; the warp
// waits on the barrier's phase.  A warp thus keeps several tiles in flight
// however few warps its interval has: the bandwidth of a memory-bound body
// inside a fused block no longer depends on its share of the block's
// warps.
//
// The geometry (stage bytes B, stages S) comes from the launch (Ctx).  For a
// body that streams tiles of a flat array the runtime sizes it for the whole
// SM -- all stream-ring warps of all resident blocks -- to about 40 KB in
// flight, where a pure stream's bandwidth peaks; a body that takes one work
// item per stage gets two stages of its item size.  Ring layout from `off`
// in the slice: nw x S
// stages of B bytes (warp w owns stages [w*S, w*S+S)), then nw x S 8-byte
// barriers.  Every wait is bounded in time; when it expires the warp sets
// kErrWaitExpired in the device error word, waits (bounded) for the copies
// it still has in flight and stops consuming its ring.

__device__ __forceinline__ unsigned long long timer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bytes of a ring of S stages of B bytes for an interval of nthreads.
__host__ __device__ constexpr size_t ring_bytes(int nthreads, unsigned B, int S)
{
    return (size_t)(nthreads / 32) * S * (B + 8);
}

struct WarpRing {
    unsigned char *data;    // this warp's stage 0 (generic address)
    unsigned bars;          // shared address of this warp's barrier 0
    unsigned bytes;         // stage size
    int stages, lane;
    unsigned *err;
    unsigned long long limit_ns;

    // True when the launch gave this interval a ring that fits its slice
    // from byte `off` (a multiple of 128).
    static __device__ bool available(const Ctx &c, size_t off)
    {
        return c.ring_stages >= 2 && c.ring_stage >= 512 && c.ring_stage % 128 == 0 &&
               smem_fits(c, off + ring_bytes(c.nthreads, c.ring_stage, c.ring_stages));
    }
    // All lanes of the warp call this, after available() held.  Stages are
    // 128-byte multiples from a 128-byte aligned start, so every stage is a
    // valid bulk-copy destination.
    __device__ void init(const Ctx &c, size_t off, unsigned long long limit = 2000000000ull)
    {
        const int nw = c.nthreads >> 5, w = c.tid >> 5;
        stages = c.ring_stages;
        const unsigned B = c.ring_stage;
        bytes = B;
        lane = c.tid & 31;
        err = c.err;
        limit_ns = limit;
        data = c.smem + off + (size_t)w * stages * B;
        bars = (unsigned)__cvta_generic_to_shared(c.smem + off + (size_t)nw * stages * B) + 8u * w * stages;
        if (lane == 0) {
            for (int s = 0; s < stages; ++s)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bars + 8u * s) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncwarp();
    }
    __device__ unsigned char *stage(int s) const { return data + (size_t)s * bytes; }

    // Lane 0: the next phase of stage s completes after `tx` bytes arrive.
    __device__ void expect(int s, unsigned tx) const
    {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bars + 8u * s), "r"(tx)
                     : "memory");
    }
    // Lane 0: bulk copy of n bytes (n % 16 == 0, src 16-byte aligned) from
    // global memory to offset `off` of stage s.
    __device__ void copy(int s, unsigned off, const void *src, unsigned n) const
    {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(stage(s)) + off;
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(dst), "l"(src), "r"(n), "r"(bars + 8u * s)
                     : "memory");
    }
    // Lane 0, before refilling a stage the warp has read: order those reads
    // before the copy engine's writes.
    __device__ void refill_fence() const { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

    // All lanes: wait for stage s's phase `parity`.  Each try suspends the
    // thread in hardware until the phase completes or kSuspendNs pass (a
    // try without the hint returns at once, and a warp spinning on it takes
    // issue slots from the warps that compute); the expiry decision is taken
    // for the whole warp (vote and lane 0's clock), so lanes never diverge.
    static constexpr unsigned kSuspendNs = 200000;
    __device__ bool wait(int s, unsigned parity) const
    {
        unsigned long long t0 = 0;
        for (unsigned it = 0;; ++it) {
            unsigned done;
            asm volatile("{\n\t.reg .pred p;\n\t"
                         "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                         "selp.u32 %0, 1, 0, p;\n\t}"
                         : "=r"(done)
                         : "r"(bars + 8u * s), "r"(parity), "n"(kSuspendNs)
                         : "memory");
            if (__all_sync(0xffffffffu, done)) return true;
            const unsigned long long now = __shfl_sync(0xffffffffu, timer_ns(), 0);
            if (it == 0) t0 = now;
            else if (now - t0 > limit_ns) return false;
        }
    }
    // All lanes, after the last wait: release the barriers' memory.
    __device__ void finish() const
    {
        __syncwarp();
        if (lane == 0)
            for (int s = 0; s < stages; ++s)
                asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bars + 8u * s) : "memory");
        __syncwarp();
    }
};

// Streams tiles first, first + step, ... < count of this warp through the
// ring: fill(s, t) runs on lane 0 and issues expect() + copy() for tile t
// into stage s; use(p, t) runs on every lane once the stage has landed.
// Returns false when a wait expired (error recorded, in-flight copies
// drained with bounded waits).
template <class Fill, class Use>
__device__ bool ring_stream(const WarpRing &r, int64_t first, int64_t step, int64_t count, Fill fill,
                            Use use)
{
    const int S = r.stages;
    if (r.lane == 0)
        for (int s = 0; s < S; ++s)
            if (first + s * step < count) fill(s, first + s * step);
    int s = 0;
    unsigned ph = 0;
    for (int64_t t = first; t < count; t += step) {
        if (!r.wait(s, ph)) {
            if (r.lane == 0 && r.err) atomicOr(r.err, kErrWaitExpired);
            for (int k = 0; k < S; ++k)   // the expired stage included
                if (t + k * step < count) r.wait((s + k) % S, ph ^ (s + k >= S ? 1u : 0u));
            return false;
        }
        use(r.stage(s), t);
        __syncwarp();
        if (r.lane == 0 && t + S * step < count) {
            r.refill_fence();
            fill(s, t + S * step);
        }
        if (++s == S) {
            s = 0;
            ph ^= 1u;
        }
    }
    return true;
}

} // namespace hf
