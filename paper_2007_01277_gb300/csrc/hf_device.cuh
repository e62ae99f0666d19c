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
};

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

// The partial barrier of Sec. 3.1: only the d_k threads of this interval
// arrive.  Intervals are whole warps, so every warp either executes it with
// all its threads or not at all, as bar.sync requires.
__device__ __forceinline__ void interval_sync(const Ctx &c)
{
    asm volatile("bar.sync %0, %1;" ::"r"(c.bar), "r"(c.nthreads) : "memory");
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

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

__host__ __device__ __forceinline__ bool aligned16(const void *p)
{
    return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

} // namespace hf
