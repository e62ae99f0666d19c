// kernels.cuh -- the kernels that host the bodies: a standalone launch, the
// 2-way horizontally fused kernel of Algorithm 1 (Sec. 3.1) and the N-way
// persistent fused kernel, plus their type-erased host launchers.
//
// 2-way fused kernel (Algorithm 1):
//   prologue   tid_k = threadIdx.x - offset_k, size_k = d_k  (the Ctx)
//   barriers   body k uses "bar.sync id_k, d_k": id 1 for the low interval,
//              id 2 for the high one (Sec. 3.1)
//   guards     warps below the split run one body, the rest the other; the
//              branch is warp-uniform (the split is a multiple of 32), the
//              structured form of the goto/label guards of Algorithm 1
//   resources  dynamic shared memory = low slice + high slice (128-byte
//              aligned); registers are what the compiler needs for both
//              bodies, optionally bounded by __maxnreg__ (Algorithm 2's r0)
#pragma once
#include <cstring>

#include "hf_launch.h"

#include "body_bn.cuh"
#include "body_fp.cuh"
#include "body_hash.cuh"
#include "body_int.cuh"
#include "body_resample.cuh"

namespace hf {

// ------------------------------------------------------------------ single
template <class B>
struct SingleParams {
    typename B::Args a;
    unsigned *err;         // device error word
    unsigned ring_stage;   // bulk-copy ring geometry chosen by the launch
    int ring_stages;
};

template <class B>
__device__ __forceinline__ void single_body(const SingleParams<B> &p)
{
    extern __shared__ __align__(128) unsigned char hf_smem[];
    Ctx c;
    c.tid = threadIdx.x;
    c.nthreads = blockDim.x;
    c.bar = 0;   // standalone: the block barrier, as the original kernel had
    c.block = blockIdx.x;
    c.grid = gridDim.x;
    c.smem = hf_smem;
    c.smem_end = dynamic_smem_end(hf_smem);
    c.err = p.err;
    c.ring_stage = p.ring_stage;
    c.ring_stages = p.ring_stages;
#ifdef HF_CHECKED_BARRIERS
    __shared__ unsigned chk_bar[2];
    if (threadIdx.x < 2) chk_bar[threadIdx.x] = 0u;
    __syncthreads();
    c.chk_bar = chk_bar;
#endif
    B::run(p.a, c);
}

// A kernel launched alone, with the registers the compiler picks; block
// sizes its registers do not allow are refused by the runtime.
template <class B>
__global__ void k_single(const __grid_constant__ SingleParams<B> p)
{
    single_body<B>(p);
}

// ------------------------------------------------------------------ pair
template <class A, class B>
struct PairParams {
    typename A::Args a;
    typename B::Args b;
    int w_split;        // warps in the low interval
    int n_low, n_high;  // threads in the low / high interval
    unsigned smem_high; // byte offset of the high interval's shared slice
    int low_is_a;       // 1: body A runs on the low interval
    unsigned *err;      // device error word
    unsigned ring_stage_low, ring_stage_high;   // ring geometry per interval
    int ring_stages_low, ring_stages_high;
};

template <class A, class B>
__device__ __forceinline__ void pair_body(const PairParams<A, B> &p)
{
    extern __shared__ __align__(128) unsigned char hf_smem[];
    const bool low = (int)(threadIdx.x >> 5) < p.w_split;
    Ctx c;
    c.block = blockIdx.x;
    c.grid = gridDim.x;
    c.err = p.err;
    const unsigned end = dynamic_smem_end(hf_smem);
    if (low) {
        c.tid = threadIdx.x;
        c.nthreads = p.n_low;
        c.bar = 1;
        c.smem = hf_smem;
        c.smem_end = min(end, (unsigned)__cvta_generic_to_shared(hf_smem) + p.smem_high);
        c.ring_stage = p.ring_stage_low;
        c.ring_stages = p.ring_stages_low;
    } else {
        c.tid = threadIdx.x - p.n_low;
        c.nthreads = p.n_high;
        c.bar = 2;
        c.smem = hf_smem + p.smem_high;
        c.smem_end = end;
        c.ring_stage = p.ring_stage_high;
        c.ring_stages = p.ring_stages_high;
    }
#ifdef HF_CHECKED_BARRIERS
    // the two intervals' software-barrier words, zeroed by the whole block
    // before it splits
    __shared__ unsigned chk_bar[2][2];
    if (threadIdx.x < 4) chk_bar[threadIdx.x >> 1][threadIdx.x & 1] = 0u;
    __syncthreads();
    c.chk_bar = chk_bar[low ? 0 : 1];
#endif
    if (low == (p.low_is_a != 0))
        A::run(p.a, c);
    else
        B::run(p.b, c);
}

template <class A, class B>
__global__ void k_pair(const __grid_constant__ PairParams<A, B> p)
{
    pair_body<A, B>(p);
}

template <class A, class B, int R>
__global__ void __maxnreg__(R) k_pair_cap(const __grid_constant__ PairParams<A, B> p)
{
    pair_body<A, B>(p);
}

// ------------------------------------------------------------------ N-way
constexpr int kNwayBlob = 4096;

struct NwayParams {
    int n_int;                                  // intervals
    int warp_begin[HF_MAX_INTERVALS + 1];       // interval i = warps [wb[i], wb[i+1])
    unsigned smem_off[HF_MAX_INTERVALS];        // shared slice of interval i
    int int_first[HF_MAX_INTERVALS + 1];        // interval i runs slots [if[i], if[i+1])
    int sched_body[HF_MAX_SCHEDULE];            // body id of slot j (slots sorted by interval)
    unsigned args_off[HF_MAX_SCHEDULE];         // argument block of slot j in blob
    unsigned char warp_int[32];                 // interval of each warp of the block
    unsigned long long *trace;                  // optional: [n_int][2] first start / last end (ns)
    unsigned *err;                              // device error word
    unsigned ring_stage[HF_MAX_INTERVALS];      // ring geometry of interval i
    int ring_stages[HF_MAX_INTERVALS];
    // The first polynomial of the schedule also gets its arguments at a
    // fixed offset of the parameter bank: its coefficients are then
    // constant-bank operands of the multiply-adds, as in a standalone
    // launch, instead of registers loaded through a run-time offset.
    int poly_slot;                              // its slot, or -1
    hf_poly_args poly;
    alignas(16) unsigned char blob[kNwayBlob];
};

__device__ __forceinline__ unsigned long long global_ns() { return timer_ns(); }

__device__ __forceinline__ void dispatch(const NwayParams &p, int j, const Ctx &c)
{
    const unsigned char *args = p.blob + p.args_off[j];
    switch (p.sched_body[j]) {
    case HF_BODY_BN_STATS: BodyBn::run(*reinterpret_cast<const BodyBn::Args *>(args), c); break;
    case HF_BODY_UPSAMPLE2X:
        BodyUpsample::run(*reinterpret_cast<const BodyUpsample::Args *>(args), c);
        break;
    case HF_BODY_MAXPOOL3S2:
        BodyMaxpool::run(*reinterpret_cast<const BodyMaxpool::Args *>(args), c);
        break;
    case HF_BODY_IM2COL3:
        BodyIm2col::run(*reinterpret_cast<const BodyIm2col::Args *>(args), c);
        break;
    case HF_BODY_HIST256: BodyHist::run(*reinterpret_cast<const BodyHist::Args *>(args), c); break;
    case HF_BODY_PHILOX:
        BodyPhilox::run(*reinterpret_cast<const BodyPhilox::Args *>(args), c);
        break;
    case HF_BODY_POLY:
        if (j == p.poly_slot) BodyPoly::run(p.poly, c);
        else BodyPoly::run(*reinterpret_cast<const BodyPoly::Args *>(args), c);
        break;
    case HF_BODY_BF16_AXPY:
        BodyBf16Axpy::run(*reinterpret_cast<const BodyBf16Axpy::Args *>(args), c);
        break;
    case HF_BODY_STREAM_TMPL:
        BodyStreamTmpl::run(*reinterpret_cast<const BodyStreamTmpl::Args *>(args), c);
        break;
    case HF_BODY_SHA256D:
        BodySha256d::run(*reinterpret_cast<const BodySha256d::Args *>(args), c);
        break;
    case HF_BODY_BLAKE256:
        BodyBlake256::run(*reinterpret_cast<const BodyBlake256::Args *>(args), c);
        break;
    case HF_BODY_BLAKE2B:
        BodyBlake2b::run(*reinterpret_cast<const BodyBlake2b::Args *>(args), c);
        break;
    default: break;
    }
}

// The interval context of interval i, rebuilt from the parameter bank and
// special registers each time it is needed, so nothing of it stays live in
// registers across a body (register pressure under a cap is what decides
// whether the fused kernel spills).
__device__ __forceinline__ Ctx interval_ctx(const NwayParams &p, int i)
{
    extern __shared__ __align__(128) unsigned char hf_smem[];
    Ctx c;
    c.tid = threadIdx.x - 32 * p.warp_begin[i];
    c.nthreads = 32 * (p.warp_begin[i + 1] - p.warp_begin[i]);
    c.bar = i + 1;
    c.block = blockIdx.x;
    c.grid = gridDim.x;
    c.smem = hf_smem + p.smem_off[i];
    const unsigned end = dynamic_smem_end(hf_smem);
    c.smem_end = i + 1 < p.n_int
                     ? min(end, (unsigned)__cvta_generic_to_shared(hf_smem) + p.smem_off[i + 1])
                     : end;
    c.err = p.err;
    c.ring_stage = p.ring_stage[i];
    c.ring_stages = p.ring_stages[i];
    return c;
}

__device__ __forceinline__ void nway_body(const NwayParams &p)
{
    const int i = p.warp_int[threadIdx.x >> 5];
    if (p.trace && (threadIdx.x & 31) == 0) atomicMin(p.trace + 2 * i, global_ns());
    const int j0 = p.int_first[i];
    for (int j = j0; j < p.int_first[i + 1]; ++j) {
        // kernels sharing an interval share its shared slice: the previous
        // one must be done with it before the next starts
        if (j > j0) interval_sync(interval_ctx(p, i));
        dispatch(p, j, interval_ctx(p, i));
    }
    if (p.trace && (threadIdx.x & 31) == 0) atomicMax(p.trace + 2 * i + 1, global_ns());
}

__global__ void __launch_bounds__(512) k_nway(const __grid_constant__ NwayParams p);
template <int R>
__global__ void __maxnreg__(R) k_nway_cap(const __grid_constant__ NwayParams p)
{
    nway_body(p);
}

// ------------------------------------------------------------------ host side
// The device error word of the current device (runtime.cu), or NULL.
unsigned *error_word();

using hfl::Instance;     // registry entry of one compiled instance
using hfl::PairLaunch;   // arguments of one 2-way launch

template <class A, class B, int R>
const void *pair_func()
{
    if constexpr (R == 0)
        return reinterpret_cast<const void *>(&k_pair<A, B>);
    else
        return reinterpret_cast<const void *>(&k_pair_cap<A, B, R>);
}

template <class A, class B, int R>
cudaError_t launch_pair(const PairLaunch &L, cudaStream_t s)
{
    PairParams<A, B> p;
    std::memset(&p, 0, sizeof p);
    std::memcpy(&p.a, L.args[0], sizeof(typename A::Args));
    std::memcpy(&p.b, L.args[1], sizeof(typename B::Args));
    p.w_split = L.w_split;
    p.n_low = L.n_low;
    p.n_high = L.n_high;
    p.smem_high = L.smem_high;
    p.low_is_a = L.low_is_a;
    p.err = L.err;
    p.ring_stage_low = L.ring_stage[0];
    p.ring_stage_high = L.ring_stage[1];
    p.ring_stages_low = L.ring_stages[0];
    p.ring_stages_high = L.ring_stages[1];
    void *kargs[] = {&p};
    return cudaLaunchKernel(pair_func<A, B, R>(), dim3(L.grid), dim3(L.d0), kargs, L.smem_total, s);
}

template <class A, class B, int R>
Instance make_pair_instance()
{
    return Instance{A::kId, B::kId, R, pair_func<A, B, R>(), &launch_pair<A, B, R>};
}

// Table accessors implemented by the instantiation units.
const Instance *pair_table_0(int *n);
const Instance *pair_table_1(int *n);
const Instance *pair_table_2(int *n);
const Instance *pair_table_3(int *n);
const Instance *pair_table_4(int *n);
const Instance *nway_table(int *n);

// Standalone kernels: one per body, no register bound.
struct SingleEntry {
    int body;
    const void *func;
    cudaError_t (*launch)(const void *args, int threads, int grid, unsigned smem, unsigned *err,
                          unsigned ring_stage, int ring_stages, cudaStream_t);
};

template <class B>
cudaError_t launch_single(const void *args, int threads, int grid, unsigned smem, unsigned *err,
                          unsigned ring_stage, int ring_stages, cudaStream_t s)
{
    SingleParams<B> p;
    std::memset(&p, 0, sizeof p);
    std::memcpy(&p.a, args, sizeof(typename B::Args));
    p.err = err;
    p.ring_stage = ring_stage;
    p.ring_stages = ring_stages;
    void *kargs[] = {&p};
    return cudaLaunchKernel(reinterpret_cast<const void *>(&k_single<B>), dim3(grid),
                            dim3(threads), kargs, smem, s);
}

const SingleEntry *single_table(int *n);

// The register caps compiled for every fused pair and the N-way kernel.
#define HF_REGCAP_LIST(X) X(32) X(40) X(48) X(64) X(96) X(128)

} // namespace hf
