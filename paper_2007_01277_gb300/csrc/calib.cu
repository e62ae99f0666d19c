// calib.cu -- pipe-throughput calibration kernels.
//
// The ideal-overlap bound of a fused launch is the larger of its HBM time
// and, for each execution pipe, the operations the constituents issue there
// divided by that pipe's throughput.  These kernels measure the throughputs
// on the running device (clock behaviour included) instead of using nominal
// figures: independent FP32 fused multiply-add chains, 32-bit integer
// multiplies (high and low halves, the Philox mix), conflict-free
// shared-memory atomic adds (the histogram's counting operation), and the
// 32-bit add / XOR / rotate mix of the hash rounds.
#include <algorithm>
#include <vector>

#include "kernels.cuh"

namespace hf {
hf_status set_last_error(hf_status s, const char *msg);   // runtime.cu
}

namespace {

constexpr int kChains = 8;

// Sink for the results the kernels keep live (written only on a condition
// that does not occur; indices stay below the block size of 256).
__device__ unsigned g_cal_sink[1024];

__global__ void k_cal_ffma(float *out, int iters)
{
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 1.0f + 1e-3f * (threadIdx.x + j);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = __fmaf_rn(a[j], 0.9999f, 1e-4f);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == -1.0f) out[threadIdx.x] = s;   // never true; keeps the chains live
}

// The Philox4x32 round itself on kChains / 2 independent register states:
// per round two products, each a high half (__umulhi) and a low half, and
// two three-input XORs.  A chain of one product and one XOR per step
// measured 1.32e13 multiplies/s while the Philox body alone, store-bound,
// already ran at 1.70e13/s, so the pipe bound is calibrated on the round.
__global__ void k_cal_imul(unsigned *out, int iters)
{
    constexpr int S = kChains / 2;
    unsigned c0[S], c1[S], c2[S], c3[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
        c0[j] = threadIdx.x * 2654435761u + j;
        c1[j] = c0[j] ^ 0x9E3779B9u;
        c2[j] = c0[j] + 0xBB67AE85u;
        c3[j] = c1[j] * 3u;
    }
    for (int i = 0; i < iters; ++i) {
        const unsigned k0 = 0x9E3779B9u * (unsigned)i, k1 = 0xBB67AE85u * (unsigned)i;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const unsigned h0 = __umulhi(0xD2511F53u, c0[j]), l0 = 0xD2511F53u * c0[j];
            const unsigned h1 = __umulhi(0xCD9E8D57u, c2[j]), l1 = 0xCD9E8D57u * c2[j];
            c0[j] = h1 ^ c1[j] ^ k0;
            c2[j] = h0 ^ c3[j] ^ k1;
            c1[j] = l1;
            c3[j] = l0;
        }
    }
    unsigned s = 0;
#pragma unroll
    for (int j = 0; j < S; ++j) s ^= c0[j] ^ c1[j] ^ c2[j] ^ c3[j];
    if (s == 0x12345678u) out[threadIdx.x] = s;
}

// One add, one XOR and one rotate (funnel shift) per step: the operation mix
// of a BLAKE G function or a SHA-256 round.
__global__ void k_cal_ialu(unsigned *out, int iters)
{
    unsigned c[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) c[j] = threadIdx.x * 2654435761u + j;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kChains; ++j) c[j] = __funnelshift_r(c[j], c[j], 7) ^ (c[j] + 0x9E3779B9u);
    unsigned s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s ^= c[j];
    if (s == 0x12345678u) out[threadIdx.x] = s;
}

__global__ void k_cal_satom(unsigned *out, int iters)
{
    extern __shared__ unsigned sh[];
    const int lane = threadIdx.x & 31;
    unsigned *mine = sh + (threadIdx.x >> 5) * 256;
    for (int i = threadIdx.x; i < blockDim.x * 8; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) atomicAdd(mine + ((lane + 32 * ((i + j) & 7)) & 255), 1u);
    __syncthreads();
    if (mine[lane] == 0xffffffffu) out[threadIdx.x] = 1;
}

// A bounded wait that nothing completes: one warp waits on an mbarrier no
// copy will ever arrive at, gives up after limit_ns and records
// kErrWaitExpired.  No copy is in flight, so giving up is safe.
// Rounds of the bounded software barrier over every warp of the block but
// `missing` (-1: none).  With every warp present each round completes; with
// one missing the others give up after limit_ns and set kErrBarrierExpired.
// No warp waits on anything another block owns.
__global__ void k_selftest_barrier(unsigned *err, int missing, int rounds, unsigned long long limit_ns,
                                   unsigned *completed)
{
    __shared__ unsigned bar[2];
    if (threadIdx.x == 0) bar[0] = bar[1] = 0u;
    __syncthreads();
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (w == missing) return;
    int done = 0;
    for (int r = 0; r < rounds; ++r) {
        if (!hf::soft_barrier(bar, nw, err, limit_ns)) break;
        ++done;
    }
    if ((threadIdx.x & 31) == 0 && completed) atomicAdd(completed, (unsigned)done);
}

__global__ void k_selftest_wait(unsigned *err, unsigned long long limit_ns)
{
    extern __shared__ __align__(128) unsigned char sm[];
    hf::Ctx c;
    c.tid = threadIdx.x;
    c.nthreads = 32;
    c.bar = 0;
    c.block = 0;
    c.grid = 1;
    c.smem = sm;
    c.smem_end = hf::dynamic_smem_end(sm);
    c.err = err;
    c.ring_stage = 512;
    c.ring_stages = 2;
    hf::WarpRing r;
    r.init(c, 0, limit_ns);
    if (!r.wait(0, 0) && threadIdx.x == 0 && err) atomicOr(err, hf::kErrWaitExpired);
    r.finish();
}

template <class F>
hf_status time_ms(F f, cudaStream_t s, float *ms)
{
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return HF_ERR_CUDA;
    f();   // warm-up
    std::vector<float> t;
    for (int r = 0; r < 5; ++r) {
        cudaEventRecord(a, s);
        f();
        cudaEventRecord(b, s);
        if (cudaEventSynchronize(b) != cudaSuccess) return HF_ERR_CUDA;
        float x = 0;
        cudaEventElapsedTime(&x, a, b);
        t.push_back(x);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    std::sort(t.begin(), t.end());
    *ms = t[2];
    return cudaGetLastError() == cudaSuccess ? HF_OK : HF_ERR_CUDA;
}

} // namespace

extern "C" hf_status hf_calibrate(int what, void *stream, double *ops_per_s)
{
    if (!ops_per_s || what < 0 || what > 3) return hf::set_last_error(HF_ERR_INVALID, "bad calibration id");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 256, blocks = 8 * sms;   // 64 warps per SM
    const int iters = 4096;
    void *out = nullptr;
    float ms = 0.f;
    hf_status st;
    cudaError_t e = cudaGetSymbolAddress(&out, g_cal_sink);
    if (e != cudaSuccess) return hf::set_last_error(HF_ERR_CUDA, cudaGetErrorString(e));
    if (what == 0) {
        st = time_ms([&] { k_cal_ffma<<<blocks, threads, 0, s>>>((float *)out, iters); }, s, &ms);
        *ops_per_s = (double)blocks * threads * iters * kChains / (ms * 1e-3);
    } else if (what == 1) {
        st = time_ms([&] { k_cal_imul<<<blocks, threads, 0, s>>>((unsigned *)out, iters); }, s, &ms);
        *ops_per_s = 4.0 * blocks * threads * iters * (kChains / 2) / (ms * 1e-3);   // 4 per round
    } else if (what == 3) {
        st = time_ms([&] { k_cal_ialu<<<blocks, threads, 0, s>>>((unsigned *)out, iters); }, s, &ms);
        *ops_per_s = 3.0 * blocks * threads * iters * kChains / (ms * 1e-3);
    } else {
        st = time_ms([&] { k_cal_satom<<<blocks, threads, 8 * threads * 4, s>>>((unsigned *)out, iters / 4); },
                     s, &ms);
        *ops_per_s = (double)blocks * threads * (iters / 4) * 8 / (ms * 1e-3);
    }
    if (st) return hf::set_last_error(st, "calibration kernel failed");
    return HF_OK;
}

extern "C" hf_status hf_selftest_barrier(int warps, int missing, int rounds, int limit_us,
                                         unsigned *d_completed, void *stream)
{
    if (warps < 1 || warps > 32 || missing < -1 || missing >= warps || rounds < 1 || rounds > 1000)
        return hf::set_last_error(HF_ERR_INVALID, "bad self-test shape");
    if (limit_us <= 0 || limit_us > 10000000) return hf::set_last_error(HF_ERR_INVALID, "limit out of range");
    k_selftest_barrier<<<1, 32 * warps, 0, static_cast<cudaStream_t>(stream)>>>(
        hf::error_word(), missing, rounds, 1000ull * limit_us, d_completed);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hf::set_last_error(HF_ERR_CUDA, cudaGetErrorString(e));
    return HF_OK;
}

extern "C" hf_status hf_selftest_wait_timeout(int limit_us, void *stream)
{
    if (limit_us <= 0 || limit_us > 10000000) return hf::set_last_error(HF_ERR_INVALID, "limit out of range");
    const size_t smem = hf::ring_bytes(32, 512, 2);
    k_selftest_wait<<<1, 32, smem, static_cast<cudaStream_t>(stream)>>>(hf::error_word(),
                                                                          1000ull * limit_us);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hf::set_last_error(HF_ERR_CUDA, cudaGetErrorString(e));
    return HF_OK;
}
