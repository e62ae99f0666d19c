// noalloc.cu -- batch-norm statistics for callers that may not allocate
// device memory.
//
// The regular batch-norm body needs scratch (per-channel counters and the
// per-tile partial sums) that the caller allocates as a workspace.  This
// variant keeps that scratch in one fixed file-scope device array instead,
// so a call allocates nothing: no cudaMalloc, no cudaFree, no allocating
// library routine.  The array is part of the library's device image: every
// GPU that loads the library holds HF_BN_NOALLOC_SCRATCH_BYTES for it until
// the process exits.
//
// Host code must not pass the array's name to a kernel: in host code that
// name is only a host-side stand-in for the symbol.  The device address is
// looked up with cudaGetSymbolAddress once per device, with that device
// current, on the first call made there.
#include <cstring>
#include <mutex>

#include "kernels.cuh"

namespace hf {
hf_status set_last_error(hf_status s, const char *msg);   // runtime.cu
}

namespace {

using hf::BodyBn;

// Counters first, then the tile partial sums (the workspace layout of the
// batch-norm body).
static __device__ __align__(256) unsigned char g_bn_scratch[HF_BN_NOALLOC_SCRATCH_BYTES];

__global__ void k_bn_noalloc(const __grid_constant__ hf::SingleParams<BodyBn> p)
{
    hf::single_body<BodyBn>(p);
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch[kMaxDevices];   // device address of g_bn_scratch, per device

hf_status scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return hf::set_last_error(HF_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return hf::set_last_error(HF_ERR_INVALID, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bn_scratch);
        if (e != cudaSuccess) return hf::set_last_error(HF_ERR_CUDA, cudaGetErrorString(e));
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    return HF_OK;
}

} // namespace

extern "C" hf_status hf_bn_stats_noalloc(const float *x, float *mean, float *var, int N, int C,
                                         int HW, int threads, int grid, void *stream)
{
    if (threads < 32 || threads > 1024 || threads % 32)
        return hf::set_last_error(HF_ERR_INVALID, "threads must be a multiple of 32 in [32, 1024]");
    if (grid < 0) return hf::set_last_error(HF_ERR_INVALID, "negative grid");
    if (N < 0 || C < 0 || HW < 0) return hf::set_last_error(HF_ERR_INVALID, "negative size");
    if (C == 0) return HF_OK;
    if (N == 0 || HW == 0) return hf::set_last_error(HF_ERR_INVALID, "empty channel");
    if (!x || !mean || !var) return hf::set_last_error(HF_ERR_INVALID, "NULL tensor");
    if ((int64_t)N * C * HW >= (int64_t)1 << 40) return hf::set_last_error(HF_ERR_INVALID, "tensor too large");

    hf_bn_stats_args a{x, mean, var, N, C, HW, nullptr};
    const size_t need = BodyBn::workspace_bytes(a);
    if (need > (size_t)HF_BN_NOALLOC_SCRATCH_BYTES)
        return hf::set_last_error(
            HF_ERR_INVALID,
            "shape needs more scratch than the fixed array holds: C * ceil(N*HW/2048) tile slots "
            "plus C counters exceed HF_BN_NOALLOC_SCRATCH_BYTES; use the workspace entry point");

    void *scratch = nullptr;
    hf_status s = scratch_address(&scratch);
    if (s) return s;
    a.workspace = scratch;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // The array keeps the previous call's contents: the counters must start
    // at zero, the partial sums are always written before they are read.
    cudaError_t e = cudaMemsetAsync(scratch, 0, BodyBn::counters_bytes(a), st);
    if (e != cudaSuccess) return hf::set_last_error(HF_ERR_CUDA, cudaGetErrorString(e));

    // dynamic shared memory as for every other launch of the body
    const size_t smem = BodyBn::smem_bytes(threads, a);
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k_bn_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return hf::set_last_error(HF_ERR_CUDA, cudaGetErrorString(e));
    if (grid == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
            (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bn_noalloc, threads, smem)) !=
                cudaSuccess)
            return hf::set_last_error(HF_ERR_CUDA, cudaGetErrorString(e));
        if (per_sm <= 0) return hf::set_last_error(HF_ERR_REGS, "block cannot be resident");
        grid = per_sm * sms;
    }
    hf::SingleParams<BodyBn> p;
    std::memset(&p, 0, sizeof p);   // no bulk-copy ring
    p.a = a;
    p.err = hf::error_word();
    k_bn_noalloc<<<grid, threads, smem, st>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return hf::set_last_error(HF_ERR_CUDA, cudaGetErrorString(e));
    return HF_OK;
}
