"""The source-level front-end: Algorithm 1 applied to CUDA source text
(Sec. 3.1, the transformation the paper's Clang tool performs, Sec. 3.3).

CPU tests check the rewriting and compile the result with NVRTC; GPU tests
run fused kernels and compare each constituent's output bit for bit with the
unmodified kernel launched alone on as many threads as its interval, and
with the oracle."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2007_01277_gb300 import workloads as W

H = pytest.importorskip("paper_2007_01277_gb300.hfuse")

# Three small kernels written for these tests: a block reduction with static
# shared memory and a barrier tree (its per-block partial sums depend on the
# block size, so equality with a standalone launch tests the remapping), a
# byte histogram on dynamic shared memory with two barriers, and an
# element-wise multiply-add without barriers.
SRC = r'''
extern "C" __global__ void block_sum(const float *__restrict__ x, int n, float *partial)
{
    __shared__ float part[1024];
    float s = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        s += x[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w /= 2) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = part[0];
}

__global__ void byte_hist(const unsigned char *x, long long n, unsigned *bins)
{
    extern __shared__ __align__(16) unsigned counts[];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) counts[i] = 0;
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        atomicAdd(&counts[x[i]], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (counts[i]) atomicAdd(&bins[i], counts[i]);
}
'''

SRC_AXPY = r'''
/* a different translation unit */
__device__ __forceinline__ float madd(float a, float x, float y) { return fmaf(a, x, y); }

__global__ void __launch_bounds__(1024) scale_add(const float *x, float *y, float a, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += blockDim.x * gridDim.x)
        y[i] = madd(a, x[i], y[i]);
}
'''


def test_rewrite_replaces_block_builtins():
    out = H.hf_src_fuse(SRC, "block_sum", None, "byte_hist", 256, 512)
    bodies = out[: out.index("hf_src_fused(")]
    assert "threadIdx" not in bodies and "blockDim" not in bodies
    assert "__syncthreads" not in bodies
    assert bodies.count("hf_bar_sync_(hf_bar_, hf_ntid_)") == 4
    assert "unsigned *counts = reinterpret_cast<unsigned *>(hf_dyn_);" in bodies
    assert "extern __shared__ __align__(16)" not in bodies
    tail = out[out.index("hf_src_fused("):]
    assert "threadIdx.x < 256u" in tail and "threadIdx.x - 256u, 256u, 2u" in tail
    assert "__launch_bounds__(512)" in out
    # blockIdx / gridDim pass through
    assert "blockIdx.x * hf_ntid_ + hf_tid_" in bodies and "gridDim.x * hf_ntid_" in bodies


def test_fused_source_compiles_with_nvrtc():
    for a, sa, b, sb, split, d0 in (("block_sum", SRC, "byte_hist", None, 256, 512),
                                    ("byte_hist", SRC, "scale_add", SRC_AXPY, 128, 384),
                                    ("byte_hist", SRC, "byte_hist", None, 64, 128)):
        out = H.hf_src_fuse(sa, a, sb, b, split, d0)
        H.hf_src_compile_check(out, "hf_src_fused")
        H.hf_src_compile_check(out, "hf_src_fused", 40)
    with pytest.raises(H.HFError) as e:
        H.hf_src_compile_check("__global__ void k() { undefined_call(); }", "k")
    assert e.value.status == -1


@pytest.mark.parametrize("src,why", [
    ("__global__ void k(int *p) { p[threadIdx.y] = 0; }", "1-D"),
    ("__global__ void k(int *p) { p[blockDim.z] = 0; }", "1-D"),
    ("__global__ void k(int *p) { dim3 t = threadIdx; p[t.x] = 0; }", "whole"),
    ("__global__ void k(int *p) { p[0] = __syncthreads_count(1); }", "not supported"),
    ("__device__ int tid() { return threadIdx.x; }\n__global__ void k(int *p) { p[tid()] = 0; }", "outside"),
    ("extern __shared__ float s[];\n__global__ void k(float *p) { p[0] = s[0]; }", "file-scope"),
    ("template <int N> __global__ void k(int *p) { p[0] = N; }", "templates"),
    ("#define TID threadIdx.x\n__global__ void k(int *p) { p[TID] = 0; }", "preprocessor"),
    ("#define SYNC() __syncthreads()\n__global__ void k(int *p) { SYNC(); p[0] = 0; }", "preprocessor"),
])
def test_unsupported_forms_are_rejected(src, why):
    with pytest.raises(H.HFError) as e:
        H.hf_src_fuse(src, "k", SRC, "byte_hist", 64, 128)
    assert e.value.status == -6
    assert why in str(e.value)


def test_comments_strings_and_pragmas_pass_through():
    # builtins named in comments or string literals are not code; pragmas and
    # macros without builtins are kept as they are
    src = r'''
#define SCALE 2.0f
// threadIdx.x in a comment, __syncthreads() too
__global__ void k(float *p, int n)
{
    const char *tag = "blockDim.x"; (void)tag;   /* threadIdx */
#pragma unroll 4
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] *= SCALE;
    __syncthreads();
}
'''
    out = H.hf_src_fuse(src, "k", SRC, "byte_hist", 64, 128)
    body = out[: out.index("hf_src_fused(")]
    assert "// threadIdx.x in a comment, __syncthreads() too" in body
    assert '"blockDim.x"' in body and "#pragma unroll 4" in body and "#define SCALE 2.0f" in body
    assert "i = hf_tid_" in body and "i += hf_ntid_" in body
    H.hf_src_compile_check(out, "hf_src_fused")


def test_bad_names_and_splits():
    with pytest.raises(H.HFError) as e:
        H.hf_src_fuse(SRC, "nope", None, "byte_hist", 64, 128)
    assert e.value.status == -1
    for split, d0 in ((100, 256), (0, 256), (256, 256), (64, 2048)):
        with pytest.raises(H.HFError) as e:
            H.hf_src_fuse(SRC, "block_sum", None, "byte_hist", split, d0)
        assert e.value.status == -2


# ------------------------------------------------------------------ GPU
gpu = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def _standalone(src, name, params, grid, block, dyn=0):
    m = H.hf_src_load(src, name)
    H.hf_src_launch(m, params, grid, block, dyn)
    torch.cuda.synchronize()
    H.hf_src_unload(m)


@gpu
@pytest.mark.parametrize("split,d0,grid,cap", [(256, 512, 40, 0), (128, 256, 7, 0), (512, 1024, 19, 32)])
def test_fused_block_sum_and_hist(split, d0, grid, cap):
    _need_gpu()
    dev = torch.device("cuda:0")
    x = W.poly_input(100003, seed=3)
    xb = W.hist_input(300007, seed=4)
    xd, xbd = x.to(dev), xb.to(dev)
    part = torch.zeros(grid, device=dev)
    bins = torch.zeros(256, dtype=torch.int32, device=dev)
    m = H.hf_src_fuse_load(SRC, "block_sum", None, "byte_hist", split, d0, cap)
    if cap:
        assert H.hf_src_query(m)["regs"] <= cap
    pa = H.KernelParams(xd, x.numel(), part)
    pb = H.KernelParams(xbd, ctypes.c_longlong(xb.numel()), bins)
    H.hf_src_launch_fused(m, pa, pb, grid, 0, 1024)
    torch.cuda.synchronize()
    H.hf_src_unload(m)
    # the histogram is exact
    assert np.array_equal(bins.cpu().numpy().view(np.uint32), oracle.hist256(xb.numpy()))
    # the reduction tree of each block equals the kernel run alone on
    # `split` threads with the same grid, bit for bit
    ref = torch.zeros(grid, device=dev)
    _standalone(SRC, "block_sum", H.KernelParams(xd, x.numel(), ref), grid, split)
    assert torch.equal(part, ref)
    assert abs(part.double().sum().item() - x.double().sum().item()) < 1e-3
    bins2 = torch.zeros(256, dtype=torch.int32, device=dev)
    _standalone(SRC, "byte_hist", H.KernelParams(xbd, ctypes.c_longlong(xb.numel()), bins2), grid,
                d0 - split, 1024)
    assert torch.equal(bins, bins2)


@gpu
def test_fused_across_sources_and_with_itself():
    _need_gpu()
    dev = torch.device("cuda:0")
    xb = W.hist_input(65536 * 3 + 5, seed=5).to(dev)
    x = W.poly_input(50001, seed=6).to(dev)
    y0 = W.poly_input(50001, seed=7)
    y = y0.to(dev)
    bins = torch.zeros(256, dtype=torch.int32, device=dev)
    m = H.hf_src_fuse_load(SRC, "byte_hist", SRC_AXPY, "scale_add", 128, 384)
    H.hf_src_launch_fused(m, H.KernelParams(xb, ctypes.c_longlong(xb.numel()), bins),
                          H.KernelParams(x, y, 0.75, x.numel()), 13, 1024, 0)
    torch.cuda.synchronize()
    H.hf_src_unload(m)
    assert np.array_equal(bins.cpu().numpy().view(np.uint32), oracle.hist256(xb.cpu().numpy()))
    # single rounding of a*x + y: compare with the float64 value rounded once
    ref = (0.75 * x.double().cpu() + y0.double()).float()
    assert torch.equal(y.cpu(), ref)
    # a kernel fused with itself, on two inputs
    xa = W.hist_input(70000, seed=8).to(dev)
    b1 = torch.zeros(256, dtype=torch.int32, device=dev)
    b2 = torch.zeros(256, dtype=torch.int32, device=dev)
    m = H.hf_src_fuse_load(SRC, "byte_hist", None, "byte_hist", 64, 320)
    H.hf_src_launch_fused(m, H.KernelParams(xa, ctypes.c_longlong(xa.numel()), b1),
                          H.KernelParams(xb, ctypes.c_longlong(xb.numel()), b2), 9, 1024, 1024)
    torch.cuda.synchronize()
    H.hf_src_unload(m)
    assert np.array_equal(b1.cpu().numpy().view(np.uint32), oracle.hist256(xa.cpu().numpy()))
    assert np.array_equal(b2.cpu().numpy().view(np.uint32), oracle.hist256(xb.cpu().numpy()))


@gpu
def test_launch_validation():
    _need_gpu()
    m = H.hf_src_load(SRC, "block_sum")
    assert H.hf_src_query(m)["max_threads"] >= 256
    x = torch.zeros(16, device="cuda")
    with pytest.raises(H.HFError):
        H.hf_src_launch(m, H.KernelParams(x, 16, x), 1, 2048)
    with pytest.raises(H.HFError):
        H.hf_src_launch(m, H.KernelParams(x, 16, x), 0, 256)
    with pytest.raises(H.HFError):   # a single module is not a fused one
        H.hf_src_launch_fused(m, H.KernelParams(), H.KernelParams(), 1)
    H.hf_src_unload(m)
