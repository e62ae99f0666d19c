"""Sizes past 32-bit indexing: every body on inputs or outputs of more than
2^31 elements (or 2^32 bytes), against the oracle.

The benchmark's workloads stay below 2^31 elements per tensor, so an index
computed in 32 bits would pass every other test.  Here each body runs once
at a size whose element (or byte) offsets cross 2^31 (2^32 for bytes), one
fused launch too, and the oracle checks the whole result where it is
integer-only and cheap on the CPU (the histogram, batch-norm), else the
planes, channels or index ranges on both sides of the 32-bit boundaries and
at the end.  Inputs are drawn by the device's seeded generator (several GB
each) and copied back for the oracle.  Device memory held at once: at most
about 17 GB.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from gpu_util import DEV, bits16, check_poly, single  # noqa: E402
from paper_2007_01277_gb300 import hfuse as H  # noqa: E402
from paper_2007_01277_gb300 import workloads as W  # noqa: E402

B31 = 1 << 31


@pytest.fixture(autouse=True)
def _release():
    yield
    torch.cuda.synchronize()
    assert H.hf_check_device_error() == 0
    torch.cuda.empty_cache()


def _ranges(n, marks, width=256):
    """[lo, hi) windows of `width` around each mark, clipped to [0, n)."""
    return [(max(0, m - width // 2), min(n, m + width // 2)) for m in marks]


def test_hist_past_4_gib():
    n = (1 << 32) + 4099
    x = W.bytes_u8(n, 21, device=DEV)
    bins = torch.zeros(256, dtype=torch.int32, device=DEV)
    single(H.HIST256, H.hist256_args(x, bins), 256, 0)
    torch.cuda.synchronize()
    got = bins.cpu().numpy().view(np.uint32)
    ref = oracle.hist256(x.cpu().numpy())
    assert np.array_equal(got, ref)
    assert int(got.astype(np.uint64).sum()) == n


def test_philox_past_4_gib_and_fused_with_hist():
    n = (1 << 28) + 3                      # 16-byte blocks: byte offsets past 2^32
    out = torch.empty((n, 4), dtype=torch.int32, device=DEV)
    single(H.PHILOX, H.philox_args(out, 0x5EED, 11), 256, 0)
    torch.cuda.synchronize()
    # block 2^27 starts at byte 2^31, block 2^28 at byte 2^32
    for lo, hi in _ranges(n, [0, 1 << 27, 1 << 28, n]):
        ref = oracle.philox4x32_10(0x5EED, hi - lo, first=11 + lo)
        assert np.array_equal(out[lo:hi].cpu().numpy().view(np.uint32), ref), (lo, hi)
    # the same sizes in one fused launch: bit-identical to the launches alone
    x = W.bytes_u8((1 << 32) + 77, 22, device=DEV)
    bins_ref = torch.zeros(256, dtype=torch.int32, device=DEV)
    single(H.HIST256, H.hist256_args(x, bins_ref), 256, 0)
    kh, kp = H.hf_register_kernel(H.HIST256), H.hf_register_kernel(H.PHILOX)
    f = H.hf_fuse(kh, kp, 128, 256, 0)
    bins = torch.zeros(256, dtype=torch.int32, device=DEV)
    out2 = torch.empty_like(out)
    H.hf_launch(f, [H.hist256_args(x, bins), H.philox_args(out2, 0x5EED, 11)], 0)
    torch.cuda.synchronize()
    assert torch.equal(bins, bins_ref) and torch.equal(out2, out)
    H.hf_destroy_fused(f)


def test_upsample_past_2g_output_elements():
    P = 32769                               # output plane 32768 starts at element 2^31
    x = W.uniform((P, 1, 128, 128), 0.0, 1.0, 23, device=DEV)
    y = torch.empty((P, 1, 256, 256), device=DEV)
    single(H.UPSAMPLE2X, H.upsample2x_args(x, y), 128, 0)
    torch.cuda.synchronize()
    planes = [0, 16383, 16384, 32767, 32768]
    ref = oracle.upsample2x(x[planes].cpu().numpy())
    got = y[planes].double().cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-5 * np.abs(ref) + 1e-30), np.max(np.abs(got - ref))


def test_maxpool_past_2g_input_elements():
    P = (1 << 17) + 1                       # input plane 2^17 starts at element 2^31
    x = W.normal((P, 1, 128, 128), 24, device=DEV)
    y = torch.empty((P, 1, 64, 64), device=DEV)
    single(H.MAXPOOL3S2, H.maxpool3s2_args(x, y), 256, 0)
    torch.cuda.synchronize()
    planes = [0, (1 << 17) - 1, 1 << 17]
    assert np.array_equal(y[planes].cpu().numpy(), oracle.maxpool3s2p1(x[planes].cpu().numpy()))


def test_im2col_past_2g_output_elements():
    C = 76200                               # 685,800 rows of 3136: 2,150,668,800 elements
    x = W.normal((1, C, 56, 56), 25, device=DEV)
    col = torch.empty((1, 9 * C, 56 * 56), device=DEV)
    single(H.IM2COL3, H.im2col3_args(x, col), 256, 0)
    torch.cuda.synchronize()
    # channel 76090's rows start past element 2^31
    for c in (0, 76089, 76090, C - 1):
        ref = oracle.im2col3(x[:, c:c + 1].cpu().numpy())
        assert np.array_equal(col[:, 9 * c: 9 * c + 9].cpu().numpy(), ref), c


def test_bn_stats_past_2g_elements():
    shape = (16385, 4, 128, 256)            # 2,147,614,720 values
    x = W.normal(shape, 26, device=DEV)
    mean, var = torch.empty(4, device=DEV), torch.empty(4, device=DEV)
    single(H.BN_STATS, H.bn_stats_args(x, mean, var, H.bn_stats_workspace(x)), 256, 0)
    torch.cuda.synchronize()
    xc = x.cpu().numpy()
    del x
    m_ref, v_ref = oracle.bn_stats(xc)
    scale = np.array([np.abs(xc[:, c]).mean(dtype=np.float64) for c in range(4)])
    m, v = mean.double().cpu().numpy(), var.double().cpu().numpy()
    assert np.all(np.abs(m - m_ref) <= 1e-5 * scale), np.abs(m - m_ref) / scale
    assert np.all(np.abs(v - v_ref) <= 1e-4 * v_ref), np.abs(v - v_ref) / v_ref


def test_poly_past_2g_elements():
    n = B31 + 100
    x = W.uniform((n,), -1.0, 1.0, 27, device=DEV)
    y = torch.empty_like(x)
    coef = W.poly_coefficients().tolist()
    single(H.POLY, H.poly_args(x, y, coef, iters=1), 256, 0)
    torch.cuda.synchronize()
    for lo, hi in _ranges(n, [0, B31, n], 512):
        check_poly(x[lo:hi].cpu(), coef, y[lo:hi], iters=1)


def test_bf16_axpy_past_2g_elements():
    n = B31 + 100
    xs = W.uniform((n,), -1.0, 1.0, 28, device=DEV).to(torch.bfloat16)
    ys = W.uniform((n,), -1.0, 1.0, 29, device=DEV).to(torch.bfloat16)
    out = torch.empty_like(xs)
    single(H.BF16_AXPY, H.bf16_axpy_args(xs, ys, out, 0.5), 256, 0)
    torch.cuda.synchronize()
    for lo, hi in _ranges(n, [0, B31, n], 512):
        ref = oracle.bf16_axpy(bits16(xs[lo:hi]), bits16(ys[lo:hi]), 0.5)
        diff = np.abs(bits16(out[lo:hi]).astype(np.int32) - ref.astype(np.int32))
        assert np.all(diff <= 1), (lo, diff.max())
