"""The checked build of the fused pairs (hf_fuse_checked): every interval
barrier of Sec. 3.1 is a bounded software barrier over the interval's warps.
Run on the pairs whose bodies synchronise (histogram + Philox, batch-norm +
histogram, batch-norm + polynomial, two stream templates with four barriers
per tile): the results match the oracle and the production fused kernel bit
for bit, and the device error word stays clear, i.e. no barrier wait ever
expired.  (A barrier made to miss its count is covered by the software
barrier's own self-test.)"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from gpu_util import DEV, check_bn, check_poly, check_stream  # noqa: E402
from paper_2007_01277_gb300 import hfuse as H  # noqa: E402
from paper_2007_01277_gb300 import workloads as W  # noqa: E402


def _both(ka, kb, split, d0, args, grid, reset, outputs):
    """Outputs of the production and the checked fused kernel."""
    res = []
    for fuse in (lambda: H.hf_fuse(ka, kb, split, d0, 0), lambda: H.hf_fuse_checked(ka, kb, split, d0)):
        f = fuse()
        reset()
        H.hf_launch(f, args, grid)
        torch.cuda.synchronize()
        res.append([t.clone() for t in outputs])
        H.hf_destroy_fused(f)
    assert H.hf_check_device_error(clear=True) == 0
    for a, b in zip(*res):
        assert torch.equal(a, b)
    return res[1]


@pytest.mark.parametrize("split,d0,grid", [(128, 256, 0), (64, 256, 7), (192, 256, 152), (256, 512, 0)])
def test_hist_philox_checked(split, d0, grid):
    xh = W.hist_input((1 << 20) + 77, seed=5).to(DEV)
    bins = torch.zeros(256, dtype=torch.int32, device=DEV)
    po = torch.empty(((1 << 14) + 3, 4), dtype=torch.int32, device=DEV)
    kh, kx = H.hf_register_kernel(H.HIST256), H.hf_register_kernel(H.PHILOX)
    args = [H.hist256_args(xh, bins), H.philox_args(po, 11)]
    b, p = _both(kh, kx, split, d0, args, grid, bins.zero_, [bins, po])
    assert np.array_equal(b.cpu().numpy().view(np.uint32), oracle.hist256(xh.cpu().numpy()))
    assert np.array_equal(p.cpu().numpy().view(np.uint32), oracle.philox4x32_10(11, po.shape[0]))


@pytest.mark.parametrize("split,d0,grid", [(256, 512, 0), (384, 512, 19), (128, 256, 0)])
def test_bn_hist_checked(split, d0, grid):
    x = W.bn_input((4, 16, 24, 24), seed=6)
    xd = x.to(DEV)
    m, v = torch.empty(16, device=DEV), torch.empty(16, device=DEV)
    xh = W.hist_input(300000, seed=7).to(DEV)
    bins = torch.zeros(256, dtype=torch.int32, device=DEV)
    kb, kh = H.hf_register_kernel(H.BN_STATS), H.hf_register_kernel(H.HIST256)
    args = [H.bn_stats_args(xd, m, v, H.bn_stats_workspace(xd)), H.hist256_args(xh, bins)]
    mm, vv, b = _both(kb, kh, split, d0, args, grid, bins.zero_, [m, v, bins])
    check_bn(x, mm, vv)
    assert np.array_equal(b.cpu().numpy().view(np.uint32), oracle.hist256(xh.cpu().numpy()))


def test_bn_poly_checked():
    x = W.bn_input((8, 64, 32, 32))
    xd = x.to(DEV)
    px = W.poly_input(1 << 15)
    pxd = px.to(DEV)
    coef = W.poly_coefficients().numpy()
    m, v, y = torch.empty(64, device=DEV), torch.empty(64, device=DEV), torch.empty_like(pxd)
    kb, kp = H.hf_register_kernel(H.BN_STATS), H.hf_register_kernel(H.POLY)
    args = [H.bn_stats_args(xd, m, v, H.bn_stats_workspace(xd)), H.poly_args(pxd, y, coef)]
    mm, vv, yy = _both(kb, kp, 256, 512, args, 0, lambda: None, [m, v, y])
    check_bn(x, mm, vv)
    check_poly(px, coef, yy)


@pytest.mark.parametrize("nb,smem", [(4, 8192), (1, 0), (3, 49152)])
def test_stream_templates_with_barriers_checked(nb, smem):
    xa = W.template_input(1 << 16, seed=21)
    xb = W.template_input(3 << 14, seed=22)
    xad, xbd = xa.to(DEV), xb.to(DEV)
    ya, yb = torch.empty_like(xad), torch.empty_like(xbd)
    k1, k2 = H.hf_register_kernel(H.STREAM_TMPL), H.hf_register_kernel(H.STREAM_TMPL)
    args = [H.stream_tmpl_args(xad, ya, 8, nb, smem), H.stream_tmpl_args(xbd, yb, 2, 4, 4096)]
    a, b = _both(k1, k2, 96, 256, args, 0, lambda: None, [ya, yb])
    check_stream(xa, a, 8, 0.999, 0.001)
    check_stream(xb, b, 2, 0.999, 0.001)


def test_checked_build_covers_only_pairs_with_barriers():
    ku, kp = H.hf_register_kernel(H.UPSAMPLE2X), H.hf_register_kernel(H.MAXPOOL3S2)
    with pytest.raises(H.HFError, match="UNSUPPORTED"):
        H.hf_fuse_checked(ku, kp, 256, 512)
    # the checked instance reports its resources like any other
    kh, kx = H.hf_register_kernel(H.HIST256), H.hf_register_kernel(H.PHILOX)
    f = H.hf_fuse_checked(kx, kh, 64, 256)
    xh = torch.zeros(1024, dtype=torch.uint8, device=DEV)
    bins = torch.zeros(256, dtype=torch.int32, device=DEV)
    po = torch.empty((64, 4), dtype=torch.int32, device=DEV)
    info = H.hf_query(f, [H.philox_args(po, 0), H.hist256_args(xh, bins)])
    assert info["blocks_per_sm"] >= 1 and info["regs"] > 0
    H.hf_destroy_fused(f)
