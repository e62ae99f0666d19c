"""Parity at the benchmark's full sizes, in the launch configurations bench.py
times, on outputs the oracle can compute one slice at a time."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from gpu_util import DEV, bits16, check_bn, check_poly, check_upsample  # noqa: E402
from paper_2007_01277_gb300 import hfuse as H  # noqa: E402
from paper_2007_01277_gb300 import workloads as W  # noqa: E402

def grid(bps):
    return bps * H.hf_device_info().sm_count


def test_upsample_maxpool_full_size_bench_config():
    """32x64x128x128 upsample + 32x128x112x112 max pool, split 256/256, cap 64,
    2 blocks/SM (the configuration the default benchmark selects)."""
    xu = W.upsample_input((32, 64, 128, 128))
    xp = W.maxpool_input((32, 128, 112, 112))
    xud, xpd = xu.to(DEV), xp.to(DEV)
    yu = torch.empty(32, 64, 256, 256, device=DEV)
    yp = torch.empty(32, 128, 56, 56, device=DEV)
    f = H.hf_fuse(H.hf_register_kernel(H.UPSAMPLE2X), H.hf_register_kernel(H.MAXPOOL3S2), 256, 512, 64)
    H.hf_launch(f, [H.upsample2x_args(xud, yu), H.maxpool3s2_args(xpd, yp)], grid(2))
    torch.cuda.synchronize()
    for n, c in [(0, 0), (5, 17), (31, 63), (16, 40)]:
        check_upsample(xu[n, c], yu[n, c])
    for n in (0, 13, 31):
        np.testing.assert_array_equal(yp[n].cpu().numpy(), oracle.maxpool3s2p1(xp[n].numpy()))


def test_hist_philox_full_size_bench_config():
    """2^28-byte histogram + 2^26 Philox blocks, split 128/128 of 256, cap 64,
    2 blocks/SM: every bin, and Philox blocks at sampled counters."""
    xh = W.hist_input(1 << 28)
    xhd = xh.to(DEV)
    bins = torch.zeros(256, dtype=torch.int32, device=DEV)
    po = torch.empty((1 << 26, 4), dtype=torch.int32, device=DEV)
    f = H.hf_fuse(H.hf_register_kernel(H.HIST256), H.hf_register_kernel(H.PHILOX), 128, 256, 64)
    H.hf_launch(f, [H.hist256_args(xhd, bins), H.philox_args(po, 0)], grid(2))
    torch.cuda.synchronize()
    ref = oracle.hist256(xh.numpy())
    assert np.array_equal(bins.cpu().numpy().view(np.uint32), ref)
    assert int(ref.sum()) == 1 << 28
    out = po.cpu().numpy().view(np.uint32)
    rng = np.random.default_rng(0)
    for i in list(rng.integers(0, 1 << 26, 64)) + [0, (1 << 26) - 1]:
        np.testing.assert_array_equal(out[i], oracle.philox4x32_10(0, 1, first=int(i))[0])


def test_bn_poly_full_size_bench_config():
    """8x64x32x32 batch-norm statistics + 2^20-element polynomial chain, split
    256/256 under a 40-register cap, resident grid."""
    x = W.bn_input((8, 64, 32, 32))
    px = W.poly_input(1 << 20)
    coef = W.poly_coefficients().numpy()
    xd, pxd = x.to(DEV), px.to(DEV)
    m, v, py = torch.empty(64, device=DEV), torch.empty(64, device=DEV), torch.empty_like(pxd)
    f = H.hf_fuse(H.hf_register_kernel(H.BN_STATS), H.hf_register_kernel(H.POLY), 256, 512, 40)
    H.hf_launch(f, [H.bn_stats_args(xd, m, v, H.bn_stats_workspace(xd)), H.poly_args(pxd, py, coef)], 0)
    torch.cuda.synchronize()
    check_bn(x, m, v)
    idx = np.random.default_rng(1).integers(0, 1 << 20, 4096)
    check_poly(px[idx], coef, py.cpu()[idx])


def test_nway8_full_size_converged_plan():
    """The eight kernels at the N-way workload's sizes in the plan the
    autotuner converges to; every kernel checked on slices."""
    sp = W.WORKLOADS["nway8"]
    xb = W.bn_input(sp["bn"])
    xi = W.im2col_input(sp["im2col"])
    xp = W.maxpool_input(sp["pool"])
    xu = W.upsample_input(sp["up"])
    xh = W.hist_input(sp["hist_n"])
    xq = W.poly_input(sp["poly_n"])
    x16, y16 = W.bf16_inputs(sp["bf16_n"])
    coef = W.poly_coefficients().numpy()
    d = {k: t.to(DEV) for k, t in dict(xb=xb, xi=xi, xp=xp, xu=xu, xh=xh, xq=xq, x16=x16, y16=y16).items()}
    mb, vb = torch.empty(256, device=DEV), torch.empty(256, device=DEV)
    ci = torch.empty(32, 576, 3136, device=DEV)
    yp = torch.empty(32, 128, 56, 56, device=DEV)
    yu = torch.empty(32, 64, 256, 256, device=DEV)
    bins = torch.zeros(256, dtype=torch.int32, device=DEV)
    po = torch.empty((sp["philox_n"], 4), dtype=torch.int32, device=DEV)
    yq = torch.empty_like(d["xq"])
    o16 = torch.empty_like(d["x16"])
    args = [H.bn_stats_args(d["xb"], mb, vb, H.bn_stats_workspace(d["xb"])), H.im2col3_args(d["xi"], ci),
            H.maxpool3s2_args(d["xp"], yp), H.upsample2x_args(d["xu"], yu), H.hist256_args(d["xh"], bins),
            H.philox_args(po, 0), H.poly_args(d["xq"], yq, coef), H.bf16_axpy_args(d["x16"], d["y16"], o16)]
    ks = [H.hf_register_kernel(b) for b in (H.BN_STATS, H.IM2COL3, H.MAXPOOL3S2, H.UPSAMPLE2X,
                                            H.HIST256, H.PHILOX, H.POLY, H.BF16_AXPY)]
    f = H.hf_fuse_n(ks, [3, 3, 2, 1, 3, 1, 0, 2], [128, 288, 352, 256], 48)
    H.hf_launch(f, args, 0)
    torch.cuda.synchronize()
    # batch-norm: channels checked with the oracle on their slice
    mean, var = mb.cpu(), vb.cpu()
    for c in (0, 77, 255):
        check_bn(xb[:, c:c + 1], mean[c:c + 1], var[c:c + 1])
    for n, c in [(0, 0), (31, 63)]:
        np.testing.assert_array_equal(ci[n, 9 * c:9 * c + 9].cpu().numpy(),
                                      oracle.im2col3(xi[n:n + 1, c:c + 1].numpy())[0])
        np.testing.assert_array_equal(yp[n, c].cpu().numpy(), oracle.maxpool3s2p1(xp[n, c].numpy()))
        check_upsample(xu[n, c], yu[n, c])
    ref = oracle.hist256(xh.numpy())
    assert np.array_equal(bins.cpu().numpy().view(np.uint32), ref)
    out = po.cpu().numpy().view(np.uint32)
    for i in (0, 12345, sp["philox_n"] - 1):
        np.testing.assert_array_equal(out[i], oracle.philox4x32_10(0, 1, first=i)[0])
    idx = np.random.default_rng(2).integers(0, sp["poly_n"], 2048)
    check_poly(xq[idx], coef, yq.cpu()[idx])
    sl = slice(0, 1 << 16)
    ref16 = oracle.bf16_axpy(bits16(x16[sl]), bits16(y16[sl]), 0.5)
    assert np.array_equal(bits16(o16[sl]), ref16)
    tail = slice(sp["bf16_n"] - 4096, sp["bf16_n"])
    assert np.array_equal(bits16(o16[tail]), oracle.bf16_axpy(bits16(x16[tail]), bits16(y16[tail]), 0.5))


def test_hash_pair_full_size_bench_config():
    """SHA-256d over 2^24 nonces + BLAKE2b over 21*2^20 nonces fused at
    384/128 of 512 under a 64-register cap, 2 blocks/SM: sampled digests
    against the oracle, every stored hit re-hashed by the oracle, and the hit
    count equal to the number of digests that pass the test."""
    hp = W.WORKLOADS["hash_pairs"]
    specs = [(H.SHA256D, hp["sha256d_n"], oracle.sha256d_scan, W.hash_header(0)),
             (H.BLAKE2B, hp["blake2b_n"], oracle.blake2b_scan, W.hash_header(1))]
    bufs, args = [], []
    for body, n, _, hdr in specs:
        dig = torch.empty(n * 32, dtype=torch.uint8, device=DEV)
        hits = torch.full((1 << 12,), -1, dtype=torch.int32, device=DEV)
        cnt = torch.zeros(1, dtype=torch.int32, device=DEV)
        bufs.append((dig, hits, cnt))
        args.append(H.hash_scan_args(hdr, n, 0, hp["target"], dig, hits, cnt))
    f = H.hf_fuse(H.hf_register_kernel(H.SHA256D), H.hf_register_kernel(H.BLAKE2B), 384, 512, 64)
    H.hf_launch(f, args, grid(2))
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    for (body, n, scan, hdr), (dig, hits, cnt) in zip(specs, bufs):
        d = dig.cpu().numpy().reshape(n, 32)
        for i in [0, n - 1] + list(rng.integers(0, n, 200)):
            assert np.array_equal(d[i], scan(hdr, int(i), 1)[0]), (H.BODY_NAMES[body], i)
        count = int(cnt.item())
        assert count == oracle.hash_hits(d, 0, hp["target"]).size > 0
        stored = hits.cpu().numpy().view(np.uint32)[: min(count, hits.numel())]
        for nonce in stored:
            ref = scan(hdr, int(nonce), 1)
            assert oracle.hash_hits(ref, int(nonce), hp["target"]).tolist() == [nonce]
