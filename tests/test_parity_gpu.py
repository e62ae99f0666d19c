"""GPU parity: every body launched alone against the FP64/exact oracle, and
every fused launch bit-identical to its bodies launched alone with the same
interval size and grid (the functional equivalence of Sec. 1.1 / Sec. 3.1),
all through the C ABI."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from gpu_util import (DEV, check_bf16, check_bn, check_poly, check_stream,  # noqa: E402
                      check_upsample, single)
from paper_2007_01277_gb300 import hfuse as H  # noqa: E402
from paper_2007_01277_gb300 import workloads as W  # noqa: E402


# ------------------------------------------------------------------ standalone vs oracle
@pytest.mark.parametrize("shape", [(2, 8, 16, 12), (3, 5, 7, 9), (8, 4, 40, 40), (8, 64, 32, 32),
                                   (1, 1, 1, 4), (5, 3, 1, 2050), (3, 5, 56, 56), (2, 3, 33, 36),
                                   (1, 2, 64, 64)])
@pytest.mark.parametrize("threads,grid", [(256, 0), (64, 3), (1024, 1)])
def test_bn_stats(shape, threads, grid):
    x = W.bn_input(shape, seed=sum(shape))
    xd = x.to(DEV)
    C = shape[1]
    mean = torch.empty(C, device=DEV)
    var = torch.empty(C, device=DEV)
    ws = H.bn_stats_workspace(xd)
    single(H.BN_STATS, H.bn_stats_args(xd, mean, var, ws), threads, grid)
    torch.cuda.synchronize()
    check_bn(x, mean, var)
    # the workspace is left clean: a second launch gives the same bits
    m2, v2 = torch.empty_like(mean), torch.empty_like(var)
    single(H.BN_STATS, H.bn_stats_args(xd, m2, v2, ws), threads, grid)
    torch.cuda.synchronize()
    assert torch.equal(mean, m2) and torch.equal(var, v2)


@pytest.mark.parametrize("shape", [(3, 5, 56, 56), (8, 64, 32, 32), (2, 3, 33, 36)])
def test_bn_bits_independent_of_launch(shape):
    """Each 2048-value tile is reduced by one warp in a fixed order and the
    tiles combine in tile order, so every launch configuration gives the
    same bits."""
    x = W.bn_input(shape, seed=7).to(DEV)
    C = shape[1]
    ws = H.bn_stats_workspace(x)
    outs = []
    for threads, grid in ((256, 0), (64, 3), (1024, 1), (128, 40), (32, 152)):
        m, v = torch.empty(C, device=DEV), torch.empty(C, device=DEV)
        single(H.BN_STATS, H.bn_stats_args(x, m, v, ws), threads, grid)
        torch.cuda.synchronize()
        outs.append((m, v))
    assert H.hf_check_device_error() == 0
    for m, v in outs[1:]:
        assert torch.equal(m, outs[0][0]) and torch.equal(v, outs[0][1])


def test_bn_workspace_counters_rearmed_after_launch():
    """Every channel's counter is zeroed by its combine, so the counter
    region is zero after each launch -- also with more blocks than can be
    resident at once and with blocks that get no tile -- and the bits do
    not depend on the launch."""
    x = W.bn_input((4, 6, 40, 40), seed=11).to(DEV)
    ws = H.bn_stats_workspace(x)
    ref = None
    for threads, grid in ((128, 4000), (1024, 1), (32, 700), (256, 0)):
        m, v = torch.empty(6, device=DEV), torch.empty(6, device=DEV)
        single(H.BN_STATS, H.bn_stats_args(x, m, v, ws), threads, grid)
        torch.cuda.synchronize()
        assert not ws[:256].any(), (threads, grid)   # 6 counters, padded to 256 B
        if ref is None:
            ref = (m, v)
            check_bn(x.cpu(), m, v)
        assert torch.equal(m, ref[0]) and torch.equal(v, ref[1])
    assert H.hf_check_device_error() == 0


def test_bn_offset_mean_and_constant_channel():
    x = W.bn_input((4, 3, 8, 8)) * 0.01 + 1000.0
    x[:, 1] = 7.25
    xd = x.to(DEV)
    mean, var = torch.empty(3, device=DEV), torch.empty(3, device=DEV)
    single(H.BN_STATS, H.bn_stats_args(xd, mean, var, H.bn_stats_workspace(xd)), 128, 2)
    torch.cuda.synchronize()
    check_bn(x, mean, var)
    assert var[1].item() == 0.0 and mean[1].item() == 7.25


@pytest.mark.parametrize("shape", [(2, 3, 20, 24), (1, 2, 9, 7), (2, 2, 128, 128), (1, 1, 10, 260),
                                   (1, 1, 1, 1), (3, 1, 17, 4), (2, 3, 37, 36), (1, 1, 1, 128)])
@pytest.mark.parametrize("threads,grid", [(256, 0), (96, 5), (512, 3), (32, 1)])
def test_upsample(shape, threads, grid):
    x = W.upsample_input(shape, seed=sum(shape))
    xd = x.to(DEV)
    y = torch.empty(shape[:-2] + (2 * shape[-2], 2 * shape[-1]), device=DEV)
    single(H.UPSAMPLE2X, H.upsample2x_args(xd, y), threads, grid)
    torch.cuda.synchronize()
    assert H.hf_check_device_error() == 0
    check_upsample(x, y)


@pytest.mark.parametrize("shape", [(2, 3, 20, 24), (2, 2, 128, 128), (1, 1, 10, 260)])
def test_upsample_output_alignments(shape):
    # outputs at byte offsets 0 and 16 take the 128-bit vector path, at 4
    # the scalar one; all give the same bits and write nothing outside y
    x = W.upsample_input(shape, seed=3)
    xd = x.to(DEV)
    n = x.numel() * 4
    outs = []
    for off in (0, 4, 1):
        buf = torch.full((n + 8,), float("nan"), device=DEV)
        y = buf[off: off + n].view(shape[:-2] + (2 * shape[-2], 2 * shape[-1]))
        single(H.UPSAMPLE2X, H.upsample2x_args(xd, y), 256, 7)
        torch.cuda.synchronize()
        assert H.hf_check_device_error() == 0
        check_upsample(x, y)
        rest = torch.cat([buf[:off], buf[off + n:]])
        assert torch.isnan(rest).all()   # nothing written outside y
        outs.append(y.clone())
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


@pytest.mark.parametrize("shape", [(2, 3, 20, 24), (1, 2, 9, 7), (2, 4, 112, 112), (1, 1, 11, 264),
                                   (1, 1, 1, 1), (2, 1, 2, 4), (3, 2, 37, 36), (1, 3, 57, 128),
                                   (1, 1, 1, 8), (2, 1, 3, 4)])
@pytest.mark.parametrize("threads,grid", [(256, 0), (96, 5), (768, 3), (32, 1)])
def test_maxpool(shape, threads, grid):
    x = W.maxpool_input(shape, seed=sum(shape))
    xd = x.to(DEV)
    H_, W_ = shape[-2:]
    y = torch.empty(shape[:-2] + ((H_ - 1) // 2 + 1, (W_ - 1) // 2 + 1), device=DEV)
    single(H.MAXPOOL3S2, H.maxpool3s2_args(xd, y), threads, grid)
    torch.cuda.synchronize()
    assert H.hf_check_device_error() == 0
    assert np.array_equal(y.cpu().numpy(), oracle.maxpool3s2p1(x.numpy()))


@pytest.mark.parametrize("shape", [(2, 3, 10, 12), (1, 2, 9, 7), (2, 4, 56, 56), (1, 2, 5, 68),
                                   (1, 1, 1, 4), (2, 2, 3, 64)])
@pytest.mark.parametrize("threads,grid", [(256, 0), (64, 7)])
def test_im2col(shape, threads, grid):
    x = W.im2col_input(shape, seed=sum(shape))
    xd = x.to(DEV)
    N, C, H_, W_ = shape
    col = torch.full((N, C * 9, H_ * W_), float("nan"), device=DEV)
    single(H.IM2COL3, H.im2col3_args(xd, col), threads, grid)
    torch.cuda.synchronize()
    assert np.array_equal(col.cpu().numpy(), oracle.im2col3(x.numpy()))


@pytest.mark.parametrize("shape", [(2, 4, 56, 56), (1, 3, 57, 60), (3, 2, 7, 64)])
def test_im2col_row_chunks(shape):
    # the grid decides how many row chunks a plane is cut into (whole planes
    # for a single warp, down to one row per half-warp for many): every
    # chunking writes every element exactly once, bit-exact
    x = W.im2col_input(shape, seed=sum(shape) + 1)
    xd = x.to(DEV)
    N, C, H_, W_ = shape
    ref = oracle.im2col3(x.numpy())
    for threads, grid in ((32, 1), (64, 40), (256, 0), (768, 3)):
        col = torch.full((N, C * 9, H_ * W_), float("nan"), device=DEV)
        single(H.IM2COL3, H.im2col3_args(xd, col), threads, grid)
        torch.cuda.synchronize()
        assert np.array_equal(col.cpu().numpy(), ref), (threads, grid)


@pytest.mark.parametrize("n,offset", [(0, 0), (1, 0), (15, 0), (16, 0), (17, 0), (1000003, 0),
                                      (100000, 1), (5 << 20, 0)])
@pytest.mark.parametrize("threads,grid", [(256, 0), (128, 3), (1024, 5)])
def test_hist(n, offset, threads, grid):
    x = W.hist_input(n + offset, seed=n)
    xd = x.to(DEV)[offset:]
    bins = torch.zeros(256, dtype=torch.int32, device=DEV)
    single(H.HIST256, H.hist256_args(xd, bins), threads, grid)
    torch.cuda.synchronize()
    assert H.hf_check_device_error() == 0
    ref = oracle.hist256(x.numpy()[offset:])
    assert np.array_equal(bins.cpu().numpy().view(np.uint32), ref)


@pytest.mark.parametrize("n,seed,first", [(1, 0, 0), (3, 0, 0), (1000, 0, 0),
                                          (4097, 0x0123456789ABCDEF, 0), (300, 7, (1 << 32) - 150)])
@pytest.mark.parametrize("threads,grid", [(256, 0), (32, 3)])
def test_philox(n, seed, first, threads, grid):
    out = torch.empty((n, 4), dtype=torch.int32, device=DEV)
    single(H.PHILOX, H.philox_args(out, seed, first), threads, grid)
    torch.cuda.synchronize()
    ref = oracle.philox4x32_10(seed, n, first=first)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), ref)


@pytest.mark.parametrize("n", [1, 2, 7, 4097])
def test_philox_output_alignments(n):
    # output at byte offsets 0 and 16 (a 16-byte but not 32-byte aligned
    # start): the same blocks, and nothing written outside the output
    ref = oracle.philox4x32_10(5, n, first=3)
    for off in (0, 1):
        buf = torch.full((n + 2, 4), -1, dtype=torch.int32, device=DEV)
        out = buf[off: off + n]
        single(H.PHILOX, H.philox_args(out, 5, 3), 64, 3)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), ref)
        rest = torch.cat([buf[:off], buf[off + n:]])
        assert (rest == -1).all()


@pytest.mark.parametrize("n,offset,iters", [(1, 0, 64), (5, 0, 64), (4099, 0, 64), (1000, 1, 64),
                                            (257, 0, 1), (64, 0, 0)])
@pytest.mark.parametrize("threads,grid", [(256, 0), (64, 3)])
def test_poly(n, offset, iters, threads, grid):
    x = W.poly_input(n + offset, seed=n)
    coef = W.poly_coefficients().numpy()
    xd = x.to(DEV)[offset:]
    y = torch.empty(n + offset, device=DEV)[offset:]
    single(H.POLY, H.poly_args(xd, y, coef, iters), threads, grid)
    torch.cuda.synchronize()
    check_poly(x[offset:], coef, y, iters)


@pytest.mark.parametrize("n", [63, 64, 65, 130, 64 * 37 + 5])
def test_poly_units_bits_independent_of_launch(n):
    """64-element warp units in a block-interleaved order: every element is
    computed exactly once whatever the grid (more warps than units, fewer,
    uneven counts, a partial last unit), with the same bits."""
    x = W.poly_input(n + 2, seed=n)
    coef = W.poly_coefficients().numpy()
    xd = x.to(DEV)
    ref = None
    for threads, grid in ((32, 1), (96, 7), (1024, 152), (64, 300), (256, 0)):
        buf = torch.full((n + 2,), float("nan"), device=DEV)
        single(H.POLY, H.poly_args(xd[1: n + 1], buf[1: n + 1], coef, 8), threads, grid)
        torch.cuda.synchronize()
        assert torch.isnan(buf[0]) and torch.isnan(buf[n + 1])   # nothing outside y
        y = buf[1: n + 1].clone()
        if ref is None:
            ref = y
            check_poly(x[1: n + 1], coef, y, 8)
        assert torch.equal(y, ref), (threads, grid)


@pytest.mark.parametrize("n,offset", [(1, 0), (9, 0), (100003, 0), (4096, 1), ((1 << 21) + 40, 0)])
@pytest.mark.parametrize("threads,grid", [(256, 0), (64, 3), (1024, 2)])
def test_bf16_axpy(n, offset, threads, grid):
    x, y = W.bf16_inputs(n + offset, seed=n)
    xd, yd = x.to(DEV)[offset:], y.to(DEV)[offset:]
    out = torch.empty(n + offset, dtype=torch.bfloat16, device=DEV)[offset:]
    single(H.BF16_AXPY, H.bf16_axpy_args(xd, yd, out, 0.5), threads, grid)
    torch.cuda.synchronize()
    assert H.hf_check_device_error() == 0
    assert check_bf16(x[offset:], y[offset:], out) == 0


@pytest.mark.parametrize("k,nbar,smem", [(0, 0, 0), (1, 1, 0), (3, 2, 4096), (8, 4, 16384),
                                         (65, 3, 48 * 1024), (256, 1, 0)])
def test_stream_template(k, nbar, smem):
    n = 4 * 1001
    x = W.template_input(n, seed=k)
    xd = x.to(DEV)
    y = torch.empty_like(xd)
    single(H.STREAM_TMPL, H.stream_tmpl_args(xd, y, k, nbar, smem, 0.999, 0.001), 128, 5)
    torch.cuda.synchronize()
    check_stream(x, y, k, 0.999, 0.001)


def test_invalid_args_rejected_before_launch():
    x = torch.zeros(8, device=DEV)
    k = H.hf_register_kernel(H.STREAM_TMPL)
    with pytest.raises(H.HFError) as e:                       # n not a multiple of 4
        H.hf_launch_single(k, H.stream_tmpl_args(x[:6], x[:6], 1), 128, 1)
    assert e.value.status == -1
    with pytest.raises(H.HFError):                            # 50 KB staging
        H.hf_launch_single(k, H.stream_tmpl_args(x, x, 1, 0, 50 * 1024), 128, 1)
    kb = H.hf_register_kernel(H.BN_STATS)
    xb = torch.zeros(1, 2, 2, 2, device=DEV)
    m = torch.empty(2, device=DEV)
    with pytest.raises(H.HFError):                            # no workspace
        H.hf_launch_single(kb, H.bn_stats_args(xb, m, m, None), 128, 1)


# ------------------------------------------------------------------ fused vs standalone
def _case(body, seed):
    """(args builder, outputs) for a small problem of each body."""
    g = seed
    if body == H.BN_STATS:
        x = W.bn_input((4, 6, 24, 20), g).to(DEV)
        ws = H.bn_stats_workspace(x)
        outs = [torch.empty(6, device=DEV), torch.empty(6, device=DEV)]
        return (lambda o: H.bn_stats_args(x, o[0], o[1], ws)), outs
    if body == H.UPSAMPLE2X:
        x = W.upsample_input((3, 2, 36, 40), g).to(DEV)
        return (lambda o: H.upsample2x_args(x, o[0])), [torch.empty(3, 2, 72, 80, device=DEV)]
    if body == H.MAXPOOL3S2:
        x = W.maxpool_input((3, 4, 42, 40), g).to(DEV)
        return (lambda o: H.maxpool3s2_args(x, o[0])), [torch.empty(3, 4, 21, 20, device=DEV)]
    if body == H.IM2COL3:
        x = W.im2col_input((2, 3, 13, 16), g).to(DEV)
        return (lambda o: H.im2col3_args(x, o[0])), [torch.empty(2, 27, 13 * 16, device=DEV)]
    if body == H.HIST256:
        x = W.hist_input(300007, g).to(DEV)
        outs = [torch.zeros(256, dtype=torch.int32, device=DEV)]
        return (lambda o: H.hist256_args(x, o[0])), outs
    if body == H.PHILOX:
        return (lambda o: H.philox_args(o[0], 99, 5)), [torch.empty(5003, 4, dtype=torch.int32, device=DEV)]
    if body == H.POLY:
        x = W.poly_input(10007, g).to(DEV)
        c = W.poly_coefficients().tolist()
        return (lambda o: H.poly_args(x, o[0], c)), [torch.empty(10007, device=DEV)]
    if body == H.BF16_AXPY:
        x, y = (t.to(DEV) for t in W.bf16_inputs(20011, g))
        return (lambda o: H.bf16_axpy_args(x, y, o[0])), [torch.empty(20011, dtype=torch.bfloat16, device=DEV)]
    if body == H.STREAM_TMPL:
        x = W.template_input(4 * 5000, g).to(DEV)
        k = 4 + seed % 9
        return (lambda o: H.stream_tmpl_args(x, o[0], k, 2, 2048)), [torch.empty(4 * 5000, device=DEV)]
    raise ValueError(body)


def _fresh(outs):
    return [torch.zeros_like(o) for o in outs]


PAIRS = [(H.BN_STATS, H.POLY), (H.UPSAMPLE2X, H.MAXPOOL3S2), (H.HIST256, H.PHILOX),
         (H.STREAM_TMPL, H.STREAM_TMPL), (H.MAXPOOL3S2, H.UPSAMPLE2X), (H.BN_STATS, H.HIST256),
         (H.IM2COL3, H.UPSAMPLE2X), (H.BF16_AXPY, H.POLY), (H.PHILOX, H.IM2COL3)]


@pytest.mark.parametrize("pair", PAIRS, ids=lambda p: "%s+%s" % (H.BODY_NAMES[p[0]], H.BODY_NAMES[p[1]]))
@pytest.mark.parametrize("split,d0,regcap,grid", [(256, 512, 0, 40), (128, 512, 32, 17),
                                                   (384, 512, 64, 0), (64, 256, 0, 3)])
def test_fused_pair_bit_exact(pair, split, d0, regcap, grid):
    a, b = pair
    mk_a, outs_a = _case(a, 1)
    mk_b, outs_b = _case(b, 2)
    ka, kb = H.hf_register_kernel(a), H.hf_register_kernel(b)
    f = H.hf_fuse(ka, kb, split, d0, regcap)
    fa, fb = _fresh(outs_a), _fresh(outs_b)
    H.hf_launch(f, [mk_a(fa), mk_b(fb)], grid=grid)
    g = grid if grid else H.hf_query(f, [mk_a(fa), mk_b(fb)])["blocks_per_sm"] * H.hf_device_info().sm_count
    sa, sb = _fresh(outs_a), _fresh(outs_b)
    H.hf_launch_single(ka, mk_a(sa), split, grid=g)
    H.hf_launch_single(kb, mk_b(sb), d0 - split, grid=g)
    torch.cuda.synchronize()
    for u, v in zip(fa + fb, sa + sb):
        assert torch.equal(u, v)
    H.hf_destroy_fused(f)


def test_fused_matches_oracle_bn_poly():
    x = W.bn_input((8, 64, 32, 32)).to(DEV)
    px = W.poly_input(1 << 16).to(DEV)
    coef = W.poly_coefficients().numpy()
    mean, var, py = torch.empty(64, device=DEV), torch.empty(64, device=DEV), torch.empty_like(px)
    f = H.hf_fuse(H.hf_register_kernel(H.BN_STATS), H.hf_register_kernel(H.POLY), 256, 512, 0)
    H.hf_launch(f, [H.bn_stats_args(x, mean, var, H.bn_stats_workspace(x)), H.poly_args(px, py, coef)])
    torch.cuda.synchronize()
    check_bn(x.cpu(), mean, var)
    check_poly(px.cpu(), coef, py)


def test_nway_eight_bodies_bit_exact():
    bodies = [H.BN_STATS, H.IM2COL3, H.MAXPOOL3S2, H.UPSAMPLE2X, H.HIST256, H.PHILOX, H.POLY, H.BF16_AXPY]
    cases = [_case(b, i + 10) for i, b in enumerate(bodies)]
    ks = [H.hf_register_kernel(b) for b in bodies]
    threads = [64] * 8
    f = H.hf_fuse_n(ks, list(range(8)), threads, 0)
    outs = [_fresh(o) for _, o in cases]
    H.hf_launch(f, [mk(o) for (mk, _), o in zip(cases, outs)], grid=23)
    ref = [_fresh(o) for _, o in cases]
    for k, (mk, _), o, t in zip(ks, cases, ref, threads):
        H.hf_launch_single(k, mk(o), t, grid=23)
    torch.cuda.synchronize()
    for fo, ro in zip(outs, ref):
        for u, v in zip(fo, ro):
            assert torch.equal(u, v)


def test_nway_shared_interval_schedule():
    """Several kernels on one interval run one after another (LPT-style
    packing) and still give the bits of their standalone launches."""
    bodies = [H.HIST256, H.STREAM_TMPL, H.BN_STATS, H.POLY, H.HIST256]
    cases = [_case(b, i + 20) for i, b in enumerate(bodies)]
    ks = [H.hf_register_kernel(b) for b in bodies]
    interval_of = [0, 0, 1, 2, 1]
    threads = [128, 256, 128]
    f = H.hf_fuse_n(ks, interval_of, threads, 0)
    outs = [_fresh(o) for _, o in cases]
    H.hf_launch(f, [mk(o) for (mk, _), o in zip(cases, outs)], grid=9)
    ref = [_fresh(o) for _, o in cases]
    for k, (mk, _), o, i in zip(ks, cases, ref, interval_of):
        H.hf_launch_single(k, mk(o), threads[i], grid=9)
    torch.cuda.synchronize()
    for fo, ro in zip(outs, ref):
        for u, v in zip(fo, ro):
            assert torch.equal(u, v)


def test_nway_kernel_cut_across_intervals():
    """One kernel's range cut into two kernels of the same body on different
    intervals (bf16 by elements, Philox by counter offset, upsample by
    planes) gives the bits of one standalone launch over the whole range."""
    n16 = 8 * 5003
    x16, y16 = (t.to(DEV) for t in W.bf16_inputs(n16, 31))
    xu = W.upsample_input((6, 1, 20, 24), 32).to(DEV)
    np_, m16, mp, mu = 10007, 8 * 2001, 4096, 2
    o16, po, yu = (torch.empty_like(x16), torch.empty((np_, 4), dtype=torch.int32, device=DEV),
                   torch.empty((6, 1, 40, 48), device=DEV))
    parts = [(H.BF16_AXPY, H.bf16_axpy_args(x16[:m16], y16[:m16], o16[:m16]), 0),
             (H.PHILOX, H.philox_args(po[:mp], 7, 5), 0),
             (H.UPSAMPLE2X, H.upsample2x_args(xu[:mu], yu[:mu]), 1),
             (H.BF16_AXPY, H.bf16_axpy_args(x16[m16:], y16[m16:], o16[m16:]), 1),
             (H.PHILOX, H.philox_args(po[mp:], 7, 5 + mp), 2),
             (H.UPSAMPLE2X, H.upsample2x_args(xu[mu:], yu[mu:]), 2)]
    ks = [H.hf_register_kernel(b) for b, _, _ in parts]
    f = H.hf_fuse_n(ks, [i for _, _, i in parts], [96, 128, 64], 0)
    H.hf_launch(f, [a for _, a, _ in parts], grid=11)
    r16, rpo, ryu = torch.empty_like(o16), torch.empty_like(po), torch.empty_like(yu)
    single(H.BF16_AXPY, H.bf16_axpy_args(x16, y16, r16), 128, 11)
    single(H.PHILOX, H.philox_args(rpo, 7, 5), 128, 11)
    single(H.UPSAMPLE2X, H.upsample2x_args(xu, ryu), 128, 11)
    torch.cuda.synchronize()
    assert H.hf_check_device_error() == 0
    assert torch.equal(o16, r16) and torch.equal(po, rpo) and torch.equal(yu, ryu)
    assert np.array_equal(rpo.cpu().numpy().view(np.uint32), oracle.philox4x32_10(7, np_, first=5))
    H.hf_destroy_fused(f)


def test_stream_wait_and_query():
    k = H.hf_register_kernel(H.POLY)
    x = torch.rand(1 << 16, device=DEV)
    y = torch.empty_like(x)
    H.hf_launch_single(k, H.poly_args(x, y, [0.01] * 33), 256)
    H.hf_stream_wait(None, 10000)
    info = H.hf_query_single(k, H.poly_args(x, y, [0.01] * 33), 256)
    assert info["regs"] > 0 and info["blocks_per_sm"] >= 1
    lim = H.hf_device_info()
    assert lim.sm_count > 0 and lim.regs_per_sm == 65536


@pytest.mark.parametrize("pair", [(H.BN_STATS, H.HIST256), (H.UPSAMPLE2X, H.MAXPOOL3S2)],
                         ids=lambda p: "%s+%s" % (H.BODY_NAMES[p[0]], H.BODY_NAMES[p[1]]))
def test_vertical_fusion_schedule_bit_exact(pair):
    """Vertical fusion (Sec. 2.2): both kernels on one interval of the whole
    block, one after the other, equal their standalone launches."""
    a, b = pair
    mk_a, outs_a = _case(a, 3)
    mk_b, outs_b = _case(b, 4)
    ka, kb = H.hf_register_kernel(a), H.hf_register_kernel(b)
    f = H.hf_fuse_n([ka, kb], [0, 0], [256], 0)
    fa, fb = _fresh(outs_a), _fresh(outs_b)
    H.hf_launch(f, [mk_a(fa), mk_b(fb)], grid=19)
    sa, sb = _fresh(outs_a), _fresh(outs_b)
    H.hf_launch_single(ka, mk_a(sa), 256, grid=19)
    H.hf_launch_single(kb, mk_b(sb), 256, grid=19)
    torch.cuda.synchronize()
    for u, v in zip(fa + fb, sa + sb):
        assert torch.equal(u, v)
