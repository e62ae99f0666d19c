"""Pins of the CPU oracle to facts outside itself (CPU only).

Each test checks one oracle function against something the paper or the
mathematics fixes -- a hand-worked grid under tests/golden/, a closed form, a
special case that reduces to a library routine, or brute force -- chosen so
that a dropped term, a wrong sign or index, or a transposed operand fails.
"""
import ctypes
import math
import os

import numpy as np
import pytest
import torch

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    """Blocks of numeric rows separated by comment lines."""
    blocks, cur = [], []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            if cur:
                blocks.append(cur)
                cur = []
            continue
        cur.append([float(v) for v in line.split()])
    if cur:
        blocks.append(cur)
    return [np.array(b) for b in blocks]


# ------------------------------------------------------------------ upsample
def test_upsample_hand_grid(orc):
    inp, out = read_golden("upsample2x_2x2.txt")
    got = orc.upsample2x(inp.astype(np.float32))
    np.testing.assert_array_equal(got, out)


def test_upsample_vs_torch_interpolate(orc):
    x = torch.rand(2, 3, 7, 5, generator=torch.Generator().manual_seed(1))
    ref = torch.nn.functional.interpolate(x.double(), scale_factor=2, mode="bilinear",
                                          align_corners=False)
    got = orc.upsample2x(x.numpy())
    np.testing.assert_allclose(got, ref.numpy(), rtol=0, atol=1e-12)


def test_upsample_constant_and_linear(orc):
    # a constant image stays constant; a ramp in x stays affine away from
    # the clamped border columns
    c = np.full((1, 4, 6), 3.5, np.float32)
    assert np.all(orc.upsample2x(c) == 3.5)
    ramp = np.tile(np.arange(8, dtype=np.float32), (3, 1))[None]
    out = orc.upsample2x(ramp)[0, 0]
    # interior outputs o in [1, 14]: value = o/2 - 0.25
    o = np.arange(1, 15)
    np.testing.assert_allclose(out[o], o / 2 - 0.25, atol=1e-15)


# ------------------------------------------------------------------ maxpool
def test_maxpool_hand_grid(orc):
    inp, out = read_golden("maxpool3s2p1_4x4.txt")
    got = orc.maxpool3s2p1(inp.astype(np.float32))
    np.testing.assert_array_equal(got, out.astype(np.float32))


@pytest.mark.parametrize("shape", [(2, 3, 9, 11), (1, 2, 112, 112), (1, 1, 1, 1)])
def test_maxpool_vs_torch(orc, shape):
    x = torch.randn(*shape, generator=torch.Generator().manual_seed(2))
    ref = torch.nn.functional.max_pool2d(x, 3, stride=2, padding=1)
    np.testing.assert_array_equal(orc.maxpool3s2p1(x.numpy()), ref.numpy())


# ------------------------------------------------------------------ im2col
def test_im2col_hand_grid(orc):
    inp, out = read_golden("im2col3_2x2.txt")
    got = orc.im2col3(inp.astype(np.float32)[None, None])
    np.testing.assert_array_equal(got[0], out.astype(np.float32))


def test_im2col_vs_torch_unfold(orc):
    x = torch.randn(2, 3, 5, 6, generator=torch.Generator().manual_seed(3))
    ref = torch.nn.functional.unfold(x, kernel_size=3, padding=1)
    np.testing.assert_array_equal(orc.im2col3(x.numpy()), ref.numpy())


# ------------------------------------------------------------------ histogram
def test_hist_vs_bincount(orc):
    x = torch.randint(0, 256, (100003,), generator=torch.Generator().manual_seed(4),
                      dtype=torch.uint8).numpy()
    bins = orc.hist256(x)
    np.testing.assert_array_equal(bins, np.bincount(x, minlength=256))
    assert bins.sum() == x.size


def test_hist_constant_and_empty(orc):
    bins = orc.hist256(np.full(1000, 7, np.uint8))
    assert bins[7] == 1000 and bins.sum() == 1000
    assert orc.hist256(np.zeros(0, np.uint8)).sum() == 0
    x = np.arange(256, dtype=np.uint8)
    assert np.all(orc.hist256(x) == 1)


# ------------------------------------------------------------------ batch norm
def test_bn_hand_channel(orc):
    shape, vals, res = read_golden("bn_stats_channel.txt")
    x = vals.astype(np.float32).reshape(shape[0].astype(int))
    mean, var = orc.bn_stats(x)
    assert mean[0] == res[0][0] and var[0] == res[0][1]


def test_bn_vs_numpy_and_invariants(orc):
    x = torch.randn(3, 5, 4, 7, generator=torch.Generator().manual_seed(5)).numpy()
    mean, var = orc.bn_stats(x)
    xd = x.astype(np.float64)
    np.testing.assert_allclose(mean, xd.mean(axis=(0, 2, 3)), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(var, xd.var(axis=(0, 2, 3)), rtol=1e-12)
    # constant channel -> variance 0; shifting a channel shifts only the mean
    c = np.full((2, 1, 3, 3), 4.0, np.float32)
    m, v = orc.bn_stats(c)
    assert m[0] == 4.0 and v[0] == 0.0
    m2, v2 = orc.bn_stats(x + np.float32(8.0))
    np.testing.assert_allclose(m2, mean + 8.0, rtol=1e-6)
    np.testing.assert_allclose(v2, var, rtol=1e-5)


# ------------------------------------------------------------------ Philox
def _curand_host_philox(seed, nwords):
    path = None
    for cand in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            L = ctypes.CDLL(cand)
            path = cand
            break
        except OSError:
            continue
    if path is None:
        pytest.skip("libcurand not found")
    gen = ctypes.c_void_p()
    assert L.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    assert L.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    out = np.zeros(nwords, np.uint32)
    assert L.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                            ctypes.c_size_t(nwords)) == 0
    L.curandDestroyGenerator(gen)
    return out.reshape(-1, 4)


@pytest.mark.parametrize("seed", [0, 0x0123456789ABCDEF])
def test_philox_vs_curand_host_generator(orc, seed):
    """cuRAND's host Philox4_32_10 generator emits block b from counter
    (b // 65536, 0, b % 65536, 0) under key (lo32(seed), hi32(seed)).  Blocks
    b = 65536 t are therefore the oracle's outputs t (counter (t, 0, 0, 0));
    the other blocks pin the round function on the third counter word."""
    T = 24
    blocks = _curand_host_philox(seed, 4 * 65536 * T)
    ours = orc.philox4x32_10(seed, T)
    np.testing.assert_array_equal(blocks[::65536][:T], ours)
    # counter (0, 0, j, 0) through the oracle's exported round function
    L = orc.lib()
    W = np.array([0x9E3779B9, 0xBB67AE85], np.uint64)
    for j in (1, 2, 12345, 65535):
        c = np.array([0, 0, j, 0], np.uint32)
        k = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
        for r in range(10):
            if r:
                k = ((k.astype(np.uint64) + W) & 0xFFFFFFFF).astype(np.uint32)
            L.or_philox_round(c.ctypes.data_as(ctypes.c_void_p),
                              k.ctypes.data_as(ctypes.c_void_p))
        np.testing.assert_array_equal(c, blocks[j])


def test_philox_weyl_constants_and_offsets(orc):
    # The key increments are the leading 32 fraction bits of the golden
    # ratio and of sqrt(3) (Salmon et al.); check them from the irrationals.
    from decimal import Decimal, getcontext
    getcontext().prec = 50
    w0 = int((Decimal(5).sqrt() - 1) / 2 * (1 << 32))
    w1 = int((Decimal(3).sqrt() - 1) * (1 << 32))
    assert (w0, w1) == (0x9E3779B9, 0xBB67AE85)
    # output i of a stream equals output 0 of the stream starting at i
    a = orc.philox4x32_10(7, 40)
    for i in (0, 5, 39):
        np.testing.assert_array_equal(orc.philox4x32_10(7, 1, first=i)[0], a[i])
    # the high counter word is used: counters 2^32 and 0 differ
    assert not np.array_equal(orc.philox4x32_10(7, 1, first=1 << 32)[0], a[0])
    # distinct counters give distinct blocks (Philox is a bijection per key)
    b = orc.philox4x32_10(3, 4096)
    assert len({tuple(r) for r in b}) == 4096


# ------------------------------------------------------------------ polynomial
def _coef(seed=0):
    g = torch.Generator().manual_seed(seed)
    return (torch.rand(33, generator=g) * 0.2 - 0.1).numpy()


def test_poly_one_step_is_polyval(orc):
    c = _coef()
    x = np.linspace(-1, 1, 101).astype(np.float32)
    got = orc.poly(x, c, iters=1)
    ref = np.polyval(c[::-1].astype(np.float64), x.astype(np.float64))
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-16)


def test_poly_closed_form(orc):
    # acc_T = p(x) (1 - x^(33T)) / (1 - x^33) for x^33 != 1
    c = _coef(1)
    x = np.array([-0.97, -0.5, -0.1, 0.3, 0.8, 0.99], np.float32)
    xd = x.astype(np.float64)
    p = np.polyval(c[::-1].astype(np.float64), xd)
    for T in (2, 64):
        ref = p * (1 - xd ** (33 * T)) / (1 - xd ** 33)
        np.testing.assert_allclose(orc.poly(x, c, iters=T), ref, rtol=1e-12)


def test_poly_special_points(orc):
    c = _coef(2)
    # x = 0: every step returns c_0
    assert orc.poly(np.zeros(3, np.float32), c)[0] == np.float64(c[0])
    # x = 1: acc_T = T * sum(c)
    np.testing.assert_allclose(orc.poly(np.ones(1, np.float32), c, iters=64)[0],
                               64 * c.astype(np.float64).sum(), rtol=1e-13)
    # the conditioning scale is sum_k |c_k| |x|^k * sum_t |x|^(33t)
    x = np.array([0.5], np.float32)
    _, b = orc.poly(x, c, iters=3, with_bound=True)
    pa = sum(abs(float(c[k])) * 0.5 ** k for k in range(33))
    np.testing.assert_allclose(b[0], pa * (1 + 0.5 ** 33 + 0.5 ** 66), rtol=1e-14)


# ------------------------------------------------------------------ bf16
def _bits(t):
    return t.view(torch.int16).numpy().view(np.uint16)


def test_bf16_rounding_vs_torch(orc):
    g = torch.Generator().manual_seed(6)
    v = (torch.randn(20000, generator=g, dtype=torch.float64) *
         torch.exp2(torch.randint(-140, 120, (20000,), generator=g).double()))
    ref = _bits(v.to(torch.bfloat16))
    got = np.array([orc.double_to_bf16(float(a)) for a in v], np.uint16)
    np.testing.assert_array_equal(got, ref)


def test_bf16_ties_to_even(orc):
    # 1 + 2^-8 lies half way between bf16 1 and 1 + 2^-7: rounds to even (1);
    # 1 + 3*2^-8 lies half way between 1+2^-7 and 1+2^-6: rounds to 1+2^-6.
    assert orc.double_to_bf16(1 + 2 ** -8) == 0x3F80
    assert orc.double_to_bf16(1 + 3 * 2 ** -8) == 0x3F82
    assert orc.double_to_bf16(-2.0) == 0xC000
    assert orc.double_to_bf16(0.0) == 0


def test_bf16_axpy_vs_torch(orc):
    g = torch.Generator().manual_seed(7)
    x = (torch.rand(5000, generator=g) * 2 - 1).to(torch.bfloat16)
    y = (torch.rand(5000, generator=g) * 2 - 1).to(torch.bfloat16)
    ref = _bits((0.5 * x.double() + y.double()).to(torch.bfloat16))
    np.testing.assert_array_equal(orc.bf16_axpy(_bits(x), _bits(y), 0.5), ref)


# ------------------------------------------------------------------ template
@pytest.mark.parametrize("k", [0, 1, 2, 3, 4, 7, 64])
def test_stream_template_closed_form(orc, k):
    a, b = 0.999, 0.001
    x = np.linspace(-1, 1, 64).astype(np.float32)
    got = orc.stream_tmpl(x, k, a, b).reshape(-1, 4)
    ad, bd = float(np.float32(a)), float(np.float32(b))
    for j in range(4):
        kj = k // 4 + (1 if j < k % 4 else 0)       # FMAs landing on component j
        v = x.reshape(-1, 4)[:, j].astype(np.float64)
        ref = ad ** kj * v + bd * (ad ** kj - 1) / (ad - 1)
        np.testing.assert_allclose(got[:, j], ref, rtol=1e-12, atol=1e-15)


# ------------------------------------------------------------------ MLP
def _mlp_data(seed, B):
    g = torch.Generator().manual_seed(seed)
    return (torch.randn(B, 24, generator=g).numpy(), torch.randn(B, generator=g).numpy(),
            torch.randn(5825, generator=g, dtype=torch.float64).numpy() * 0.2)


def test_mlp_grad_finite_differences(orc):
    X, Y, P = _mlp_data(8, 16)
    assert orc.mlp_nparam() == 5825
    loss, g = orc.mlp_loss_grad(P, X, Y)
    rng = np.random.default_rng(0)
    for i in list(rng.choice(5825, 40, replace=False)) + [5824, 0, 1535, 1600]:
        h = 1e-6
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (orc.mlp_loss_grad(Pp, X, Y)[0] - orc.mlp_loss_grad(Pm, X, Y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i


def test_mlp_vs_torch_autograd(orc):
    X, Y, P = _mlp_data(9, 32)
    t = torch.tensor(P, requires_grad=True)
    o = 0
    W1 = t[o:o + 1536].view(64, 24); o += 1536
    b1 = t[o:o + 64]; o += 64
    W2 = t[o:o + 4096].view(64, 64); o += 4096
    b2 = t[o:o + 64]; o += 64
    w3 = t[o:o + 64]; o += 64
    b3 = t[o]
    xt = torch.tensor(X, dtype=torch.float64)
    h = torch.relu(xt @ W1.T + b1)
    h = torch.relu(h @ W2.T + b2)
    y = h @ w3 + b3
    loss = ((y - torch.tensor(Y, dtype=torch.float64)) ** 2).mean()
    loss.backward()
    l2, g = orc.mlp_loss_grad(P, X, Y)
    np.testing.assert_allclose(l2, loss.item(), rtol=1e-13)
    np.testing.assert_allclose(g, t.grad.numpy(), rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(orc.mlp_forward(P, X), y.detach().numpy(), rtol=1e-13)


def test_adam_vs_torch(orc):
    rng = np.random.default_rng(1)
    P = rng.standard_normal(50)
    t = torch.tensor(P.copy(), requires_grad=True)
    opt = torch.optim.Adam([t], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    m, v = np.zeros(50), np.zeros(50)
    for step in range(1, 6):
        g = rng.standard_normal(50)
        t.grad = torch.tensor(g)
        opt.step()
        orc.adam_step(P, g, m, v, step)
    np.testing.assert_allclose(P, t.detach().numpy(), rtol=1e-12, atol=1e-15)


# ------------------------------------------------------------------ Sec. 2.1 / Alg. 2
def test_occupancy_worked_example(orc):
    (rows,) = read_golden("occupancy_sec2_1.txt")
    for r in rows.astype(int):
        assert orc.blocks_per_sm(*r[:6]) == r[6]


def test_register_bound_worked_example(orc):
    blocks = read_golden("fused_example_sec2_3.txt")
    for r in blocks[1].astype(int):
        assert orc.register_bound(*r[:8]) == r[8]
    # hand-derived: the bound restores the original kernels' block count
    # b1 = 65536/(256*64) = 4, b2 = 65536/(256*32) = 8, threads 2048/512 = 4
    assert orc.register_bound(65536, 98304, 2048, 256, 64, 256, 32, 0) == 32
    # shared memory can be the binding term: 98304/40000 = 2 -> r0 = 64
    assert orc.register_bound(65536, 98304, 2048, 256, 32, 256, 32, 40000) == 64
    # the fused block does not fit at all -> 0
    assert orc.register_bound(65536, 98304, 2048, 256, 32, 256, 32, 100000) == 0


def test_alg2_search_matches_bruteforce(orc):
    rng = np.random.default_rng(2)
    for trial in range(20):
        d0 = 1024
        table = {}
        for d1 in range(128, d0, 128):
            table[(d1, None)] = float(rng.integers(1, 50))
            table[(d1, 32)] = float(rng.integers(1, 50))
        d, r, t = orc.alg2_search(d0, lambda d1, rr: table[(d1, rr)], lambda d1: 32)
        best = min(table.values())
        assert t == best and table[(d, r)] == best
        # first-found wins on ties: splits ascending, unbounded before bounded
        order = [(d1, rr) for d1 in range(128, d0, 128) for rr in (None, 32)]
        first = next(k for k in order if table[k] == best)
        assert (d, r) == first
