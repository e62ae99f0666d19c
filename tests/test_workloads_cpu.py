"""The seeded input recipe (the only code the CUDA path and the oracle share):
the same seed gives the same bytes, the distributions and shapes are the ones
the workloads state, and the 8-way workload moves the bytes its roofline is
computed from."""
import numpy as np
import torch

from paper_2007_01277_gb300 import workloads as W


def test_same_seed_same_bytes_and_plain_cpu_generator():
    a, b = W.bn_input((2, 3, 8, 8), seed=5), W.bn_input((2, 3, 8, 8), seed=5)
    assert torch.equal(a, b)
    assert not torch.equal(a, W.bn_input((2, 3, 8, 8), seed=6))
    # the CPU path is torch's CPU generator seeded with the seed, drawn once
    ref = torch.randn(2, 3, 8, 8, generator=torch.Generator().manual_seed(5))
    assert torch.equal(a, ref)
    u = W.uniform((1000,), -1.0, 1.0, 9)
    ref = torch.rand(1000, generator=torch.Generator().manual_seed(9)) * 2.0 - 1.0
    assert torch.equal(u, ref)


def test_distributions_follow_the_recipe():
    x = W.bn_input((8, 64, 32, 32))                       # ~N(0, 1)
    assert abs(x.mean().item()) < 0.01 and abs(x.std().item() - 1.0) < 0.01
    u = W.upsample_input((4, 64, 32, 32))                 # ~U(0, 1)
    assert u.min().item() >= 0.0 and u.max().item() < 1.0 and abs(u.mean().item() - 0.5) < 0.01
    p = W.poly_input(1 << 16)                             # ~U(-1, 1)
    assert p.min().item() >= -1.0 and p.max().item() < 1.0
    c = W.poly_coefficients()                             # 33 values ~U(-0.1, 0.1)
    assert c.shape == (33,) and c.abs().max().item() <= 0.1
    h = W.hist_input(1 << 20)                             # ~U[0, 255] bytes
    counts = np.bincount(h.numpy(), minlength=256)
    assert h.dtype == torch.uint8 and counts.min() > 0
    assert abs(counts.mean() - (1 << 20) / 256) < 1e-9 and counts.std() / counts.mean() < 0.05
    x16, y16 = W.bf16_inputs(4096)
    assert x16.dtype == torch.bfloat16 and x16.abs().max().item() <= 1.0
    assert not torch.equal(x16, y16)


def test_nway8_workload_bytes():
    sp = W.WORKLOADS["nway8"]
    f32 = 4
    bn = np.prod(sp["bn"]) * f32
    N, C, H, Wd = sp["im2col"]
    im2col = N * C * H * Wd * f32 * (1 + 9)
    P = np.prod(sp["pool"][:2])
    pool = P * sp["pool"][2] * sp["pool"][3] * f32 + P * 56 * 56 * f32
    Pu = np.prod(sp["up"][:2])
    up = Pu * sp["up"][2] * sp["up"][3] * f32 * (1 + 4)
    hist = sp["hist_n"]
    philox = sp["philox_n"] * 16
    poly = sp["poly_n"] * f32 * 2
    bf16 = sp["bf16_n"] * 2 * 3
    total = bn + im2col + pool + up + hist + philox + poly + bf16
    # the algorithmic bytes of the 8-way roofline: 2564.8 MB (outputs of
    # batch-norm statistics and the histogram are a few KB and left out)
    assert abs(total / 1e6 - 2564.8) < 0.1, total / 1e6
