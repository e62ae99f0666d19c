"""Seeded synthetic inputs and workload shapes.

This module is the only code shared by the CUDA path and the CPU oracle: it
draws inputs with ``torch.Generator().manual_seed(seed)`` on the CPU and holds
none of the method's arithmetic.  Shapes and value distributions follow the
five workloads the library is measured on (none of them is a public dataset;
the paper's own inputs are unstated, Sec. 4.3 only says sizes were chosen so
that paired kernels take similar time).
"""
from __future__ import annotations

import math

import torch

# Workload shapes.  Each entry names the constituent kernels and their sizes.
WORKLOADS = {
    # batch-norm statistics on FP32 NCHW 8x64x32x32 ~N(0,1) fused with the
    # 64-step degree-32 Horner chain on 2^20 FP32 ~U(-1,1); 256+256 threads.
    "bn_poly_small": dict(bn=(8, 64, 32, 32), poly_n=1 << 20, d0=512, split=256),
    # bilinear x2 of 32x64x128x128 ~U(0,1) with 3x3/s2/p1 max-pool of
    # 32x128x112x112 ~N(0,1); splits 1:3, 1:1, 3:1 of a 512-thread block.
    "upsample_maxpool": dict(up=(32, 64, 128, 128), pool=(32, 128, 112, 112), d0=512,
                             splits=(128, 256, 384)),
    # 256-bin histogram of 2^28 bytes ~U[0,255] with Philox4x32-10 producing
    # 2^26 outputs of 16 bytes; splits 1:7 .. 7:1 warps of a 256-thread block.
    "hist_philox": dict(hist_n=1 << 28, philox_n=1 << 26, d0=256,
                        regcaps=(0, 32, 40, 48, 64, 96), blocks_per_sm=(1, 2, 3, 4)),
    # eight uneven kernels in one persistent launch.
    "nway8": dict(bn=(64, 256, 56, 56), im2col=(32, 64, 56, 56), pool=(32, 128, 112, 112),
                  up=(32, 64, 128, 128), hist_n=1 << 26, philox_n=1 << 24,
                  poly_n=1 << 22, bf16_n=1 << 27),
    # the three compute-bound hash scans over one random 80-byte header:
    # nonces 0 .. n-1 each, sized so that each alone takes about the same
    # time; target 2^16 accepts about one nonce in 65536.
    "hash_pairs": dict(sha256d_n=1 << 24, blake256_n=1 << 25, blake2b_n=21 << 20, target=1 << 16),
}

POLY_ITERS = 64
POLY_DEGREE = 32
BF16_ALPHA = 0.5
SEED = 0


def gen(seed: int, device=None) -> torch.Generator:
    """The seeded generator: on the CPU by default.  Inputs of several GB
    (the tests past 32-bit indexing) are drawn by the device's generator
    instead, and the oracle gets the same bytes copied back."""
    g = torch.Generator(device=device) if device is not None else torch.Generator()
    return g.manual_seed(int(seed))


def normal(shape, seed: int, device=None) -> torch.Tensor:
    """float32 ~N(0,1)."""
    return torch.randn(*shape, generator=gen(seed, device), dtype=torch.float32, device=device)


def uniform(shape, lo: float, hi: float, seed: int, device=None) -> torch.Tensor:
    """float32 ~U(lo, hi)."""
    t = torch.rand(*shape, generator=gen(seed, device), dtype=torch.float32, device=device)
    return t.mul_(hi - lo).add_(lo)


def bytes_u8(n: int, seed: int, device=None) -> torch.Tensor:
    """uint8 ~U[0, 255]."""
    return torch.randint(0, 256, (n,), generator=gen(seed, device), dtype=torch.uint8, device=device)


def bf16_uniform(n: int, seed: int) -> torch.Tensor:
    """bfloat16 ~U(-1, 1) (drawn in float32, stored as bfloat16)."""
    return uniform((n,), -1.0, 1.0, seed).to(torch.bfloat16)


def poly_coefficients(seed: int = SEED) -> torch.Tensor:
    """The 33 coefficients c_0..c_32 ~U(-0.1, 0.1)."""
    return uniform((POLY_DEGREE + 1,), -0.1, 0.1, seed + 1000)


def bn_input(shape, seed: int = SEED):
    return normal(shape, seed)


def poly_input(n: int, seed: int = SEED):
    return uniform((n,), -1.0, 1.0, seed + 1)


def upsample_input(shape, seed: int = SEED):
    return uniform(shape, 0.0, 1.0, seed + 2)


def maxpool_input(shape, seed: int = SEED):
    return normal(shape, seed + 3)


def im2col_input(shape, seed: int = SEED):
    return normal(shape, seed + 4)


def hist_input(n: int, seed: int = SEED):
    return bytes_u8(n, seed + 5)


def bf16_inputs(n: int, seed: int = SEED):
    return bf16_uniform(n, seed + 6), bf16_uniform(n, seed + 7)


def hash_header(seed: int = SEED) -> bytes:
    """An 80-byte block header of uniform random bytes; the scans overwrite
    its bytes 76..79 with each item's nonce."""
    return bytes(bytes_u8(80, seed + 9).numpy().tobytes())


def template_input(n: int, seed: int = SEED):
    return uniform((n,), -1.0, 1.0, seed + 8)


def log_uniform_int(lo: int, hi: int, g: torch.Generator) -> int:
    """An integer ~ 2^U(log2 lo, log2 hi), rounded down to a multiple of 4."""
    u = torch.rand((), generator=g).item()
    v = math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
    return max(4, int(v) // 4 * 4)
