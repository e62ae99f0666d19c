"""CPU oracle for the horizontal-fusion hot path -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
binding in ``paper_2007_01277_gb300``) never imports it, and this package
imports nothing from the product: the only code both sides use is the seeded
input generator module, which holds none of the method's arithmetic.

The numerical work lives in ``hf_oracle.c`` (plain C, double precision or
exact integers); this module compiles it with gcc, loads it with ctypes and
wraps it for numpy arrays.  The pure-Python pieces below are the search of
Algorithm 2 (Sec. 3.2) run over a table of measured times, and the regret and
speedup definitions used for reporting.

Parity status of each function (what pins it, in ``tests/test_oracle_pins.py``):
  bn_stats      numpy mean/var, shift invariance, hand-worked channel
  upsample2x    hand-worked 2x2 grid, torch interpolate in float64
  maxpool3s2p1  hand-worked 4x4 grid, torch max_pool2d
  im2col3       hand-worked 2x2 grid, torch unfold
  hist256       numpy bincount, totals, constant input
  philox        cuRAND host generator, Weyl constants from sqrt(5), sqrt(3)
  poly          numpy polyval, closed-form geometric sum, x = 0 case
  bf16_axpy     torch float64 -> bfloat16 rounding, exact-tie cases
  stream_tmpl   closed form of the affine recurrence
  mlp           finite differences and torch autograd in float64
  register_bound / blocks_per_sm   the worked example of Sec. 2.1
  alg2_search   brute-force argmin over the same table
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

MLP_IN = 24
MLP_H = 64


def build(force: bool = False) -> str:
    """Compile hf_oracle.c into liboracle.so next to it (plain gcc, no
    contraction of multiply-adds so that the double arithmetic is the one
    written in the source)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    subprocess.check_call([
        "gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
        "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i32, i64, u64, f64 = ctypes.c_int, ctypes.c_long, ctypes.c_uint64, ctypes.c_double
        sig = {
            "or_bn_stats": (None, [P, i32, i32, i32, P, P]),
            "or_upsample2x": (None, [P, i32, i32, i32, P]),
            "or_maxpool3s2p1": (None, [P, i32, i32, i32, P]),
            "or_im2col3": (None, [P, i32, i32, i32, i32, P]),
            "or_hist256": (None, [P, i64, P]),
            "or_philox4x32_10": (None, [u64, u64, i64, P]),
            "or_philox_round": (None, [P, P]),
            "or_poly": (None, [P, i64, P, i32, P, P]),
            "or_double_to_bf16": (ctypes.c_uint16, [f64]),
            "or_bf16_axpy": (None, [P, P, f64, i64, P]),
            "or_stream_tmpl": (None, [P, i64, i32, ctypes.c_float, ctypes.c_float, P]),
            "or_mlp_nparam": (i32, []),
            "or_mlp_forward": (None, [P, P, i32, P]),
            "or_mlp_loss_grad": (f64, [P, P, P, i32, P]),
            "or_adam_step": (None, [P, P, P, P, i32, i32, f64, f64, f64, f64]),
            "or_blocks_per_sm": (i32, [i32] * 6),
            "or_register_bound": (i32, [i32] * 8),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


# ---------------------------------------------------------------- kernels
def bn_stats(x):
    """Per-channel mean and biased variance of an NCHW float32 array."""
    x = _f32(x)
    N, C, H, W = x.shape
    mean = np.zeros(C, np.float64)
    var = np.zeros(C, np.float64)
    lib().or_bn_stats(_p(x), N, C, H * W, _p(mean), _p(var))
    return mean, var


def upsample2x(x):
    """Bilinear x2 upsampling (half-pixel centres) of an (..., H, W) array."""
    x = _f32(x)
    H, W = x.shape[-2:]
    P = int(np.prod(x.shape[:-2]))
    out = np.zeros(x.shape[:-2] + (2 * H, 2 * W), np.float64)
    lib().or_upsample2x(_p(x), P, H, W, _p(out))
    return out


def maxpool3s2p1(x):
    x = _f32(x)
    H, W = x.shape[-2:]
    P = int(np.prod(x.shape[:-2]))
    out = np.zeros(x.shape[:-2] + ((H - 1) // 2 + 1, (W - 1) // 2 + 1), np.float32)
    lib().or_maxpool3s2p1(_p(x), P, H, W, _p(out))
    return out


def im2col3(x):
    x = _f32(x)
    N, C, H, W = x.shape
    out = np.zeros((N, C * 9, H * W), np.float32)
    lib().or_im2col3(_p(x), N, C, H, W, _p(out))
    return out


def hist256(x):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.uint8)).reshape(-1)
    bins = np.zeros(256, np.uint32)
    lib().or_hist256(_p(x), x.size, _p(bins))
    return bins


def philox4x32_10(seed: int, n: int, first: int = 0):
    """n outputs of 4 uint32 words: counter (first+i, 0, 0) under key seed."""
    out = np.zeros((n, 4), np.uint32)
    lib().or_philox4x32_10(seed, first, n, _p(out))
    return out


def poly(x, coef, iters: int = 64, with_bound: bool = False):
    x = _f32(x).reshape(-1)
    c = _f32(coef).reshape(-1)
    assert c.size == 33
    out = np.zeros(x.size, np.float64)
    bound = np.zeros(x.size, np.float64) if with_bound else None
    lib().or_poly(_p(x), x.size, _p(c), iters, _p(out),
                  _p(bound) if with_bound else None)
    return (out, bound) if with_bound else out


def double_to_bf16(v: float) -> int:
    return int(lib().or_double_to_bf16(float(v)))


def bf16_axpy(x_bits, y_bits, alpha: float):
    """x_bits, y_bits: uint16 arrays holding bfloat16 bit patterns."""
    x = np.ascontiguousarray(np.asarray(x_bits, np.uint16)).reshape(-1)
    y = np.ascontiguousarray(np.asarray(y_bits, np.uint16)).reshape(-1)
    out = np.zeros(x.size, np.uint16)
    lib().or_bf16_axpy(_p(x), _p(y), float(alpha), x.size, _p(out))
    return out


def stream_tmpl(x, k: int, a: float, b: float):
    x = _f32(x).reshape(-1)
    assert x.size % 4 == 0
    out = np.zeros(x.size, np.float64)
    lib().or_stream_tmpl(_p(x), x.size, int(k), float(a), float(b), _p(out))
    return out


# ---------------------------------------------------------------- MLP
def mlp_nparam() -> int:
    return int(lib().or_mlp_nparam())


def mlp_forward(params, X):
    P = np.ascontiguousarray(params, np.float64)
    X = _f32(X)
    y = np.zeros(X.shape[0], np.float64)
    lib().or_mlp_forward(_p(P), _p(X), X.shape[0], _p(y))
    return y


def mlp_loss_grad(params, X, Y):
    P = np.ascontiguousarray(params, np.float64)
    X, Y = _f32(X), _f32(Y)
    g = np.zeros(P.size, np.float64)
    loss = lib().or_mlp_loss_grad(_p(P), _p(X), _p(Y), X.shape[0], _p(g))
    return loss, g


def adam_step(params, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam update of float64 arrays params, m, v."""
    g = np.ascontiguousarray(grad, np.float64)
    lib().or_adam_step(_p(params), _p(g), _p(m), _p(v), params.size, int(t),
                       lr, beta1, beta2, eps)


# ---------------------------------------------------------------- Sec. 2.1 / Alg. 2
def blocks_per_sm(sm_regs, sm_smem, sm_threads, threads, regs, smem):
    return int(lib().or_blocks_per_sm(sm_regs, sm_smem, sm_threads, threads, regs, smem))


def register_bound(sm_regs, sm_smem, sm_threads, d1, nregs1, d2, nregs2, smem_fused):
    return int(lib().or_register_bound(sm_regs, sm_smem, sm_threads, d1, nregs1,
                                       d2, nregs2, smem_fused))


def alg2_search(d0: int, profile, bound, step: int = 128):
    """Algorithm 2 (Sec. 3.2) over measured times.

    profile(d1, r) returns the time of the fused kernel with d1 threads for
    the first kernel and register bound r (None = no bound); bound(d1) returns
    the r0 of the register-bound formula for that split.  The loop visits
    d1 = step, 2*step, ... < d0, profiles without a bound then with r0, and
    keeps the first strictly faster configuration.  Returns (d1*, r*, t*)."""
    t_best, d_best, r_best = float("inf"), None, None
    d1 = step
    while d1 < d0:
        t = profile(d1, None)
        if t < t_best:
            t_best, d_best, r_best = t, d1, None
        r0 = bound(d1)
        t = profile(d1, r0)
        if t < t_best:
            t_best, d_best, r_best = t, d1, r0
        d1 += step
    return d_best, r_best, t_best


def regret(times_model_choice: float, times_best: float) -> float:
    """Relative extra time of the model's pick over the exhaustive optimum,
    both read from the same exhaustive table."""
    return times_model_choice / times_best - 1.0


def speedup(t_base: float, t_fused: float):
    """The two readings of 'X% faster': (ratio T_base/T_fused, saving
    (T_base - T_fused)/T_base)."""
    return t_base / t_fused, (t_base - t_fused) / t_base
