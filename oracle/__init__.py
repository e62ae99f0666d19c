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
  sha256 / sha256d_scan     hashlib.sha256 (applied twice for the scan)
  blake2b / blake2b_scan    hashlib.blake2b
  blake2s       hashlib.blake2s; pins the 32-bit rounds BLAKE-256 shares
  blake256 / blake256_scan  rounds and sigma table pinned through blake2s,
                the pi constants through mpmath; the BLAKE-256 framing
                (constant XOR, counter words, padding) is "parity unpinned":
                no published test vector is within reach
  hash constants  square and cube roots of primes and the digits of pi,
                derived here from their definitions; pinned by the library
                hashes above and by mpmath
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "hf_oracle.c"), os.path.join(_HERE, "hf_oracle_hash.c")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

MLP_IN = 24
MLP_H = 64


def build(force: bool = False) -> str:
    """Compile hf_oracle.c into liboracle.so next to it (plain gcc, no
    contraction of multiply-adds so that the double arithmetic is the one
    written in the source)."""
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    subprocess.check_call([
        "gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
        "-o", tmp] + _SRCS + ["-lm"])
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
            "or_sha256_compress": (None, [P, P, P]),
            "or_sha256": (None, [P, u64, P, P, P]),
            "or_sha256d_scan": (None, [P, ctypes.c_uint32, i64, P, P, P]),
            "or_blake256_compress": (None, [P, P, u64, P]),
            "or_blake256": (None, [P, u64, P, P, P]),
            "or_blake256_scan": (None, [P, ctypes.c_uint32, i64, P, P, P]),
            "or_blake2s": (None, [P, u64, i32, P, P]),
            "or_blake2b": (None, [P, u64, i32, P, P]),
            "or_blake2b_scan": (None, [P, ctypes.c_uint32, i64, P, P]),
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


# ---------------------------------------------------------------- hashes
# Constants of the hash functions, derived from their definitions with exact
# integer arithmetic.
def _primes(n: int):
    ps = []
    k = 2
    while len(ps) < n:
        if all(k % p for p in ps if p * p <= k):
            ps.append(k)
        k += 1
    return ps


def _iroot(x: int, k: int) -> int:
    """floor(x ** (1/k)) of a non-negative integer, by bisection."""
    lo, hi = 0, 1 << (x.bit_length() // k + 1)
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if mid ** k <= x:
            lo = mid
        else:
            hi = mid - 1
    return lo


def sha256_constants():
    """(K, H0) of FIPS 180-4: K_t = the first 32 bits of the fractional part
    of the cube root of the t-th prime (t < 64, Sec. 4.2.2); H0_i = the first
    32 bits of the fractional part of the square root of the i-th prime
    (i < 8, Sec. 5.3.3)."""
    ps = _primes(64)
    K = np.array([_iroot(p << 96, 3) & 0xFFFFFFFF for p in ps], np.uint32)
    H0 = np.array([_iroot(p << 64, 2) & 0xFFFFFFFF for p in ps[:8]], np.uint32)
    return K, H0


def blake2b_iv():
    """BLAKE2b's IV (RFC 7693 Sec. 2.6): the first 64 bits of the fractional
    parts of the square roots of the first eight primes."""
    return np.array([_iroot(p << 128, 2) & 0xFFFFFFFFFFFFFFFF for p in _primes(8)], np.uint64)


def pi_words(nwords: int = 16):
    """The first 32*nwords bits of the fractional part of pi as big-endian
    32-bit words (BLAKE-256's constants), from Machin's formula
    pi = 16 atan(1/5) - 4 atan(1/239) in fixed point with 64 guard bits."""
    bits = 32 * nwords + 64
    one = 1 << bits

    def atan_inv(x):
        total, term, k = 0, one // x, 0
        while term:
            total += term // (2 * k + 1) if k % 2 == 0 else -(term // (2 * k + 1))
            term //= x * x
            k += 1
        return total

    frac = (16 * atan_inv(5) - 4 * atan_inv(239) - 3 * one) >> 64
    return np.array([(frac >> (32 * (nwords - 1 - i))) & 0xFFFFFFFF for i in range(nwords)],
                    np.uint32)


_HASH_CONST = {}


def _hc():
    if not _HASH_CONST:
        K, H0 = sha256_constants()
        _HASH_CONST.update(K=K, H0=H0, U=pi_words(16), B2B=blake2b_iv())
    return _HASH_CONST


def _bytes(msg) -> np.ndarray:
    a = np.frombuffer(bytes(msg), np.uint8).copy()
    return a if a.size else np.zeros(1, np.uint8)


def sha256(msg) -> bytes:
    c, m, out = _hc(), _bytes(msg), np.zeros(32, np.uint8)
    lib().or_sha256(_p(m), len(bytes(msg)), _p(c["K"]), _p(c["H0"]), _p(out))
    return out.tobytes()


def blake256(msg) -> bytes:
    c, m, out = _hc(), _bytes(msg), np.zeros(32, np.uint8)
    lib().or_blake256(_p(m), len(bytes(msg)), _p(c["H0"]), _p(c["U"]), _p(out))
    return out.tobytes()


def blake2s(msg, nn: int = 32) -> bytes:
    c, m, out = _hc(), _bytes(msg), np.zeros(nn, np.uint8)
    lib().or_blake2s(_p(m), len(bytes(msg)), nn, _p(c["H0"]), _p(out))
    return out.tobytes()


def blake2b(msg, nn: int = 32) -> bytes:
    c, m, out = _hc(), _bytes(msg), np.zeros(nn, np.uint8)
    lib().or_blake2b(_p(m), len(bytes(msg)), nn, _p(c["B2B"]), _p(out))
    return out.tobytes()


def _header(header) -> np.ndarray:
    h = np.frombuffer(bytes(header), np.uint8).copy()
    assert h.size == 80
    return h


def sha256d_scan(header, first: int, n: int) -> np.ndarray:
    """[n, 32] digests SHA-256(SHA-256(header)) with the nonce first + i as a
    little-endian uint32 in bytes 76..79 of the 80-byte header."""
    c, h, out = _hc(), _header(header), np.zeros((max(n, 1), 32), np.uint8)
    lib().or_sha256d_scan(_p(h), first, n, _p(c["K"]), _p(c["H0"]), _p(out))
    return out[:n]


def blake256_scan(header, first: int, n: int) -> np.ndarray:
    c, h, out = _hc(), _header(header), np.zeros((max(n, 1), 32), np.uint8)
    lib().or_blake256_scan(_p(h), first, n, _p(c["H0"]), _p(c["U"]), _p(out))
    return out[:n]


def blake2b_scan(header, first: int, n: int) -> np.ndarray:
    c, h, out = _hc(), _header(header), np.zeros((max(n, 1), 32), np.uint8)
    lib().or_blake2b_scan(_p(h), first, n, _p(c["B2B"]), _p(out))
    return out[:n]


def hash_hits(digests: np.ndarray, first: int, target: int) -> np.ndarray:
    """Sorted nonces whose digest bytes 28..31, read as a little-endian
    uint32, are at most target: the scan's acceptance test."""
    w = digests[:, 28:32].copy().view("<u4").reshape(-1)
    idx = np.nonzero(w <= np.uint32(target))[0].astype(np.uint64)
    return np.sort(((idx + np.uint64(first)) & np.uint64(0xFFFFFFFF)).astype(np.uint32))
