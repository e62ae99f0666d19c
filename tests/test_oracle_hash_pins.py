"""Pins of the hash oracle (the SHA256 / Blake256 / Blake2B kernels of
Sec. 4.1) against things other than itself: Python's hashlib (SHA-256,
BLAKE2b, BLAKE2s), mpmath for the constants, and properties of the scan."""
import hashlib
import struct

import numpy as np
import pytest

import oracle
from paper_2007_01277_gb300 import workloads as W

# message lengths around every block and padding boundary of 64- and
# 128-byte blocks (55/56: the SHA length field no longer fits; 111/112 the
# same for 128-byte blocks)
LENGTHS = (0, 1, 3, 32, 55, 56, 57, 63, 64, 65, 80, 111, 112, 119, 120, 127, 128, 129, 191, 192, 300)


def _msgs():
    rng = np.random.default_rng(7)
    return [rng.integers(0, 256, n, dtype=np.uint8).tobytes() for n in LENGTHS]


def test_sha256_matches_hashlib():
    for m in _msgs():
        assert oracle.sha256(m) == hashlib.sha256(m).digest(), len(m)


def test_blake2b_matches_hashlib():
    for m in _msgs():
        assert oracle.blake2b(m, 64) == hashlib.blake2b(m).digest(), len(m)
        assert oracle.blake2b(m, 32) == hashlib.blake2b(m, digest_size=32).digest(), len(m)


def test_blake2s_matches_hashlib():
    # BLAKE2s runs the same 32-bit rounds (G, rotations 16/12/8/7, the
    # column/diagonal order and the sigma table) as BLAKE-256 with the
    # constant XOR switched off: this pins that shared code
    for m in _msgs():
        assert oracle.blake2s(m) == hashlib.blake2s(m).digest(), len(m)
        assert oracle.blake2s(m, 16) == hashlib.blake2s(m, digest_size=16).digest(), len(m)


def test_hash_constants_match_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 700
    K, H0 = oracle.sha256_constants()
    primes = [p for p in range(2, 400) if all(p % q for q in range(2, int(p ** 0.5) + 1))][:64]
    for t, p in enumerate(primes):
        frac = mpmath.cbrt(p) - mpmath.floor(mpmath.cbrt(p))
        assert int(K[t]) == int(mpmath.floor(frac * 2 ** 32)), t
    for i, p in enumerate(primes[:8]):
        frac = mpmath.sqrt(p) - mpmath.floor(mpmath.sqrt(p))
        assert int(H0[i]) == int(mpmath.floor(frac * 2 ** 32)), i
        assert int(oracle.blake2b_iv()[i]) == int(mpmath.floor(frac * 2 ** 64)), i
    U = oracle.pi_words(16)
    f = int(mpmath.floor((mpmath.pi - 3) * mpmath.mpf(2) ** 512))
    assert [int(u) for u in U] == [(f >> (32 * (15 - i))) & 0xFFFFFFFF for i in range(16)]


def _with_nonce(header, nonce):
    return header[:76] + struct.pack("<I", nonce & 0xFFFFFFFF)


def test_sha256d_scan_is_double_sha256_with_the_nonce():
    header = W.hash_header(3)
    first = 0xFFFFFFF0   # the nonce wraps past 2^32 - 1
    d = oracle.sha256d_scan(header, first, 40)
    for i in range(40):
        h = _with_nonce(header, first + i)
        assert d[i].tobytes() == hashlib.sha256(hashlib.sha256(h).digest()).digest(), i


def test_blake2b_scan_matches_hashlib():
    header = W.hash_header(4)
    d = oracle.blake2b_scan(header, 12345, 40)
    for i in range(40):
        h = _with_nonce(header, 12345 + i)
        assert d[i].tobytes() == hashlib.blake2b(h, digest_size=32).digest(), i


def test_blake256_scan_hashes_the_header_with_each_nonce():
    header = W.hash_header(5)
    d = oracle.blake256_scan(header, 77, 16)
    for i in range(16):
        assert d[i].tobytes() == oracle.blake256(_with_nonce(header, 77 + i)), i
    # distinct nonces give distinct digests; the header's own nonce bytes
    # are ignored
    assert len({r.tobytes() for r in d}) == 16
    other = header[:76] + b"\xde\xad\xbe\xef"
    assert np.array_equal(oracle.blake256_scan(other, 77, 16), d)


def test_blake256_distinguishes_padding_cases():
    # messages that differ only in length (zero bytes appended) must hash
    # differently: the length field, the final 1 bit and the counter rule
    # all separate them, including the 55-byte case where the two padding
    # bits share one byte and the 64-byte case whose last block holds no
    # message bit
    seen = set()
    for n in range(0, 130):
        seen.add(oracle.blake256(bytes(n)))
    assert len(seen) == 130


def test_hash_hits_brute_force():
    rng = np.random.default_rng(0)
    d = rng.integers(0, 256, (500, 32), dtype=np.uint8)
    target = 1 << 28
    got = oracle.hash_hits(d, 1000, target)
    want = [1000 + i for i in range(500) if int.from_bytes(d[i, 28:32].tobytes(), "little") <= target]
    assert got.tolist() == want
    assert oracle.hash_hits(d, 0, 0xFFFFFFFF).size == 500
    # nonces wrap modulo 2^32 and the set comes back sorted after the wrap
    got = oracle.hash_hits(d, 0xFFFFFF00, target)
    assert got.tolist() == sorted((0xFFFFFF00 + i) % (1 << 32) for i in range(500)
                                  if int.from_bytes(d[i, 28:32].tobytes(), "little") <= target)
