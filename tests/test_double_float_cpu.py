"""The double-float addition batch-norm's channel combine uses (Knuth's
TwoSum of the high parts plus the low parts, renormalised), restated with
numpy float32 operations: it must be commutative bit for bit -- the reason
a butterfly leaves the same value on every lane -- and as accurate as the
~48-bit format promises."""
import numpy as np

f32 = np.float32


def df_add(a, b):
    s = f32(a[0] + b[0])
    bb = f32(s - a[0])
    e = f32(f32(a[0] - f32(s - bb)) + f32(b[0] - bb))
    e = f32(e + f32(a[1] + b[1]))
    hi = f32(s + e)
    return hi, f32(e - f32(hi - s))


def test_twosum_error_is_exact():
    rng = np.random.default_rng(0)
    for _ in range(2000):
        a, b = (f32(v) for v in rng.standard_normal(2) * 10.0 ** rng.integers(-6, 7, 2))
        s = f32(a + b)
        bb = f32(s - a)
        e = f32(f32(a - f32(s - bb)) + f32(b - bb))
        # a + b == s + e exactly (checked in float64, which holds both sums)
        assert np.float64(a) + np.float64(b) == np.float64(s) + np.float64(e)


def test_double_float_add_is_commutative_bit_for_bit():
    rng = np.random.default_rng(1)
    for _ in range(5000):
        x = [df_add((f32(v), f32(0)), (f32(w), f32(0))) for v, w in rng.standard_normal((2, 2)) * 1e3]
        assert df_add(x[0], x[1]) == df_add(x[1], x[0])


def test_butterfly_sum_matches_float64():
    # 32 lanes each summing a few FP32 partials, then a 5-level butterfly:
    # every lane ends with the same pair, close to the float64 sum
    rng = np.random.default_rng(2)
    parts = (rng.standard_normal(98) * 1e4).astype(np.float32)
    lanes = []
    for l in range(32):
        acc = (f32(0), f32(0))
        for t in range(l, 98, 32):
            acc = df_add(acc, (parts[t], f32(0)))
        lanes.append(acc)
    for m in (16, 8, 4, 2, 1):
        lanes = [df_add(lanes[l], lanes[l ^ m]) for l in range(32)]
    assert all(v == lanes[0] for v in lanes)
    exact = float(np.sum(parts.astype(np.float64)))
    got = float(lanes[0][0]) + float(lanes[0][1])
    assert abs(got - exact) <= 1e-12 * float(np.sum(np.abs(parts.astype(np.float64))))
