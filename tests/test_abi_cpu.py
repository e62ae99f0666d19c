"""The C-ABI library on the CPU: it loads, exports every entry point that
include/hfuse.h declares, its argument blocks match the binding, and the
host-side validation rejects bad configurations before touching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    from paper_2007_01277_gb300 import build as B
    B.build()
    from paper_2007_01277_gb300 import hfuse
    return hfuse


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(hf_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_exports_every_declared_symbol(H):
    names = declared_functions()
    assert "hf_launch" in names and "hf_fuse" in names and "hf_register_kernel" in names
    lib = ctypes.CDLL(H.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_argument_block_sizes_match(H):
    for body, T in enumerate(H.ARGS_TYPES):
        assert H.lib.hf_args_size(body) == ctypes.sizeof(T), H.BODY_NAMES[body]
    assert H.lib.hf_args_size(99) == 0


def test_status_strings(H):
    for code in H.STATUS:
        assert H.lib.hf_status_string(code)


def test_register_kernel_validation(H):
    with pytest.raises(H.HFError) as e:
        H.hf_register_kernel(42)
    assert e.value.status == -1
    with pytest.raises(H.HFError):
        H.hf_register_kernel(H.POLY, min_threads=48)
    with pytest.raises(H.HFError):
        H.hf_register_kernel(H.POLY, min_threads=512, max_threads=256)
    k = H.hf_register_kernel(H.POLY, 64, 512, 64)
    H.hf_destroy_kernel(k)


@pytest.mark.parametrize("split,d0", [(0, 512), (512, 512), (100, 512), (256, 500), (512, 2048)])
def test_fuse_rejects_bad_splits(H, split, d0):
    a = H.hf_register_kernel(H.BN_STATS)
    b = H.hf_register_kernel(H.POLY)
    with pytest.raises(H.HFError) as e:
        H.hf_fuse(a, b, split, d0, 0)
    assert e.value.status == -2


def test_fuse_respects_kernel_ranges_and_caps(H):
    a = H.hf_register_kernel(H.HIST256, 128, 256, 128)
    b = H.hf_register_kernel(H.PHILOX)
    with pytest.raises(H.HFError) as e:       # 96 threads below hist's minimum
        H.hf_fuse(a, b, 96, 512, 0)
    assert e.value.status == -2
    with pytest.raises(H.HFError) as e:       # 192 not a multiple of its 128 step
        H.hf_fuse(a, b, 192, 512, 0)
    assert e.value.status == -2
    with pytest.raises(H.HFError) as e:
        H.hf_fuse(a, b, 128, 512, 33)
    assert e.value.status == -6


def test_fuse_checked_validation(H):
    # the checked build validates like hf_fuse and exists only for pairs
    # whose bodies have barriers; both are decided before any CUDA call
    a, b = H.hf_register_kernel(H.HIST256), H.hf_register_kernel(H.PHILOX)
    with pytest.raises(H.HFError) as e:
        H.hf_fuse_checked(a, b, 100, 512)
    assert e.value.status == -2
    u, m = H.hf_register_kernel(H.UPSAMPLE2X), H.hf_register_kernel(H.MAXPOOL3S2)
    with pytest.raises(H.HFError) as e:
        H.hf_fuse_checked(u, m, 256, 512)
    assert e.value.status == -6


def test_fuse_n_validation(H):
    ks = [H.hf_register_kernel(H.POLY) for _ in range(3)]
    with pytest.raises(H.HFError) as e:       # 16 intervals: only 15 barrier ids
        H.hf_fuse_n(ks[:1] * 16, list(range(16)), [32] * 16)
    assert e.value.status in (-3, -1)
    with pytest.raises(H.HFError) as e:
        H.hf_fuse_n(ks, [0, 1, 1], [512, 512, 64])          # block > 1024
    assert e.value.status == -2
    with pytest.raises(H.HFError) as e:
        H.hf_fuse_n(ks, [0, 0, 0], [256, 256])              # interval 1 idle
    assert e.value.status == -1


def test_regcaps(H):
    caps = H.hf_regcaps()
    assert caps == sorted(caps) and {32, 40, 48, 64, 96} <= set(caps)


def test_register_bound_host_arithmetic(H, orc):
    """The library's Algorithm 2 bound agrees with the oracle's on the
    paper's worked numbers and on a sweep."""
    lim = H.DeviceLimits(152, 65536, 98304, 2048, 232448, 0, 10, 3)
    assert H.hf_register_bound(lim, 896, 32, 128, 32, 1024) == 32
    for d1 in range(128, 1024, 128):
        for r1 in (24, 32, 40, 64, 96):
            for r2 in (16, 32, 72):
                for sm in (0, 1024, 40000):
                    want = orc.register_bound(65536, 98304, 2048, d1, r1, 1024 - d1, r2, sm)
                    assert H.hf_register_bound(lim, d1, r1, 1024 - d1, r2, sm) == want


def test_template_features_hand_example(H):
    """hf_tmpl_features on a hand-computed pair (host arithmetic only)."""
    import math
    a = H.StreamTmplArgs(None, None, 1 << 20, 4, 2, 4096, 0.999, 0.001)
    b = H.StreamTmplArgs(None, None, 1 << 28, 0, 0, 0, 0.999, 0.001)
    f = H.hf_tmpl_features(a, b, 64, 256, 0, 2, 40, 0, 6785.9, 3.8e13)
    assert len(f) == 24
    ta = max(8 * 2 ** 20 / 6785.9e9, 4 * 2 ** 20 / 4 / 3.8e13) * 1e6
    tb = 8 * 2 ** 28 / 6785.9e9 * 1e6
    want_a = [20 / 28, math.log2(5) / 8, 0.5, 4096 / 49152, math.log2(1 + ta) / 12,
              (2 ** 20 / 3.8e13) / (8 * 2 ** 20 / 6785.9e9 + 2 ** 20 / 3.8e13), 64 / 256,
              2 * 2 / 64, ta / (ta + tb)]
    want_b = [1.0, 0.0, 0.0, 0.0, math.log2(1 + tb) / 12, 0.0, 192 / 256, 6 * 2 / 64, tb / (ta + tb)]
    want_c = [1.0, 0.5, 0.25, 40 / 255, 0.0, 4096 * 2 / 233472]
    assert f == pytest.approx(want_a + want_b + want_c, rel=1e-5, abs=1e-7)
    with pytest.raises(H.HFError):
        H.hf_tmpl_features(a, b, 0, 256, 0, 2, 40, 0, 6785.9, 3.8e13)


def test_ring_plan_geometry(H):
    """Stream rings: about 40 KB in flight per SM over the SM's stream-ring
    warps, in stages of 1, 2 or 4 KB, 2 to 4 per warp; below a body's
    minimum share it drops its ring and the share is recomputed over the
    rest.  Item rings: two stages of the item size, outside that share."""
    S, I = H.RING_STREAM, H.RING_ITEM
    # 8 ring warps: 5 KB per warp -> 4 KB stages, 2 of them
    assert H.hf_ring_plan([8], [S], [1024], 1) == ([4096], [2], [1])
    # 4 warps: 10 KB per warp -> 4 KB stages, 1 + round(2.5) = 4 (the cap)
    assert H.hf_ring_plan([4], [S], [1024], 1) == ([4096], [4], [1])
    # 2 warps: 20 KB per warp -> still 4 stages of 4 KB
    assert H.hf_ring_plan([2], [S], [1024], 1) == ([4096], [4], [1])
    # 32 warps: 1.25 KB -> 1 KB stages, 2 of them
    assert H.hf_ring_plan([16], [S], [1024], 2) == ([1024], [2], [1])
    # 64 warps: 640 B per warp, below 1 KB -> register loads
    assert H.hf_ring_plan([16], [S], [1024], 4) == ([0], [0], [0])
    # two ring intervals of 16 warps: 1.25 KB each misses the second one's
    # 2 KB minimum; it drops out and the first gets 2.5 KB -> 2 KB stages
    assert H.hf_ring_plan([16, 16], [S, S], [1024, 2048], 1) == ([2048, 0], [2, 0], [1, 0])
    # intervals without a ring never get one
    assert H.hf_ring_plan([4, 28], [0, S], [1024, 1024], 1) == ([0, 1024], [0, 2], [0, 1])
    # an item interval keeps two 4 KB stages whatever the warps and does not
    # count against the stream share: 8 stream warps still get 5 KB each
    assert H.hf_ring_plan([16, 8], [I, S], [4096, 1024], 2) == ([4096, 2048], [2, 2], [1, 1])
    assert H.hf_ring_plan([4, 8], [I, S], [4000, 1024], 1) == ([4096, 4096], [2, 2], [1, 1])
    with pytest.raises(H.HFError):
        H.hf_ring_plan([4], [S], [1024], 0)
    with pytest.raises(H.HFError):
        H.hf_ring_plan([4], [3], [1024], 1)


def test_pair_features_reduce_to_template_features(H):
    """hf_pair_features generalises hf_tmpl_features: on two stream
    templates the 24 features agree bit for bit (host arithmetic only)."""
    import random
    rng = random.Random(7)
    kt1, kt2 = H.hf_register_kernel(H.STREAM_TMPL), H.hf_register_kernel(H.STREAM_TMPL)
    pk = H.pipe_peaks(6785.9, 3.8e13, 1.75e13, 9.66e12, 3.0e13)
    for _ in range(200):
        def spec():
            return H.StreamTmplArgs(None, None, 4 * rng.randint(1, 1 << 26), rng.choice([0, 1, 2, 4, 64, 256]),
                                    rng.randint(0, 4), 16 * rng.randint(0, 3072), 0.999, 0.001)
        a, b = spec(), spec()
        d0 = rng.choice([256, 512, 1024])
        split = 32 * rng.randint(1, d0 // 32 - 1)
        cap, bps = rng.choice([0, 32, 64, 96]), rng.randint(1, 4)
        regs, spill = rng.randint(24, 255), rng.choice([0, 16, 400])
        want = H.hf_tmpl_features(a, b, split, d0, cap, bps, regs, spill, 6785.9, 3.8e13)
        got = H.hf_pair_features(kt1, kt2, [a, b], split, d0, cap, bps, regs, spill, pk)
        assert got == want


def test_body_work_hand_values(H):
    """Algorithmic bytes and operations of one launch, worked by hand."""
    w = H.hf_body_work_of(H.BN_STATS, H.BnStatsArgs(None, None, None, 2, 3, 16, None))
    assert (w["bytes"], w["ffma"]) == (4 * 96 + 8 * 3, 2 * 96)
    w = H.hf_body_work_of(H.UPSAMPLE2X, H.Upsample2xArgs(None, None, 2, 4, 8))
    assert w["bytes"] == 4 * 64 + 16 * 64
    w = H.hf_body_work_of(H.MAXPOOL3S2, H.Maxpool3s2Args(None, None, 1, 5, 7))   # 5x7 -> 3x4
    assert w["bytes"] == 4 * 35 + 4 * 12
    w = H.hf_body_work_of(H.IM2COL3, H.Im2col3Args(None, None, 1, 2, 3, 4))
    assert w["bytes"] == 4 * 24 * 10
    w = H.hf_body_work_of(H.HIST256, H.Hist256Args(None, None, 1000))
    assert (w["bytes"], w["smem_atomic"], w["barriers"]) == (2024, 1000, 2)
    w = H.hf_body_work_of(H.PHILOX, H.PhiloxArgs(None, 10, 0, 0))
    assert (w["bytes"], w["imul"]) == (160, 400)
    w = H.hf_body_work_of(H.POLY, H.PolyArgs(None, None, 100, 64))
    assert (w["bytes"], w["ffma"]) == (800, 100 * 64 * 33)
    w = H.hf_body_work_of(H.BF16_AXPY, H.Bf16AxpyArgs(None, None, None, 50, 0.5))
    assert w["bytes"] == 300
    w = H.hf_body_work_of(H.STREAM_TMPL, H.StreamTmplArgs(None, None, 64, 8, 3, 0, 1.0, 0.0))
    assert (w["bytes"], w["ffma"], w["barriers"]) == (512, 128, 3)
