"""Host-side arithmetic of the benchmark line: the ideal-overlap bound, the
roofline of its dominant term, and the spread of the timed steps."""
import pytest

import bench

PEAKS = {"ffma": 3.8e13, "imul": 1.32e13, "smem_atomic": 9.66e12, "ialu": 3.0e13}


def test_ideal_is_the_largest_term():
    # 928 MB at 6785.9 GB/s is 136.75 us; 1e9 FMAs at 3.8e13/s is 26.3 us
    t, terms = bench.ideal_us(928.0e6, {"ffma": 1e9}, PEAKS, 6785.9)
    assert t == pytest.approx(136.75, abs=0.01)
    assert terms["hbm"] == pytest.approx(136.75, abs=0.01) and terms["ffma"] == pytest.approx(26.32, abs=0.01)


def test_roofline_follows_the_dominant_term():
    nbytes, hbm = 928.0e6, 6785.9
    # memory-bound: HBM roofline, fraction = ideal / measured
    _, terms = bench.ideal_us(nbytes, {"ffma": 1e9}, PEAKS, hbm)
    r = bench.dominant_roofline(terms, nbytes, {"ffma": 1e9}, PEAKS, 154.9, hbm, "measured", 123)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] == 123
    assert r["frac"] == pytest.approx(136.75 / 154.9, abs=1e-3)
    # FMA-bound: ALU roofline on the FMA pipe, in Tops/s
    ops = {"ffma": 2.214e9}
    _, terms = bench.ideal_us(6.3e6, ops, PEAKS, hbm)
    r = bench.dominant_roofline(terms, 6.3e6, ops, PEAKS, 64.0, hbm, "measured", None)
    assert r["bound"] == "alu" and r["pipe"] == "ffma" and r["unit"] == "Tops/s"
    assert r["achieved"] == pytest.approx(2.214e9 / 64e-6 / 1e12, rel=1e-3)
    assert r["frac"] == pytest.approx(2.214e9 / 3.8e13 / 64e-6, abs=1e-3)


def test_spread():
    s = bench.spread([float(v) for v in range(1, 101)])
    assert s == {"median": 51.0, "p10": 11.0, "p90": 90.0}
    assert bench.spread([7.0]) == {"median": 7.0, "p10": 7.0, "p90": 7.0}


def test_cpu_slices_cover_every_index_once():
    for n in (0, 1, 7, 64, 100, 257):
        for parts in (1, 3, 8, 16):
            r = bench._ranges(n, parts)
            assert [i for lo, hi in r for i in range(lo, hi)] == list(range(n))
            assert len(r) <= parts and all(hi > lo for lo, hi in r)


def test_reference_arm_and_cpu_baseline_time_the_same_sample():
    # both go through cpu_jobs: same jobs, same description
    jobs, scale, desc = bench.cpu_jobs("bn_poly", 4)
    assert scale == 1.0 and "whole workload" in desc
    # 64 channels and 2^20 elements in 4 slices each
    assert len(jobs) == 8
    assert bench.cpu_jobs("bn_poly", 4)[0] is jobs      # drawn once, cached


def test_e2e_record_is_the_median_run():
    link = {"h2d_gbs": 210.0, "d2h_gbs": 192.0, "h2d_alone_us": 5677.0, "d2h_alone_us": 7141.0,
            "both_directions_us": 8016.0}
    r = bench.e2e_record([8209.5, 13153.6, 8190.7], 1191706624, 1373113344, 20, link)
    assert r["value"] == 8209.5 and r["runs_us"] == [8209.5, 13153.6, 8190.7]
    assert r["h2d_bytes_per_step"] == 1191706624 and r["d2h_bytes_per_step"] == 1373113344
    assert r["copy_bound_us"] == 8016.0 and "median of 3 runs of 20 steps" in r["mode"]
