"""GPU tests of the runtime around the kernels: CUDA-graph capture, the N-way
autotuner, Algorithm 2 and the exhaustive profile, pipe calibration and the
bounded stream wait -- all through the C ABI."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from gpu_util import DEV, check_bn, check_poly  # noqa: E402
from paper_2007_01277_gb300 import hfuse as H  # noqa: E402
from paper_2007_01277_gb300 import workloads as W  # noqa: E402


def _bn_poly():
    x = W.bn_input((4, 16, 24, 24)).to(DEV)
    px = W.poly_input(1 << 15).to(DEV)
    coef = W.poly_coefficients().numpy()
    m, v, y = torch.empty(16, device=DEV), torch.empty(16, device=DEV), torch.empty_like(px)
    ws = H.bn_stats_workspace(x)
    args = [H.bn_stats_args(x, m, v, ws), H.poly_args(px, y, coef)]
    return x, px, coef, (m, v, y, ws), args


def test_graph_replay_matches_eager_launch():
    x, px, coef, (m, v, y, _ws), args = _bn_poly()
    f = H.hf_fuse(H.hf_register_kernel(H.BN_STATS), H.hf_register_kernel(H.POLY), 256, 512, 0)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        H.hf_launch(f, args, 0, s)
        torch.cuda.synchronize()
        ref = [t.clone() for t in (m, v, y)]
        for t in (m, v, y):
            t.zero_()
        torch.cuda.synchronize()
        H.hf_graph_begin(s)
        H.hf_launch(f, args, 0, s)
        g = H.hf_graph_end(s)
        for _ in range(3):
            H.hf_graph_launch(g, s)
        torch.cuda.synchronize()
    for a, b in zip(ref, (m, v, y)):
        assert torch.equal(a, b)
    check_bn(x.cpu(), m, v)
    check_poly(px.cpu(), coef, y)
    H.hf_graph_destroy(g)


def test_autotune_nway_plan_is_valid_and_correct():
    x, px, coef, (m, v, y, _ws), bp_args = _bn_poly()
    xh = W.hist_input(1 << 20).to(DEV)
    bins = torch.zeros(256, dtype=torch.int32, device=DEV)
    po = torch.empty((1 << 14, 4), dtype=torch.int32, device=DEV)
    args = bp_args + [H.hist256_args(xh, bins), H.philox_args(po, 5)]
    ks = [H.hf_register_kernel(b) for b in (H.BN_STATS, H.POLY, H.HIST256, H.PHILOX)]
    plan, single = H.hf_autotune_nway(ks, args, max_evals=20, reps=2)
    assert len(single) == 4 and all(t > 0 for t in single)
    n_int = plan["n_intervals"]
    # the tuner's seeds use blocks of 512, 768 or 1024 threads
    assert 1 <= n_int <= 4 and sum(plan["interval_threads"]) in (512, 768, 1024)
    assert all(t % 32 == 0 and t > 0 for t in plan["interval_threads"])
    assert set(plan["interval_of"]) == set(range(n_int))
    # the seeds (at most 3 block sizes x 5 caps x 2 packings) and the final
    # re-timing of at most 5 finalists are always done
    assert plan["time_us"] > 0 and plan["evals"] <= 20 + 30 + 5
    f = H.hf_fuse_n(ks, plan["interval_of"], plan["interval_threads"], plan["regcap"])
    bins.zero_()
    H.hf_launch(f, args, plan["grid"])
    torch.cuda.synchronize()
    check_bn(x.cpu(), m, v)
    check_poly(px.cpu(), coef, y)
    assert np.array_equal(bins.cpu().numpy().view(np.uint32), oracle.hist256(xh.cpu().numpy()))
    assert np.array_equal(po.cpu().numpy().view(np.uint32), oracle.philox4x32_10(5, 1 << 14))


def test_profile_pair_and_alg2():
    x, px, coef, (m, v, y, _ws), args = _bn_poly()
    ka, kb = H.hf_register_kernel(H.BN_STATS), H.hf_register_kernel(H.POLY)
    table = H.hf_profile_pair(ka, kb, args, 512, [128, 256, 384], [0, 64], [1, 2], reps=2)
    assert len(table) == 12
    ok = [p for p in table if p["status"] == 0]
    assert ok and all(p["time_us"] > 0 for p in ok)
    assert all(p["grid"] == p["blocks_per_sm"] * H.hf_device_info().sm_count for p in ok)
    best, trace = H.hf_search_alg2(ka, kb, args, 512, step=128, reps=2)
    assert best["split"] in (128, 256, 384) and best["time_us"] > 0
    assert best["time_us"] == min(p["time_us"] for p in trace if p["status"] == 0)
    # the visited splits follow Algorithm 2: ascending, unbounded before bounded
    splits = [p["split"] for p in trace]
    assert splits == sorted(splits)


def test_autotune_modes():
    x, px, coef, (m, v, y, _ws), args = _bn_poly()
    ka, kb = H.hf_register_kernel(H.BN_STATS), H.hf_register_kernel(H.POLY)
    ex = H.hf_autotune(ka, kb, args, 256, H.TUNE_EXHAUSTIVE, reps=2)
    a2 = H.hf_autotune(ka, kb, args, 256, H.TUNE_ALG2, reps=2)
    for p in (ex, a2):
        assert p["status"] == 0 and p["time_us"] > 0 and p["split"] % 32 == 0 and 0 < p["split"] < 256
    assert ex["regcap"] in [0] + H.hf_regcaps()
    # the exhaustive table contains Algorithm 2's candidates: its pick is no
    # slower, up to timing noise
    assert ex["time_us"] <= 1.2 * a2["time_us"]
    # the returned point launches and computes the same result
    f = H.hf_fuse(ka, kb, ex["split"], 256, ex["regcap"])
    H.hf_launch(f, args, ex["grid"])
    torch.cuda.synchronize()
    check_poly(px.cpu(), coef, y.cpu())
    check_bn(x.cpu(), m, v)
    with pytest.raises(H.HFError):
        H.hf_autotune(ka, kb, args, 256, 7)


def test_calibration_in_plausible_range():
    lim = H.hf_device_info()
    ffma = H.hf_calibrate(H.CAL_FFMA)
    # between 20% and 110% of 128 FMA/clk/SM at 2.1 GHz
    nominal = lim.sm_count * 128 * 2.1e9
    assert 0.2 * nominal < ffma < 1.1 * nominal
    assert H.hf_calibrate(H.CAL_IMUL) > 0
    assert H.hf_calibrate(H.CAL_SMEM_ATOMIC) > 0
    # at most 128 integer ALU lanes per SM per clock
    assert 0.05 * nominal < H.hf_calibrate(H.CAL_IALU) < 1.1 * nominal
    with pytest.raises(H.HFError):
        H.hf_calibrate(4)


def test_stream_wait_times_out_on_long_kernel():
    """A launch-timeout check without any fault: a long polynomial chain
    is still running after 1 ms, then completes within the larger limit."""
    k = H.hf_register_kernel(H.POLY)
    x = torch.rand(1 << 22, device=DEV)
    y = torch.empty_like(x)
    s = torch.cuda.Stream()
    a = H.poly_args(x, y, [0.01] * 33, iters=4000)
    torch.cuda.synchronize()
    H.hf_launch_single(k, a, 256, 152, s)
    with pytest.raises(H.HFError) as e:
        H.hf_stream_wait(s, 1)
    assert e.value.status == -8
    H.hf_stream_wait(s, 60000)


def test_bounded_wait_expires_and_sets_the_error_word():
    """A device-side wait that nothing completes gives up after its limit and
    reports it through the error word; the context stays usable."""
    torch.cuda.synchronize()
    H.hf_check_device_error(clear=True)
    H.hf_selftest_wait_timeout(2000)
    torch.cuda.synchronize()
    assert H.hf_check_device_error(clear=True) & H.ERR_WAIT_EXPIRED
    assert H.hf_check_device_error() == 0
    x = torch.arange(1024, dtype=torch.float32, device="cuda")
    assert float(x.sum().item()) == 1023 * 1024 / 2
    with pytest.raises(H.HFError):
        H.hf_selftest_wait_timeout(0)


@pytest.mark.parametrize("warps", [1, 4, 32])
def test_soft_barrier_completes_with_every_warp(warps):
    """The bounded software barrier: every round completes when all warps
    arrive, and no error is reported."""
    torch.cuda.synchronize()
    H.hf_check_device_error(clear=True)
    done = torch.zeros(1, dtype=torch.int32, device="cuda")
    H.hf_selftest_barrier(warps, -1, 50, 500000, done)
    torch.cuda.synchronize()
    assert int(done.item()) == 50 * warps
    assert H.hf_check_device_error() == 0


def test_soft_barrier_gives_up_on_a_missing_warp():
    """A barrier count that is never reached (one warp skips it) ends in a
    bounded time with bit 2 of the error word instead of a hang; the context
    stays usable."""
    torch.cuda.synchronize()
    H.hf_check_device_error(clear=True)
    done = torch.zeros(1, dtype=torch.int32, device="cuda")
    H.hf_selftest_barrier(8, 3, 5, 2000, done)
    torch.cuda.synchronize()
    assert int(done.item()) == 0
    assert H.hf_check_device_error(clear=True) & H.ERR_BARRIER_EXPIRED
    assert H.hf_check_device_error() == 0
    x = torch.arange(1024, dtype=torch.float32, device="cuda")
    assert float(x.sum().item()) == 1023 * 1024 / 2
    for bad in ((0, -1, 1, 10), (33, -1, 1, 10), (4, 4, 1, 10), (4, -1, 0, 10), (4, -1, 1, 0)):
        with pytest.raises(H.HFError):
            H.hf_selftest_barrier(*bad)


def _snapped_bound(ka, kb, args, d1, d0, lim, caps):
    """The bound Algorithm 2 attaches to split d1 (Sec. 3.2): r0 from the
    oracle's register-bound formula with the registers of each kernel
    compiled alone and the fused kernel's shared memory, snapped down to
    the nearest compiled cap (None when no cap lies at or below r0)."""
    ra = H.hf_query_single(ka, args[0], d1)["regs"]
    rb = H.hf_query_single(kb, args[1], d0 - d1)["regs"]
    f0 = H.hf_fuse(ka, kb, d1, d0, 0)
    smem = H.hf_query(f0, args)["smem_bytes"]
    H.hf_destroy_fused(f0)
    r0 = oracle.register_bound(lim.regs_per_sm, lim.smem_per_sm, lim.threads_per_sm, d1, ra,
                               d0 - d1, rb, smem)
    below = [c for c in caps if c <= r0]
    return max(below) if below else None


@pytest.mark.parametrize("d0,step", [(512, 128), (256, 64)])
def test_alg2_pick_matches_oracle_search_on_its_own_trace(d0, step):
    """hf_search_alg2's measured trace fed to oracle.alg2_search and to a
    brute-force argmin: the visited (split, bound) sequence, r0 and the
    pick (tie rule included) must agree exactly."""
    x, px, coef, (m, v, y, _ws), args = _bn_poly()
    ka, kb = H.hf_register_kernel(H.BN_STATS), H.hf_register_kernel(H.POLY)
    lim = H.hf_device_info()
    caps = H.hf_regcaps()
    best, trace = H.hf_search_alg2(ka, kb, args, d0, step=step, reps=2)
    bounds = {d1: _snapped_bound(ka, kb, args, d1, d0, lim, caps) for d1 in range(step, d0, step)}
    # every split unbounded, then (if a compiled cap lies at or below r0) bounded
    want = []
    for d1 in range(step, d0, step):
        want.append((d1, 0))
        if bounds[d1] is not None:
            want.append((d1, bounds[d1]))
    assert [(p["split"], p["regcap"]) for p in trace] == want
    inf = float("inf")
    times = {(p["split"], p["regcap"]): (p["time_us"] if p["status"] == 0 else inf) for p in trace}
    d_o, r_o, t_o = oracle.alg2_search(
        d0, lambda d1, r: times.get((d1, 0 if r is None else r), inf), lambda d1: bounds[d1], step)
    assert (best["split"], best["regcap"], best["time_us"]) == (d_o, 0 if r_o is None else r_o, t_o)
    # brute force: the first point of the trace with the smallest time
    first_min = min(range(len(trace)), key=lambda i: (times[(trace[i]["split"], trace[i]["regcap"])], i))
    assert (trace[first_min]["split"], trace[first_min]["regcap"]) == (best["split"], best["regcap"])
    # Algorithm 2's candidates at the blocks/SM it launches with are points of
    # the exhaustive grid: the exhaustive table's argmin is never slower than
    # the oracle's Algorithm 2 run over that same table
    splits = list(range(step, d0, step))
    cap_set = sorted({0} | {c for c in bounds.values() if c is not None})
    table = H.hf_profile_pair(ka, kb, args, d0, splits, cap_set, [1, 2, 3, 4], reps=2)
    ok = [p for p in table if p["status"] == 0]
    occ = {}
    for p in ok:
        k = (p["split"], p["regcap"])
        if k not in occ or p["blocks_per_sm"] > occ[k]["blocks_per_sm"]:
            occ[k] = p
    _d, _r, t_tab = oracle.alg2_search(
        d0, lambda d1, r: occ[(d1, 0 if r is None else r)]["time_us"] if (d1, 0 if r is None else r) in occ
        else inf, lambda d1: bounds[d1], step)
    assert min(p["time_us"] for p in ok) <= t_tab
