"""Benchmark of the horizontally fused hot path on one GB300.

Default workload: eight uneven kernels in one persistent launch captured in a
CUDA graph -- batch-norm statistics of FP32 64x256x56x56, im2col 3x3 of
32x64x56x56, 3x3/s2/p1 max pooling of 32x128x112x112, bilinear x2 upsampling
of 32x64x128x128, a 256-bin histogram of 2^26 bytes, 2^24 Philox4x32-10
blocks, a 64-step degree-32 Horner chain on 2^22 floats and a bf16 scale+add
of 2^27 elements.  One step = one graph launch of the autotuned fused plan
over all eight.  Reported beside the fused time: the same kernels back to
back on one stream and on eight concurrent streams (the native baseline of
Sec. 4.1), the ideal-overlap bound max(total bytes / HBM bandwidth, ops /
pipe peak), and three fused pairs measured the same way (fused vs serial vs
two streams): batch-norm + polynomial (memory+compute, small), histogram +
Philox (memory+compute) and upsample + max pool (memory+memory), each with
the exhaustive search, Algorithm 2 (Sec. 3.2) and the naive even split.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload nway8|<pair>|cost_model|table2|ratio_sweep]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2007_01277_gb300 import workloads as _W  # noqa: E402  (seeded input recipes)

METRIC = ("fused vs serial/2-stream time (µs), % of ideal-overlap roofline, model regret")
UP_SHAPE = (32, 64, 128, 128)
POOL_SHAPE = (32, 128, 112, 112)
WORKLOAD = ("upsample2x FP32 32x64x128x128 ~U(0,1) + maxpool3x3s2p1 FP32 32x128x112x112 "
            "~N(0,1), fused in one launch")


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def algorithmic_bytes():
    n_up_in = 32 * 64 * 128 * 128
    n_pool_in = 32 * 128 * 112 * 112
    return 4 * (n_up_in * 5 + n_pool_in + n_pool_in // 4)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """Samples the SM clock and the clock-event reasons every millisecond
    while the timed region runs, through read-only NVML queries (ctypes on
    libnvidia-ml); nvidia-smi at 50 ms if NVML cannot be loaded."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_device):
        self.dev = torch_device
        self.samples = []
        self.max_mhz = None
        self.reasons = set()
        self.stop = threading.Event()
        self.nvml = None
        self.proc = None

    def _open_nvml(self):
        import ctypes
        import torch
        L = ctypes.CDLL("libnvidia-ml.so.1")
        if L.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        h = ctypes.c_void_p()
        pr = torch.cuda.get_device_properties(self.dev)
        bus = "%08X:%02X:%02X.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        if L.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) != 0:
            raise OSError("no NVML handle for " + bus)
        self.L, self.h, self.ct = L, h, ctypes
        m = ctypes.c_uint()
        if L.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(m)) == 0:
            self.max_mhz = float(m.value)
        self.nvml = True

    def _poll_nvml(self):
        c, r = self.ct.c_uint(), self.ct.c_ulonglong()
        get_r = getattr(self.L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.L.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop.is_set():
            if self.L.nvmlDeviceGetClockInfo(self.h, 1, self.ct.byref(c)) == 0:
                self.samples.append(float(c.value))
            if get_r(self.h, self.ct.byref(r)) == 0:
                for bit, name in self.REASONS.items():
                    if r.value & bit:
                        self.reasons.add(name)
            time.sleep(0.001)

    def _poll_smi(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            try:
                self.samples.append(float(parts[0]))
                self.max_mhz = float(parts[1])
            except (ValueError, IndexError):
                continue
            for nm, v in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                              "sw_power_cap"], parts[2:6]):
                if v.lower() == "active":
                    self.reasons.add(nm)

    def __enter__(self):
        try:
            self._open_nvml()
            self.t = threading.Thread(target=self._poll_nvml, daemon=True)
        except OSError:
            import torch
            idx = os.environ.get("CUDA_VISIBLE_DEVICES", str(torch.cuda.current_device())).split(",")[0]
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", idx, "--query-gpu=clocks.sm,clocks.max.sm,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._poll_smi, daemon=True)
        self.t.start()
        time.sleep(0.005)
        return self

    def __exit__(self, *exc):
        self.stop.set()
        if self.proc is not None:
            self.proc.terminate()
        self.t.join(timeout=5)

    def summary(self):
        s = self.samples
        return {"sm_mhz": statistics.median(s) if s else None, "sm_max_mhz": self.max_mhz,
                "reasons": sorted(self.reasons), "samples": len(s),
                "source": "nvml" if self.nvml else "nvidia-smi"}


# ------------------------------------------------------------------ workloads
def _mb(n):
    return n / 1e6


PAIR_SPECS = {
    # bilinear x2 of 32x64x128x128 + 3x3/s2/p1 max pool of 32x128x112x112
    "upsample_maxpool": dict(d0=512, splits=(128, 256, 384), caps=(0, 40, 48, 64, 96), bps=(1, 2, 3),
                             flush=False, name="fused_upsample_maxpool",
                             desc=WORKLOAD),
    # 2^28-byte histogram + 2^26 Philox4x32-10 blocks
    "hist_philox": dict(d0=256, splits=tuple(range(32, 256, 32)), caps=(0, 32, 40, 48, 64, 96),
                        bps=(1, 2, 3, 4), flush=False, name="fused_hist_philox",
                        desc="hist256 of 2^28 u8 ~U[0,255] + Philox4x32-10 producing 2^26 blocks "
                             "(seed 0), fused in one launch"),
    # batch-norm stats of 8x64x32x32 + 64-step degree-32 Horner chain on 2^20
    "bn_poly": dict(d0=512, splits=(128, 256, 384), caps=(0, 32, 40, 48, 64, 96), bps=(1, 2, 3, 4),
                    flush=True, name="fused_bn_poly",
                    desc="bn stats FP32 8x64x32x32 ~N(0,1) + 64x degree-32 Horner on 2^20 FP32 "
                         "~U(-1,1), fused in one launch"),
}
# the compute+compute pairs of the three hash scans (Sec. 4.2's negative
# case): each scan over one random 80-byte header, sized to ~2 ms alone
_HP = _W.WORKLOADS["hash_pairs"]
HASH_N = {h: _HP[h + "_n"] for h in ("sha256d", "blake256", "blake2b")}
# 32-bit integer operations per hash as the definitions state them (a
# three-input add or XOR counts once, a rotate once, a 64-bit operation
# twice): SHA-256 compression 64 x 14 + 48 x 10 = 1376, two per nonce;
# BLAKE-256 14 rounds x 8 G x 14; BLAKE2b 12 rounds x 8 G x 22
HASH_OPS = {"sha256d": 2 * 1376, "blake256": 14 * 8 * 14, "blake2b": 12 * 8 * 22}
for _a, _b in (("sha256d", "blake256"), ("sha256d", "blake2b"), ("blake256", "blake2b")):
    PAIR_SPECS[_a + "_" + _b] = dict(
        d0=512, splits=tuple(range(64, 512, 64)), caps=(0, 48, 64, 96), bps=(1, 2, 3, 4), flush=True,
        name="fused_%s_%s" % (_a, _b), hashes=(_a, _b),
        desc="%s nonce scan (%d nonces) + %s nonce scan (%d nonces) of a random 80-byte header, "
             "fused in one launch" % (_a, HASH_N[_a], _b, HASH_N[_b]))


def make_pair(name, H, W, dev):
    """(body ids, arg blocks, tensors, algorithmic bytes, pipe ops, host inputs, outputs)."""
    import torch
    if name == "upsample_maxpool":
        xu_h = W.upsample_input(UP_SHAPE).pin_memory()
        xp_h = W.maxpool_input(POOL_SHAPE).pin_memory()
        xu, xp = xu_h.to(dev), xp_h.to(dev)
        yu = torch.empty(UP_SHAPE[:2] + (256, 256), device=dev)
        yp = torch.empty(POOL_SHAPE[:2] + (56, 56), device=dev)
        return ((H.UPSAMPLE2X, H.MAXPOOL3S2), [H.upsample2x_args(xu, yu), H.maxpool3s2_args(xp, yp)],
                algorithmic_bytes(), {}, [(xu_h, xu), (xp_h, xp)], [yu, yp])
    if name == "hist_philox":
        xh_h = W.hist_input(1 << 28).pin_memory()
        xh = xh_h.to(dev)
        bins = torch.zeros(256, dtype=torch.int32, device=dev)
        out = torch.empty((1 << 26, 4), dtype=torch.int32, device=dev)
        nbytes = (1 << 28) + 256 * 4 + (1 << 26) * 16
        ops = {"imul": (1 << 26) * 40, "smem_atomic": 1 << 28}
        return ((H.HIST256, H.PHILOX), [H.hist256_args(xh, bins), H.philox_args(out, 0)], nbytes, ops,
                [(xh_h, xh)], [bins, out])
    if name == "bn_poly":
        xb_h = W.bn_input((8, 64, 32, 32)).pin_memory()
        xq_h = W.poly_input(1 << 20).pin_memory()
        xb, xq = xb_h.to(dev), xq_h.to(dev)
        m, v = torch.empty(64, device=dev), torch.empty(64, device=dev)
        yq = torch.empty_like(xq)
        ws = H.bn_stats_workspace(xb)
        nbytes = xb.numel() * 4 + 2 * 64 * 4 + 2 * xq.numel() * 4
        ops = {"ffma": (1 << 20) * 64 * 33 + 2 * xb.numel()}
        return ((H.BN_STATS, H.POLY), [H.bn_stats_args(xb, m, v, ws),
                                       H.poly_args(xq, yq, W.poly_coefficients().tolist())],
                nbytes, ops, [(xb_h, xb), (xq_h, xq)], [m, v, yq, ws])
    if name in PAIR_SPECS and "hashes" in PAIR_SPECS[name]:
        ids = {"sha256d": H.SHA256D, "blake256": H.BLAKE256, "blake2b": H.BLAKE2B}
        args, outs = [], []
        for k, hname in enumerate(PAIR_SPECS[name]["hashes"]):
            cnt = torch.zeros(1, dtype=torch.int32, device=dev)
            hits = torch.zeros(1 << 12, dtype=torch.int32, device=dev)
            args.append(H.hash_scan_args(W.hash_header(k), HASH_N[hname], 0,
                                         W.WORKLOADS["hash_pairs"]["target"], None, hits, cnt))
            outs += [cnt, hits]
        hs = PAIR_SPECS[name]["hashes"]
        ops = {"ialu": sum(HASH_N[h] * HASH_OPS[h] for h in hs)}
        return (tuple(ids[h] for h in hs), args, 0, ops, [], outs)
    raise SystemExit("unknown pair workload " + name)


PIPE_DESC = {"ffma": "independent FP32 FMA chains", "imul": "32-bit integer multiplies",
             "smem_atomic": "conflict-free shared-memory atomics",
             "ialu": "32-bit add/XOR/rotate mix"}


def pipe_peaks(H, stream):
    return {"ffma": H.hf_calibrate(H.CAL_FFMA, stream), "imul": H.hf_calibrate(H.CAL_IMUL, stream),
            "smem_atomic": H.hf_calibrate(H.CAL_SMEM_ATOMIC, stream),
            "ialu": H.hf_calibrate(H.CAL_IALU, stream)}


def spread(per):
    """Median and 10th / 90th percentiles of the per-step times (us)."""
    q = sorted(per)
    pick = lambda f: q[min(int(f * (len(q) - 1) + 0.5), len(q) - 1)]
    return {"median": round(pick(0.5), 3), "p10": round(pick(0.1), 3), "p90": round(pick(0.9), 3)}


def dominant_roofline(terms, nbytes, ops, peaks, t_us, hbm_gbs, peak_kind, traffic):
    """The roofline of the term that bounds the ideal: HBM bytes, or the
    operations of the busiest pipe against its calibrated rate."""
    dom = max(terms, key=terms.get)
    if dom != "hbm":
        achieved = ops[dom] / (t_us * 1e-6) / 1e12
        return {"bound": "alu", "pipe": dom, "achieved": round(achieved, 3),
                "peak": round(peaks[dom] / 1e12, 3), "unit": "Tops/s",
                "frac": round(achieved * 1e12 / peaks[dom], 4), "traffic": traffic,
                "peak_source": "measured in this run: %s (calibration kernel)" % PIPE_DESC[dom]}
    achieved = nbytes / (t_us * 1e-6) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_gbs, "unit": "GB/s",
            "frac": round(achieved / hbm_gbs, 4), "traffic": traffic, "peak_source": peak_kind}


def ideal_us(nbytes, ops, peaks, hbm_gbs):
    terms = {"hbm": nbytes / (hbm_gbs * 1e9) * 1e6}
    for k, v in ops.items():
        terms[k] = v / peaks[k] * 1e6
    return max(terms.values()), {k: round(v, 2) for k, v in terms.items()}


class Ctx:
    """Per-run state: device, streams, distributed group, timing helpers."""

    def __init__(self, args):
        import torch
        self.torch = torch
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        self.dev = torch.device("cuda", local)
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl")
            self.dist = dist
        self.stream = torch.cuda.Stream(device=self.dev)
        self.flush_buf = None
        self.args = args

    def flush(self):
        if self.flush_buf is None:
            self.flush_buf = self.torch.empty(512 << 20, dtype=self.torch.uint8, device=self.dev)
        self.flush_buf.zero_()

    def timed(self, fn, reps, warm=2, flush=False):
        torch = self.torch
        s = self.stream
        with torch.cuda.stream(s):
            for _ in range(warm):
                fn()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
            for i in range(reps):
                if flush:
                    self.flush()
                ev[2 * i].record(s)
                fn()
                ev[2 * i + 1].record(s)
            torch.cuda.synchronize()
        return [ev[2 * i].elapsed_time(ev[2 * i + 1]) * 1e3 for i in range(reps)]

    def barrier(self):
        if self.dist:
            self.dist.barrier()
        self.torch.cuda.synchronize()

    def max_over_ranks(self, v):
        return max_over_ranks(v, self.dist, self.dev)


def pipelined_e2e(cx, slots, steps, warm=2):
    """End-to-end time per step with two buffer sets.  Step i copies its
    inputs from pinned host memory into set i % 2 (one copy stream), runs
    the launch on them (the compute stream) and copies every output back to
    pinned host memory (a second copy stream); step i + 1's input copy thus
    overlaps step i's output copy, the two directions running on separate
    copy engines.  Events keep a set from being overwritten while step
    i - 2 still uses it.  slots[b] = (h2d [(host, dev)], d2h [(dev, host)],
    launch(stream))."""
    torch = cx.torch
    s_in, s_k, s_out = (torch.cuda.Stream(device=cx.dev) for _ in range(3))
    ev_in, ev_k, ev_out = ([torch.cuda.Event() for _ in range(2)] for _ in range(3))
    used = [False, False]

    def step(i):
        b = i % 2
        h2d, d2h, launch = slots[b]
        if used[b]:
            s_in.wait_event(ev_k[b])     # step i - 2's launch has read these inputs
            s_k.wait_event(ev_out[b])    # and its outputs have left
        with torch.cuda.stream(s_in):
            for h, d in h2d:
                d.copy_(h, non_blocking=True)
        ev_in[b].record(s_in)
        s_k.wait_event(ev_in[b])
        launch(s_k)
        ev_k[b].record(s_k)
        s_out.wait_event(ev_k[b])
        with torch.cuda.stream(s_out):
            for d, h in d2h:
                h.copy_(d, non_blocking=True)
        ev_out[b].record(s_out)
        used[b] = True

    for i in range(warm):
        step(i)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    for i in range(warm, warm + steps):
        step(i)
    e1.record(s_out)   # after the last output copy, which follows every other step's work
    e1.synchronize()
    return e0.elapsed_time(e1) * 1e3 / steps


def e2e_runs(cx, slots, steps, runs=3):
    """`runs` independent runs of pipelined_e2e (us per step each).  The
    host link's rate with both directions busy changes from run to run on a
    shared host (8.2 to 15 ms per step for the 8-way workload within one
    process, with or without the launch in between), so the line reports
    the median run and keeps every run."""
    return [pipelined_e2e(cx, slots, steps) for _ in range(runs)]


def link_rates(cx, h2d, d2h, reps=3):
    """Host-device link rates seen in this run: every input copied in alone
    (one stream), every output copied out alone, then both directions at
    once; best of `reps` each.  h2d = [(pinned host, device)], d2h =
    [(device, pinned host)]."""
    torch = cx.torch
    s1, s2 = torch.cuda.Stream(device=cx.dev), torch.cuda.Stream(device=cx.dev)
    nin = sum(d.numel() * d.element_size() for _, d in h2d)
    nout = sum(d.numel() * d.element_size() for d, _ in d2h)

    def once(do_in, do_out):
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(s1)
        s2.wait_event(e0)
        if do_in:
            with torch.cuda.stream(s1):
                for h, d in h2d:
                    d.copy_(h, non_blocking=True)
        if do_out:
            with torch.cuda.stream(s2):
                for d, h in d2h:
                    h.copy_(d, non_blocking=True)
        e1.record(s1)
        e2.record(s2)
        torch.cuda.synchronize()
        return max(e0.elapsed_time(e1), e0.elapsed_time(e2)) * 1e3

    t_in = min(once(True, False) for _ in range(reps))
    t_out = min(once(False, True) for _ in range(reps))
    t_both = min(once(True, True) for _ in range(reps))
    return {"h2d_gbs": round(nin / (t_in * 1e3), 1), "d2h_gbs": round(nout / (t_out * 1e3), 1),
            "h2d_alone_us": round(t_in, 1), "d2h_alone_us": round(t_out, 1),
            "both_directions_us": round(t_both, 1)}


def e2e_record(runs, h2d, d2h, steps, link):
    """The end-to-end object: per-step time with the copies inside the timed
    region (the median of `runs`, each listed), the bytes each way, the link
    rates measured in the same process and the copy-only bound they imply
    (both directions at once, per step)."""
    return {"value": round(statistics.median(runs), 2), "unit": "us", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": steps, "runs_us": [round(t, 1) for t in runs],
            "link": link, "copy_bound_us": link["both_directions_us"],
            "mode": "double-buffered: step i+1's inputs copy in while step i's outputs copy out; "
                    "median of %d runs of %d steps" % (len(runs), steps)}


def max_over_ranks(value, dist=None, device=None):
    """The slowest rank's time: every rank contributes its own and gets the
    maximum back (one all-reduce; replicas exchange nothing else)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def run_pair(cx, name, sub=False, peaks=None):
    """One fused pair: exhaustive search, Algorithm 2, naive split, VFuse,
    then the fused launch timed against serial and two-stream launches.
    With sub=True it returns the compact record embedded in the default
    line (no end-to-end leg)."""
    import torch

    from paper_2007_01277_gb300 import hfuse as H
    from paper_2007_01277_gb300 import workloads as W
    spec = PAIR_SPECS[name]
    bodies, args, nbytes, ops, host_in, outs = make_pair(name, H, W, cx.dev)
    ka, kb = H.hf_register_kernel(bodies[0]), H.hf_register_kernel(bodies[1])
    lim = H.hf_device_info()
    st, d0, fl = cx.stream, spec["d0"], spec["flush"]

    # exhaustive search over (split, regcap, blocks/SM) -- outside the timed region
    table = H.hf_profile_pair(ka, kb, args, d0, list(spec["splits"]), list(spec["caps"]),
                              list(spec["bps"]), reps=5, flush_l2=fl, stream=st)
    ok = [p for p in table if p["status"] == 0]
    best = min(ok, key=lambda p: p["time_us"])
    alg2, a2_trace = H.hf_search_alg2(ka, kb, args, d0, step=128 if d0 >= 512 else 64, reps=5,
                                      flush_l2=fl, stream=st)
    naive = [p for p in ok if p["split"] == d0 // 2 and p["regcap"] == 0]
    naive = min(naive, key=lambda p: -p["blocks_per_sm"]) if naive else None
    # vertical fusion (Sec. 2.2): every thread runs one kernel, then the other
    vfuse = None
    for dv in (256, 512):
        try:
            fv = H.hf_fuse_n([ka, kb], [0, 0], [dv], 0)
        except H.HFError:
            continue
        iv = H.hf_query(fv, args)
        tv = H.hf_time_fused(fv, args, iv["blocks_per_sm"] * lim.sm_count, reps=5, flush_l2=fl,
                             stream=st)[0]
        H.hf_destroy_fused(fv)
        if vfuse is None or tv < vfuse[0]:
            vfuse = (tv, dv)
    fused = H.hf_fuse(ka, kb, best["split"], d0, best["regcap"])
    grid = best["grid"]

    def best_single(k, a):
        res = []
        for thr in (128, 256, 512):
            info = H.hf_query_single(k, a, thr)
            g = info["blocks_per_sm"] * lim.sm_count
            t = statistics.median(cx.timed(lambda: H.hf_launch_single(k, a, thr, g, st), 5, flush=fl))
            res.append((t, thr, g))
        return min(res)

    ta, thr_a, g_a = best_single(ka, args[0])
    tb, thr_b, g_b = best_single(kb, args[1])
    s2 = torch.cuda.Stream(device=cx.dev)
    ev_f, ev_j = torch.cuda.Event(), torch.cuda.Event()

    def step_fused():
        H.hf_launch(fused, args, grid, st)

    def step_serial():
        H.hf_launch_single(ka, args[0], thr_a, g_a, st)
        H.hf_launch_single(kb, args[1], thr_b, g_b, st)

    def step_two():
        ev_f.record(st)
        s2.wait_event(ev_f)
        H.hf_launch_single(ka, args[0], thr_a, g_a, st)
        H.hf_launch_single(kb, args[1], thr_b, g_b, s2)
        ev_j.record(s2)
        st.wait_event(ev_j)

    K, Wm = cx.args.steps, cx.args.warmup
    cx.barrier()
    with ClockSampler(cx.dev) as clk:
        per = cx.timed(step_fused, K, warm=Wm, flush=fl)
    cx.barrier()
    t_fused = cx.max_over_ranks(statistics.mean(per))
    t_serial = statistics.median(cx.timed(step_serial, max(5, K // 4), warm=Wm, flush=fl))
    t_two = statistics.median(cx.timed(step_two, max(5, K // 4), warm=Wm, flush=fl))
    # the fused launch captured in a CUDA graph (one graph launch per step)
    H.hf_graph_begin(st)
    step_fused()
    g_fused = H.hf_graph_end(st)
    t_graph = statistics.median(cx.timed(lambda: H.hf_graph_launch(g_fused, st), max(5, K // 4),
                                         warm=Wm, flush=fl))
    H.hf_graph_destroy(g_fused)

    hbm, peak_kind = measured_peaks()
    peaks = peaks or pipe_peaks(H, st)
    t_ideal, terms = ideal_us(nbytes, ops, peaks, hbm)
    roofline = dominant_roofline(terms, nbytes, ops, peaks, t_fused, hbm, peak_kind,
                                 load_traffic(spec["name"]))
    info = H.hf_query(fused, args)
    search = {"exhaustive_best_us": round(best["time_us"], 3), "points": len(ok),
              "alg2": {k: alg2[k] for k in ("split", "regcap", "blocks_per_sm", "time_us")},
              "alg2_trace": [[p[k] for k in ("split", "regcap", "blocks_per_sm", "regs", "spill_bytes")]
                             + [round(p["time_us"], 2)] for p in a2_trace],
              "exhaustive_best": {k: best[k] for k in ("split", "regcap", "blocks_per_sm", "regs",
                                                       "spill_bytes")},
              "naive_even_split_us": round(naive["time_us"], 3) if naive else None,
              "vfuse_us": round(vfuse[0], 3) if vfuse else None,
              "vfuse_block": vfuse[1] if vfuse else None}
    cfg = {"split": best["split"], "d0": d0, "regcap": best["regcap"], "grid": grid,
           "regs": info["regs"], "spill_bytes": info["spill_bytes"],
           "l2": "L2 flushed (512 MB write) before every timed launch" if fl else
                 "inputs larger than L2 (%.0f MB touched per step)" % _mb(nbytes)}
    standalone = {H.BODY_NAMES[bodies[0]]: round(ta, 3), H.BODY_NAMES[bodies[1]]: round(tb, 3),
                  "threads": [thr_a, thr_b]}
    if sub:
        rec = {"workload": spec["desc"], "fused_us": round(t_fused, 3), "serial_us": round(t_serial, 3),
               "two_stream_us": round(t_two, 3), "fused_graph_us": round(t_graph, 3),
               "fused_spread_us": spread(per), "standalone_us": standalone,
               "speedup_vs_best_native": round(min(t_serial, t_two) / t_fused, 4),
               "ideal_us": round(t_ideal, 3), "ideal_terms_us": terms,
               "frac_of_ideal": round(t_ideal / t_fused, 4), "roofline": roofline,
               "config": cfg, "search": search, "steps": K, "clocks": clk.summary()}
        H.hf_destroy_fused(fused)
        return rec
    # end to end: a second buffer set, inputs in and every output out per step
    _b2, args2, _n2, _o2, host_in2, outs2 = make_pair(name, H, W, cx.dev)
    slots = []
    for a_, hin, outs_ in ((args, host_in, outs), (args2, host_in2, outs2)):
        hout = [torch.empty(o.shape, dtype=o.dtype, pin_memory=True) for o in outs_]
        slots.append((hin, list(zip(outs_, hout)),
                      lambda s_, a_=a_: H.hf_launch(fused, a_, grid, s_)))
    t_e2e = e2e_runs(cx, slots, max(20, K))
    h2d = sum(d.numel() * d.element_size() for _, d in host_in)
    if "hashes" in spec:
        h2d += 80 * len(args)   # the headers travel in the launch's parameter block
    d2h = sum(o.numel() * o.element_size() for o in outs)
    link = link_rates(cx, slots[0][0], slots[0][1])
    cfg["parallelism"] = "replicas" if cx.world > 1 else "single"
    cfg["workload"] = spec["desc"]
    return {
        "metric": METRIC, "value": round(t_fused, 3), "unit": "us",
        "n_gpus": cx.world, "steps": K, "warmup": Wm, "ms_per_step": round(t_fused / 1e3, 6),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": {"hist_philox": "u8/u32"}.get(name, "u32/u64" if "hashes" in spec else "f32"),
        "data": "synthetic (seeded torch.Generator, CPU-drawn)",
        "config": cfg,
        "serial_us": round(t_serial, 3), "two_stream_us": round(t_two, 3),
        "fused_graph_us": round(t_graph, 3), "fused_spread_us": spread(per),
        "standalone_us": standalone,
        "speedup_vs_best_native": round(min(t_serial, t_two) / t_fused, 4),
        "ideal_us": round(t_ideal, 3), "ideal_terms_us": terms, "frac_of_ideal": round(t_ideal / t_fused, 4),
        "pipe_peaks_per_s": {k: float("%.4g" % v) for k, v in peaks.items()},
        "search": search,
        "roofline": roofline,
        "e2e": e2e_record(t_e2e, h2d, d2h, max(20, K), link),
        "gpu_launches": K,
        "clocks": clk.summary(),
    }


# the fused pairs reported inside the default (8-way) line
SUB_PAIRS = ("bn_poly", "hist_philox", "upsample_maxpool")

NWAY_DESC = ("8 kernels in one persistent CUDA-graph launch: bn stats 64x256x56x56, im2col 3x3 "
             "32x64x56x56, maxpool 32x128x112x112, upsample 32x64x128x128, hist 2^26 u8, "
             "Philox 2^24 blocks, 64x degree-32 Horner on 2^22, bf16 axpy on 2^27")


def run_nway(cx):
    import torch

    from paper_2007_01277_gb300 import hfuse as H
    from paper_2007_01277_gb300 import workloads as W
    dev, st = cx.dev, cx.stream
    sp = W.WORKLOADS["nway8"]

    def make_set():
        """Device tensors and argument blocks of the eight kernels (inputs,
        outputs and the argument list)."""
        xb = W.bn_input(sp["bn"]).to(dev)
        mb, vb = torch.empty(sp["bn"][1], device=dev), torch.empty(sp["bn"][1], device=dev)
        ws = H.bn_stats_workspace(xb)
        xi = W.im2col_input(sp["im2col"]).to(dev)
        ci = torch.empty(sp["im2col"][0], sp["im2col"][1] * 9, sp["im2col"][2] * sp["im2col"][3], device=dev)
        xp = W.maxpool_input(sp["pool"]).to(dev)
        yp = torch.empty(sp["pool"][:2] + (56, 56), device=dev)
        xu = W.upsample_input(sp["up"]).to(dev)
        yu = torch.empty(sp["up"][:2] + (256, 256), device=dev)
        xh = W.hist_input(sp["hist_n"]).to(dev)
        bins = torch.zeros(256, dtype=torch.int32, device=dev)
        po = torch.empty((sp["philox_n"], 4), dtype=torch.int32, device=dev)
        xq = W.poly_input(sp["poly_n"]).to(dev)
        yq = torch.empty_like(xq)
        x16, y16 = (t.to(dev) for t in W.bf16_inputs(sp["bf16_n"]))
        o16 = torch.empty_like(x16)
        a_ = [H.bn_stats_args(xb, mb, vb, ws), H.im2col3_args(xi, ci), H.maxpool3s2_args(xp, yp),
              H.upsample2x_args(xu, yu), H.hist256_args(xh, bins), H.philox_args(po, 0),
              H.poly_args(xq, yq, W.poly_coefficients().tolist()), H.bf16_axpy_args(x16, y16, o16)]
        return [xb, xi, xp, xu, xh, xq, x16, y16], [mb, vb, ci, yp, yu, bins, po, yq, o16], a_

    ins, outs, args = make_set()
    xb, xi, xp, xu, xh, xq, x16, y16 = ins
    mb, vb, ci, yp, yu, bins, po, yq, o16 = outs
    bodies = [H.BN_STATS, H.IM2COL3, H.MAXPOOL3S2, H.UPSAMPLE2X, H.HIST256, H.PHILOX, H.POLY, H.BF16_AXPY]
    ks = [H.hf_register_kernel(b) for b in bodies]
    nbytes = sum(t.numel() * t.element_size() for t in (xb, xi, ci, xp, yp, xu, yu, xh, po, xq, yq, x16, y16, o16))
    ops = {"ffma": sp["poly_n"] * 64 * 33, "imul": sp["philox_n"] * 40, "smem_atomic": sp["hist_n"]}

    plan, single = H.hf_autotune_nway(ks, args, max_evals=cx.args.nway_evals, reps=5, stream=st)
    fused = H.hf_fuse_n(ks, plan["interval_of"], plan["interval_threads"], plan["regcap"])
    lim = H.hf_device_info()
    grid = plan["grid"]
    # standalone configurations for the baselines: 256 threads, resident grid
    cfg = []
    for k, a in zip(ks, args):
        info = H.hf_query_single(k, a, 256)
        cfg.append((k, a, 256, info["blocks_per_sm"] * lim.sm_count))
    streams = [torch.cuda.Stream(device=dev) for _ in range(len(ks))]
    ev_f = torch.cuda.Event()
    ev_j = [torch.cuda.Event() for _ in ks]

    def issue_fused():
        H.hf_launch(fused, args, grid, st)

    def issue_serial():
        for k, a, t, g in cfg:
            H.hf_launch_single(k, a, t, g, st)

    def issue_nstream():
        ev_f.record(st)
        for s_, (k, a, t, g), e in zip(streams, cfg, ev_j):
            s_.wait_event(ev_f)
            H.hf_launch_single(k, a, t, g, s_)
            e.record(s_)
        for e in ev_j:
            st.wait_event(e)

    graphs = {}
    with torch.cuda.stream(st):
        for nm, fn in (("fused", issue_fused), ("serial", issue_serial), ("nstream", issue_nstream)):
            fn()
            torch.cuda.synchronize()
            H.hf_graph_begin(st)
            fn()
            graphs[nm] = H.hf_graph_end(st)
    K, Wm = cx.args.steps, cx.args.warmup
    cx.barrier()
    with ClockSampler(dev) as clk:
        per = cx.timed(lambda: H.hf_graph_launch(graphs["fused"], st), K, warm=Wm)
    cx.barrier()
    t_fused = cx.max_over_ranks(statistics.mean(per))
    t_serial = statistics.median(cx.timed(lambda: H.hf_graph_launch(graphs["serial"], st), max(5, K // 4), warm=Wm))
    t_nstream = statistics.median(cx.timed(lambda: H.hf_graph_launch(graphs["nstream"], st), max(5, K // 4), warm=Wm))
    t_fused_nograph = statistics.median(cx.timed(issue_fused, max(5, K // 4), warm=Wm))
    # end to end: every input from pinned host memory, the graph, every output
    # back, with a second buffer set (and its own graph) so that consecutive
    # steps' copies overlap
    ins2, outs2, args2 = make_set()
    with torch.cuda.stream(st):
        H.hf_launch(fused, args2, grid, st)
        torch.cuda.synchronize()
        H.hf_graph_begin(st)
        H.hf_launch(fused, args2, grid, st)
        graph2 = H.hf_graph_end(st)
    slots = []
    for ins_, outs_, g_ in ((ins, outs, graphs["fused"]), (ins2, outs2, graph2)):
        hin = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in ins_]
        for h, d in zip(hin, ins_):
            h.copy_(d)
        hout = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in outs_]
        slots.append((list(zip(hin, ins_)), list(zip(outs_, hout)),
                      lambda s_, g_=g_: H.hf_graph_launch(g_, s_)))
    t_e2e = e2e_runs(cx, slots, max(20, K))
    e2e = e2e_record(t_e2e, sum(t.numel() * t.element_size() for t in ins),
                     sum(t.numel() * t.element_size() for t in outs), max(20, K),
                     link_rates(cx, slots[0][0], slots[0][1]))
    hbm, peak_kind = measured_peaks()
    peaks = pipe_peaks(H, st)
    t_ideal, terms = ideal_us(nbytes, ops, peaks, hbm)
    for g in graphs.values():
        H.hf_graph_destroy(g)
    H.hf_graph_destroy(graph2)
    H.hf_destroy_fused(fused)
    # the fused pairs, each measured the same way (fused vs serial vs two
    # streams, exhaustive search, Algorithm 2, naive split, VFuse)
    pairs = {}
    if not cx.args.no_pairs:
        for nm in SUB_PAIRS:
            pairs[nm] = run_pair(cx, nm, sub=True, peaks=peaks)
            torch.cuda.empty_cache()
    # the learned cost model on the same three pairs (trained on the
    # built-in pairs at other sizes; regret read from the exhaustive table
    # of the workload size), beside Algorithm 2 and the naive even split
    cost = None
    if not cx.args.no_pairs and not cx.args.no_cost_model:
        from paper_2007_01277_gb300 import costmodel as CM
        cost = CM.run_builtin(dev, hbm_gbs=hbm,
                              log=lambda m: print(m, file=sys.stderr, flush=True))
    return {
        "metric": METRIC, "value": round(t_fused, 3), "unit": "us",
        "n_gpus": cx.world, "steps": K, "warmup": Wm, "ms_per_step": round(t_fused / 1e3, 6),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32/bf16/u8/u32",
        "data": "synthetic (seeded torch.Generator, CPU-drawn)",
        "config": {"workload": NWAY_DESC, "plan": plan, "l2": "inputs larger than L2 (%.0f MB per step)" % _mb(nbytes),
                   "parallelism": "replicas" if cx.world > 1 else "single"},
        "serial_us": round(t_serial, 3), "n_stream_us": round(t_nstream, 3),
        "fused_no_graph_us": round(t_fused_nograph, 3), "fused_spread_us": spread(per),
        "standalone_us": {H.BODY_NAMES[b]: round(t, 2) for b, t in zip(bodies, single)},
        "speedup_vs_best_native": round(min(t_serial, t_nstream) / t_fused, 4),
        "ideal_us": round(t_ideal, 3), "ideal_terms_us": terms, "frac_of_ideal": round(t_ideal / t_fused, 4),
        "pipe_peaks_per_s": {k: float("%.4g" % v) for k, v in peaks.items()},
        "roofline": dominant_roofline(terms, nbytes, ops, peaks, t_fused, hbm, peak_kind,
                                      load_traffic("nway8")),
        "e2e": e2e, "gpu_launches": K, "clocks": clk.summary(),
        "pairs": pairs,
        "cost_model": cost,
    }


def run_cost_model(cx):
    import tempfile

    from paper_2007_01277_gb300 import costmodel as CM
    hbm, peak_kind = measured_peaks()
    db = cx.args.cost_db or os.path.join(tempfile.gettempdir(), "hfuse_cost_profile.jsonl")
    res, _P, _norm = CM.run(cx.dev, db, n_pairs=600, n_train=500, steps=cx.args.cost_steps,
                            reps=3, hbm_gbs=hbm, log=lambda m: print(m, file=sys.stderr, flush=True))
    r = res["regret"]
    return {
        "metric": METRIC, "value": round(100 * r["mean"], 3), "unit": "% regret (mean, 100 held-out pairs)",
        "n_gpus": cx.world, "steps": cx.args.cost_steps, "warmup": 0, "ms_per_step": None,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (600 generated stream-template pairs, seed 0)",
        "config": {"workload": "learned cost model: 600 parametric stream-kernel pairs, exhaustive "
                               "profile of 168 configs each, MLP 24-64-64-1 trained on 500, "
                               "regret on 100 held out", "profile_db": os.path.basename(db)},
        "cost_model": res,
    }


def run_experiment(cx, which):
    import math

    from paper_2007_01277_gb300 import experiments as E
    if which == "table2":
        rows = E.table2(cx.dev)
        sp = [r["hfuse_alg2"]["ratio"] for r in rows.values()]
        desc = ("the ten pairs of the five deep-learning kernels at execution-time ratio ~1 "
                "(Table 2's setting): native two-stream vs HFuse (Algorithm 2, no-cap best, "
                "RegCap), naive even split, VFuse")
        extra = {"pairs": rows}
    else:
        series = E.ratio_sweep(cx.dev)
        sp = [r["hfuse_alg2"]["ratio"] for s in series.values() for r in s]
        desc = ("execution-time-ratio sweep (Fig. 3's protocol): hist+maxpool with maxpool "
                "scaled, bn+hist with bn scaled, 1/8x..4x")
        extra = {"series": series}
    geo = math.exp(sum(math.log(v) for v in sp) / len(sp))
    line = {"metric": METRIC, "value": round(geo, 4),
            "unit": "geomean T_native/T_hfuse (Algorithm 2 pick, native = two streams)",
            "n_gpus": cx.world, "steps": None, "warmup": None, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/u8",
            "data": "synthetic (seeded torch.Generator, CPU-drawn)",
            "config": {"workload": desc}}
    line.update(extra)
    return line


def run_ours(args):
    cx = Ctx(args)
    if args.workload in ("table2", "ratio_sweep"):
        line = run_experiment(cx, args.workload)
    elif args.workload == "cost_model":
        line = run_cost_model(cx)
    elif args.workload == "nway8":
        line = run_nway(cx)
    else:
        line = run_pair(cx, args.workload)
    if cx.rank == 0 and not args.no_cpu_baseline:
        cb = cpu_baseline_for(args.workload)
        if cb is not None:
            line["cpu_baseline"] = cb
    if cx.rank == 0:
        print(json.dumps(line), flush=True)
    if cx.dist:
        cx.dist.barrier()
        cx.dist.destroy_process_group()


def load_traffic(name):
    """DRAM bytes per launch of the fused kernel from the committed ncu
    summary (dram__bytes_read.sum + dram__bytes_write.sum), if any."""
    p = os.path.join(ROOT, "profiles", name + "_traffic.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        parts = line.split()
        if len(parts) == 2 and parts[0] == "traffic_bytes_per_launch":
            return int(parts[1])
    return None


# ------------------------------------------------------------------ CPU oracle
def _ranges(n, parts):
    """`parts` contiguous [lo, hi) ranges that cover 0 .. n-1 (empty ones dropped)."""
    step = max(1, -(-n // max(1, parts)))
    return [(lo, min(n, lo + step)) for lo in range(0, n, step)]


_CPU_JOBS = {}


def cpu_jobs(workload, cores):
    """The oracle over the workload as independent jobs for `cores` host
    threads: (jobs, scale, description).  Every kernel's input is cut into
    about `cores` contiguous slices (images, channels, element or counter
    ranges); the oracle's C routines release the interpreter lock, so the
    slices run in parallel.  The deep-learning, histogram, Philox,
    polynomial and bf16 workloads are computed whole (scale 1); the hash
    scans on a fixed slice of their nonces, scaled.  Inputs are drawn once
    and cached, outside any timing."""
    key = (workload, cores)
    if key in _CPU_JOBS:
        return _CPU_JOBS[key]
    import numpy as np

    import oracle
    from paper_2007_01277_gb300 import workloads as W
    jobs = []

    def images(fn, x):
        for lo, hi in _ranges(x.shape[0], cores):
            jobs.append(lambda a=x[lo:hi]: fn(a))

    def channels(x):
        for lo, hi in _ranges(x.shape[1], cores):
            jobs.append(lambda a=np.ascontiguousarray(x[:, lo:hi]): oracle.bn_stats(a))

    def flat(fn, x):
        for lo, hi in _ranges(x.shape[0], cores):
            jobs.append(lambda a=x[lo:hi]: fn(a))

    def philox(n):
        for lo, hi in _ranges(n, cores):
            jobs.append(lambda lo=lo, hi=hi: oracle.philox4x32_10(0, hi - lo, first=lo))

    coef = W.poly_coefficients().numpy()
    poly = lambda a: oracle.poly(a, coef)
    scale, desc = 1.0, "the whole workload"
    if workload == "nway8":
        sp = W.WORKLOADS["nway8"]
        channels(W.bn_input(sp["bn"]).numpy())
        images(oracle.im2col3, W.im2col_input(sp["im2col"]).numpy())
        images(oracle.maxpool3s2p1, W.maxpool_input(sp["pool"]).numpy())
        images(oracle.upsample2x, W.upsample_input(sp["up"]).numpy())
        flat(oracle.hist256, W.hist_input(sp["hist_n"]).numpy())
        philox(sp["philox_n"])
        flat(poly, W.poly_input(sp["poly_n"]).numpy())
        x16, y16 = (t.view(torch_int16()).numpy().view(np.uint16) for t in W.bf16_inputs(sp["bf16_n"]))
        for lo, hi in _ranges(x16.shape[0], cores):
            jobs.append(lambda a=x16[lo:hi], b=y16[lo:hi]: oracle.bf16_axpy(a, b, W.BF16_ALPHA))
        desc = "the whole workload (all 8 kernels), each input cut into %d slices" % cores
    elif workload == "upsample_maxpool":
        images(oracle.upsample2x, W.upsample_input(UP_SHAPE).numpy())
        images(oracle.maxpool3s2p1, W.maxpool_input(POOL_SHAPE).numpy())
        desc = "the whole workload (both kernels), cut into image slices"
    elif workload == "hist_philox":
        flat(oracle.hist256, W.hist_input(1 << 28).numpy())
        philox(1 << 26)
        desc = "the whole workload (both kernels), cut into byte and counter ranges"
    elif workload == "bn_poly":
        channels(W.bn_input((8, 64, 32, 32)).numpy())
        flat(poly, W.poly_input(1 << 20).numpy())
        desc = "the whole workload (both kernels), cut into channel and element ranges"
    elif workload in PAIR_SPECS and "hashes" in PAIR_SPECS[workload]:
        scans = {"sha256d": oracle.sha256d_scan, "blake256": oracle.blake256_scan,
                 "blake2b": oracle.blake2b_scan}
        hs = PAIR_SPECS[workload]["hashes"]
        per = 1 << 16
        # the same fraction of each scan, so that one scale factor applies
        frac = per / max(HASH_N[h] for h in hs)
        for k, h in enumerate(hs):
            n = max(cores, int(HASH_N[h] * frac))
            hdr = W.hash_header(k)
            for lo, hi in _ranges(n, cores):
                jobs.append(lambda lo=lo, hi=hi, h=h, hdr=hdr: scans[h](hdr, lo, hi - lo))
        scale = 1.0 / frac
        desc = "%.4f of each scan's nonces, scaled x%.0f" % (frac, scale)
    else:
        return None
    _CPU_JOBS[key] = (jobs, scale, desc)
    return _CPU_JOBS[key]


def _pool_time(jobs, cores):
    from concurrent.futures import ThreadPoolExecutor
    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        list(ex.map(lambda f: f(), jobs))
    return time.perf_counter() - t0


def cpu_sample_us(workload, cores):
    """One timed run of the oracle on the workload's sample (us, scaled)."""
    jobs, scale, _desc = cpu_jobs(workload, cores)
    return _pool_time(jobs, cores) * scale * 1e6


def cpu_baseline_for(workload: str, reps: int = 3):
    """The cpu_baseline object: the median of `reps` runs of the oracle on
    the workload's sample, spread over every host core, and one run of the
    same jobs on a single thread.  The reference arm times the same sample
    per step."""
    cores = os.cpu_count() or 1
    if cpu_jobs(workload, cores) is None:
        return None
    jobs, scale, desc = cpu_jobs(workload, cores)
    v = statistics.median(cpu_sample_us(workload, cores) for _ in range(reps))
    one = _pool_time(jobs, 1) * scale * 1e6
    return {"value": round(v, 1), "unit": "us", "cores": cores, "kind": "oracle",
            "sample": "%s; median of %d runs" % (desc, reps),
            "single_thread_us": round(one, 1)}


def torch_int16():
    import torch
    return torch.int16


def run_reference(args):
    """The reference arm: the oracle (the paper has no code) timed on the
    host cores, one run of the same sample as cpu_baseline per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    got = cpu_jobs(args.workload, cores)
    if got is None:
        print(json.dumps({"impl": "reference", "unavailable": "no CPU oracle sample for workload "
                          + args.workload}), flush=True)
        return
    desc = got[2]
    for _ in range(args.warmup):
        cpu_sample_us(args.workload, cores)
    per = [cpu_sample_us(args.workload, cores) for _ in range(args.steps)]
    v = round(statistics.median(per), 1)
    wl = NWAY_DESC if args.workload == "nway8" else PAIR_SPECS.get(args.workload, {}).get("desc", args.workload)
    line = {"metric": METRIC, "value": v, "unit": "us", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v / 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded torch.Generator, CPU-drawn)", "impl": "reference",
            "config": {"workload": wl, "sample": desc},
            "cpu_baseline": {"value": v, "unit": "us", "cores": cores, "kind": "oracle",
                             "sample": "%s; median of %d steps" % (desc, args.steps)},
            "step_spread_us": spread(per),
            "e2e": {"value": v, "unit": "us", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", default="nway8",
                    choices=sorted(PAIR_SPECS) + ["nway8", "cost_model", "table2", "ratio_sweep"])
    ap.add_argument("--cost-db", default=None)
    ap.add_argument("--cost-steps", type=int, default=20000)
    ap.add_argument("--nway-evals", type=int, default=10000)
    ap.add_argument("--no-pairs", action="store_true",
                    help="8-way workload only: skip the fused-pair records")
    ap.add_argument("--no-cost-model", action="store_true",
                    help="8-way workload only: skip the learned-model record")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
