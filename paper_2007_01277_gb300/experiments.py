"""The paper's comparison experiments on GB300 (Sec. 4.1-4.3).

table2()       Table 2's setting: the ten pairs of the five deep-learning
               kernels (batch-norm statistics, histogram, max pool, upsample,
               im2col) at sizes where each kernel alone takes about the same
               time (execution-time ratio ~1, Sec. 4.3).  Per pair: the native
               execution (two concurrent streams, Sec. 4.1) and serial
               launches, HFuse without a register bound (best split, "N-RegCap")
               and with Algorithm 2's bound r0 ("RegCap"), the naive even split
               without profiling, and vertical fusion (VFuse: every thread runs
               one kernel then the other, Sec. 2.2), which is the one-interval
               schedule of the N-way kernel.
ratio_sweep()  Fig. 3's protocol: one kernel's input size is scaled to sweep
               the ratio of the two kernels' times; HFuse (Algorithm 2),
               naive and VFuse against the native execution at each ratio.

Speedup is reported both ways the paper's "X% faster" can be read:
T_native / T and (T_native - T) / T_native.
"""
from __future__ import annotations

import statistics

import torch

from . import hfuse as H
from . import workloads as W

DL_BODIES = ("bn", "hist", "maxpool", "upsample", "im2col")
D0 = 512
SPLITS = tuple(range(64, D0, 64))


def _make(kind, scale, dev):
    """(body id, argument block, tensors) of one deep-learning kernel at the
    ratio-1 size times `scale` (batch dimension or byte count)."""
    def nb(n):
        return max(1, int(round(n * scale)))
    if kind == "bn":
        x = W.bn_input((nb(64), 256, 56, 56)).to(dev)
        m, v = torch.empty(256, device=dev), torch.empty(256, device=dev)
        ws = H.bn_stats_workspace(x)
        return H.BN_STATS, H.bn_stats_args(x, m, v, ws)
    if kind == "hist":
        x = W.hist_input(max(1 << 16, int((1 << 27) * scale)) // 16 * 16).to(dev)
        b = torch.zeros(256, dtype=torch.int32, device=dev)
        return H.HIST256, H.hist256_args(x, b)
    if kind == "maxpool":
        x = W.maxpool_input((nb(32), 128, 112, 112)).to(dev)
        y = torch.empty(x.shape[:2] + (56, 56), device=dev)
        return H.MAXPOOL3S2, H.maxpool3s2_args(x, y)
    if kind == "upsample":
        x = W.upsample_input((nb(16), 64, 128, 128)).to(dev)
        y = torch.empty(x.shape[:2] + (256, 256), device=dev)
        return H.UPSAMPLE2X, H.upsample2x_args(x, y)
    if kind == "im2col":
        x = W.im2col_input((nb(32), 64, 56, 56)).to(dev)
        c = torch.empty(x.shape[0], 576, 3136, device=dev)
        return H.IM2COL3, H.im2col3_args(x, c)
    raise ValueError(kind)


class _Timer:
    def __init__(self, dev):
        self.stream = torch.cuda.Stream(device=dev)
        self.s2 = torch.cuda.Stream(device=dev)
        self.lim = H.hf_device_info()
        self.ev = (torch.cuda.Event(), torch.cuda.Event())

    def single(self, k, a):
        best = None
        for thr in (128, 256, 512):
            try:
                info = H.hf_query_single(k, a, thr)
            except H.HFError:
                continue
            g = info["blocks_per_sm"] * self.lim.sm_count
            t = H.hf_time_single(k, a, thr, g, reps=7, flush_l2=False, stream=self.stream)[0]
            if best is None or t < best[0]:
                best = (t, thr, g)
        return best

    def native(self, ka, a, cfg_a, kb, b, cfg_b, reps=15):
        """Two concurrent streams (the paper's native execution) and serial."""
        st, s2 = self.stream, self.s2
        f, j = self.ev

        def two():
            f.record(st)
            s2.wait_event(f)
            H.hf_launch_single(ka, a, cfg_a[1], cfg_a[2], st)
            H.hf_launch_single(kb, b, cfg_b[1], cfg_b[2], s2)
            j.record(s2)
            st.wait_event(j)

        def serial():
            H.hf_launch_single(ka, a, cfg_a[1], cfg_a[2], st)
            H.hf_launch_single(kb, b, cfg_b[1], cfg_b[2], st)

        out = []
        for fn in (two, serial):
            with torch.cuda.stream(st):
                fn()
                fn()
                ts = []
                for _ in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(st)
                    fn()
                    e1.record(st)
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1) * 1e3)
            out.append(statistics.median(ts))
        return out

    def fused(self, f, args):
        info = H.hf_query(f, args)
        g = info["blocks_per_sm"] * self.lim.sm_count
        return H.hf_time_fused(f, args, g, reps=7, flush_l2=False, stream=self.stream)[0], info

    def vfuse(self, ka, kb, args):
        best = None
        for d0 in (256, 512):
            try:
                f = H.hf_fuse_n([ka, kb], [0, 0], [d0], 0)
            except H.HFError:
                continue
            t, info = self.fused(f, args)
            H.hf_destroy_fused(f)
            if best is None or t < best[0]:
                best = (t, d0)
        return best


def _speed(t_native, t):
    return {"ratio": round(t_native / t, 4), "saving": round((t_native - t) / t_native, 4)}


def pair_row(tm, ka, a, kb, b):
    ca, cb = tm.single(ka, a), tm.single(kb, b)
    t_two, t_serial = tm.native(ka, a, ca, kb, b, cb)
    t_native = t_two
    args = [a, b]
    table = H.hf_profile_pair(ka, kb, args, D0, list(SPLITS), [0], [1, 2, 3, 4], reps=5,
                              flush_l2=False, stream=tm.stream)
    ok = [p for p in table if p["status"] == 0]
    nreg = min(ok, key=lambda p: p["time_us"])
    alg2, trace = H.hf_search_alg2(ka, kb, args, D0, step=64, reps=5, flush_l2=False, stream=tm.stream)
    capped = [p for p in trace if p["status"] == 0 and p["regcap"] > 0]
    regcap = min(capped, key=lambda p: p["time_us"]) if capped else None
    naive_pts = [p for p in ok if p["split"] == D0 // 2]
    naive = max(naive_pts, key=lambda p: p["blocks_per_sm"]) if naive_pts else None
    vf = tm.vfuse(ka, kb, args)
    row = {
        "t_alone_us": [round(ca[0], 2), round(cb[0], 2)], "time_ratio": round(ca[0] / cb[0], 3),
        "native_two_stream_us": round(t_two, 2), "serial_us": round(t_serial, 2),
        "hfuse_nregcap": {"us": round(nreg["time_us"], 2), "split": nreg["split"],
                          "blocks_per_sm": nreg["blocks_per_sm"], "regs": nreg["regs"],
                          **_speed(t_native, nreg["time_us"])},
        "hfuse_alg2": {"us": round(alg2["time_us"], 2), "split": alg2["split"], "regcap": alg2["regcap"],
                       **_speed(t_native, alg2["time_us"])},
        "hfuse_regcap": None if regcap is None else {
            "us": round(regcap["time_us"], 2), "split": regcap["split"], "regcap": regcap["regcap"],
            "regs": regcap["regs"], "spill": regcap["spill_bytes"], **_speed(t_native, regcap["time_us"])},
        "naive_even": None if naive is None else {"us": round(naive["time_us"], 2),
                                                  **_speed(t_native, naive["time_us"])},
        "vfuse": None if vf is None else {"us": round(vf[0], 2), "d0": vf[1], **_speed(t_native, vf[0])},
    }
    return row


def table2(dev):
    tm = _Timer(dev)
    rows = {}
    for i, ka_name in enumerate(DL_BODIES):
        for kb_name in DL_BODIES[i + 1:]:
            ida, a = _make(ka_name, 1.0, dev)
            idb, b = _make(kb_name, 1.0, dev)
            ka, kb = H.hf_register_kernel(ida), H.hf_register_kernel(idb)
            rows[ka_name + "+" + kb_name] = pair_row(tm, ka, a, kb, b)
            del a, b
            torch.cuda.empty_cache()
    return rows


def ratio_sweep(dev, pairs=(("hist", "maxpool", "maxpool"), ("bn", "hist", "bn")),
                scales=(0.125, 0.25, 0.5, 1.0, 2.0, 4.0)):
    """For each (A, B, scaled kernel): rows at each scale of the marked kernel."""
    tm = _Timer(dev)
    out = {}
    for an, bn, which in pairs:
        series = []
        for s in scales:
            ida, a = _make(an, s if which == an else 1.0, dev)
            idb, b = _make(bn, s if which == bn else 1.0, dev)
            ka, kb = H.hf_register_kernel(ida), H.hf_register_kernel(idb)
            r = pair_row(tm, ka, a, kb, b)
            r["scale"] = s
            series.append(r)
            del a, b
            torch.cuda.empty_cache()
        out["%s+%s (scaled: %s)" % (an, bn, which)] = series
    return out
