"""Named launch cases for profiling (ncu) and quick timing.

    python -m paper_2007_01277_gb300.profile_cases CASE [--launches N]
           [--split S] [--regcap R] [--bps B] [--threads T] [--scale F]

Allocates only what CASE needs, launches its kernel(s) N times on one stream
and prints the median CUDA-event time per launch.  Cases:
  fused_up_pool   upsample x2 32x64x128x128 + maxpool 32x128x112x112 fused
  up, pool        the same kernels alone
  fused_hist_philox  2^28-byte histogram + 2^26 Philox blocks fused
  hist, philox    alone
  fused_bn_poly   bn stats 8x64x32x32 + polynomial chain on 2^20 fused
  bn, poly        alone
  bn_large        bn stats 64x256x56x56
  im2col          im2col 32x64x56x56
  bf16            bf16 scale+add on 2^27
  fused_sha256d_blake2b  SHA-256d scan of 2^24 nonces + BLAKE2b scan of
                  21*2^20 nonces fused (hits only, target 2^16)
  sha256d, blake256, blake2b  the hash scans alone (2^24, 2^25, 21*2^20)
  nway8           the eight kernels of the N-way workload in one launch with a
                  fixed plan (--plan "io;threads;cap", default an autotuned
                  4-interval plan of one 512-thread block, no register cap)
--scale shrinks the batch dimension (and 1-D sizes) by F for small captures.
"""
from __future__ import annotations

import argparse
import statistics

import torch

from . import hfuse as H
from . import workloads as W


def build(case, scale, dev):
    s = max(scale, 1e-6)

    def nb(n):
        return max(1, int(round(n * s)))

    def n1(n):
        return max(1024, int(n * s) // 1024 * 1024)

    out = {}
    if case in ("fused_up_pool", "up"):
        x = W.upsample_input((nb(32), 64, 128, 128)).to(dev)
        y = torch.empty(x.shape[:2] + (256, 256), device=dev)
        out["up"] = (H.UPSAMPLE2X, H.upsample2x_args(x, y), (x, y))
    if case in ("fused_up_pool", "pool"):
        x = W.maxpool_input((nb(32), 128, 112, 112)).to(dev)
        y = torch.empty(x.shape[:2] + (56, 56), device=dev)
        out["pool"] = (H.MAXPOOL3S2, H.maxpool3s2_args(x, y), (x, y))
    if case in ("fused_hist_philox", "hist"):
        x = W.hist_input(n1(1 << 28)).to(dev)
        b = torch.zeros(256, dtype=torch.int32, device=dev)
        out["hist"] = (H.HIST256, H.hist256_args(x, b), (x, b))
    if case in ("fused_hist_philox", "philox"):
        o = torch.empty((n1(1 << 26), 4), dtype=torch.int32, device=dev)
        out["philox"] = (H.PHILOX, H.philox_args(o, 0), (o,))
    if case in ("fused_bn_poly", "bn"):
        x = W.bn_input((8, 64, 32, 32)).to(dev)
        m, v = torch.empty(64, device=dev), torch.empty(64, device=dev)
        ws = H.bn_stats_workspace(x)
        out["bn"] = (H.BN_STATS, H.bn_stats_args(x, m, v, ws), (x, m, v, ws))
    if case in ("fused_bn_poly", "poly"):
        x = W.poly_input(n1(1 << 20)).to(dev)
        y = torch.empty_like(x)
        out["poly"] = (H.POLY, H.poly_args(x, y, W.poly_coefficients().tolist()), (x, y))
    if case == "bn_large":
        x = W.bn_input((nb(64), 256, 56, 56)).to(dev)
        m, v = torch.empty(256, device=dev), torch.empty(256, device=dev)
        ws = H.bn_stats_workspace(x)
        out["bn"] = (H.BN_STATS, H.bn_stats_args(x, m, v, ws), (x, m, v, ws))
    if case == "im2col":
        x = W.im2col_input((nb(32), 64, 56, 56)).to(dev)
        c = torch.empty(x.shape[0], 576, 3136, device=dev)
        out["im2col"] = (H.IM2COL3, H.im2col3_args(x, c), (x, c))
    if case == "bf16":
        x, y = (t.to(dev) for t in W.bf16_inputs(n1(1 << 27)))
        o = torch.empty_like(x)
        out["bf16"] = (H.BF16_AXPY, H.bf16_axpy_args(x, y, o), (x, y, o))
    hp = W.WORKLOADS["hash_pairs"]
    for k, (hname, body) in enumerate((("sha256d", H.SHA256D), ("blake256", H.BLAKE256),
                                       ("blake2b", H.BLAKE2B))):
        if case == hname or (case.startswith("fused_") and hname in case.split("_")[1:]):
            cnt = torch.zeros(1, dtype=torch.int32, device=dev)
            hits = torch.zeros(1 << 12, dtype=torch.int32, device=dev)
            a = H.hash_scan_args(W.hash_header(k), n1(hp[hname + "_n"]), 0, hp["target"], None,
                                 hits, cnt)
            out[hname] = (body, a, (cnt, hits))
    if case == "nway8":
        sp = W.WORKLOADS["nway8"]
        xb = W.bn_input((nb(64),) + sp["bn"][1:]).to(dev)
        m, v = torch.empty(256, device=dev), torch.empty(256, device=dev)
        ws = H.bn_stats_workspace(xb)
        out["bn"] = (H.BN_STATS, H.bn_stats_args(xb, m, v, ws), ())
        xi = W.im2col_input((nb(32),) + sp["im2col"][1:]).to(dev)
        ci = torch.empty(xi.shape[0], 576, 3136, device=dev)
        out["im2col"] = (H.IM2COL3, H.im2col3_args(xi, ci), ())
        xp = W.maxpool_input((nb(32),) + sp["pool"][1:]).to(dev)
        yp = torch.empty(xp.shape[:2] + (56, 56), device=dev)
        out["pool"] = (H.MAXPOOL3S2, H.maxpool3s2_args(xp, yp), ())
        xu = W.upsample_input((nb(32),) + sp["up"][1:]).to(dev)
        yu = torch.empty(xu.shape[:2] + (256, 256), device=dev)
        out["up"] = (H.UPSAMPLE2X, H.upsample2x_args(xu, yu), ())
        xh = W.hist_input(n1(sp["hist_n"])).to(dev)
        bins = torch.zeros(256, dtype=torch.int32, device=dev)
        out["hist"] = (H.HIST256, H.hist256_args(xh, bins), ())
        po = torch.empty((n1(sp["philox_n"]), 4), dtype=torch.int32, device=dev)
        out["philox"] = (H.PHILOX, H.philox_args(po, 0), ())
        xq = W.poly_input(n1(sp["poly_n"])).to(dev)
        out["poly"] = (H.POLY, H.poly_args(xq, torch.empty_like(xq), W.poly_coefficients().tolist()), ())
        x16, y16 = (t.to(dev) for t in W.bf16_inputs(n1(sp["bf16_n"])))
        out["bf16"] = (H.BF16_AXPY, H.bf16_axpy_args(x16, y16, torch.empty_like(x16)), ())
    if not out:
        raise SystemExit("unknown case " + case)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case")
    ap.add_argument("--launches", type=int, default=5)
    ap.add_argument("--split", type=int, default=0)
    ap.add_argument("--d0", type=int, default=512)
    ap.add_argument("--regcap", type=int, default=0)
    ap.add_argument("--bps", type=int, default=0)
    ap.add_argument("--threads", type=int, default=256)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--plan", default="1,3,2,1,3,2,0,1;256,128,96,32;0")
    a = ap.parse_args()
    dev = torch.device("cuda:0")
    parts = build(a.case, a.scale, dev)
    lim = H.hf_device_info()
    stream = torch.cuda.Stream()
    names = list(parts)
    if len(names) > 2:
        io, thr, cap = a.plan.split(";")
        io = [int(v) for v in io.split(",")]
        thr = [int(v) for v in thr.split(",")]
        ks = [H.hf_register_kernel(parts[nm][0]) for nm in names]
        args = [parts[nm][1] for nm in names]
        f = H.hf_fuse_n(ks, io, thr, int(cap))
        info = H.hf_query(f, args)
        grid = (a.bps or info["blocks_per_sm"]) * lim.sm_count

        def launch():
            H.hf_launch(f, args, grid, stream)
        desc = "N-way %s intervals %s cap %s grid %d regs %d" % (names, thr, cap, grid, info["regs"])
    elif len(names) == 2:
        ka = H.hf_register_kernel(parts[names[0]][0])
        kb = H.hf_register_kernel(parts[names[1]][0])
        split = a.split or a.d0 // 2
        f = H.hf_fuse(ka, kb, split, a.d0, a.regcap)
        args = [parts[names[0]][1], parts[names[1]][1]]
        info = H.hf_query(f, args)
        grid = (a.bps or info["blocks_per_sm"]) * lim.sm_count

        def launch():
            H.hf_launch(f, args, grid, stream)
        desc = "fused %s+%s split %d/%d regcap %d grid %d regs %d" % (
            names[0], names[1], split, a.d0 - split, a.regcap, grid, info["regs"])
    else:
        k = H.hf_register_kernel(parts[names[0]][0])
        args = parts[names[0]][1]
        info = H.hf_query_single(k, args, a.threads)
        grid = (a.bps or info["blocks_per_sm"]) * lim.sm_count

        def launch():
            H.hf_launch_single(k, args, a.threads, grid, stream)
        desc = "%s threads %d grid %d regs %d" % (names[0], a.threads, grid, info["regs"])
    ts = []
    with torch.cuda.stream(stream):
        for _ in range(a.launches):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            launch()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3)
    print("%s: median %.2f us over %d launches" % (desc, statistics.median(ts), a.launches))


if __name__ == "__main__":
    main()
