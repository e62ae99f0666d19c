"""Thin ctypes binding of libhfuse.so (the C ABI of include/hfuse.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  The entry points keep the C names (``hf_register_kernel``,
``hf_fuse``, ``hf_launch`` ...); the helpers at the end build argument
blocks from torch tensors, which serve only as device memory.  Importing this
module loads the library and raises if it has not been built -- there is no
fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhfuse.so")

HF_OK = 0
STATUS = {0: "HF_OK", -1: "HF_ERR_INVALID", -2: "HF_ERR_SPLIT", -3: "HF_ERR_BARRIER",
          -4: "HF_ERR_SMEM", -5: "HF_ERR_REGS", -6: "HF_ERR_UNSUPPORTED", -7: "HF_ERR_CUDA",
          -8: "HF_ERR_TIMEOUT"}

(BN_STATS, UPSAMPLE2X, MAXPOOL3S2, IM2COL3, HIST256, PHILOX, POLY, BF16_AXPY, STREAM_TMPL,
 SHA256D, BLAKE256, BLAKE2B) = range(12)
BODY_NAMES = ["bn_stats", "upsample2x", "maxpool3s2", "im2col3", "hist256", "philox", "poly",
              "bf16_axpy", "stream_tmpl", "sha256d", "blake256", "blake2b"]
HASH_BODIES = (SHA256D, BLAKE256, BLAKE2B)
MAX_INTERVALS = 15
MAX_SCHEDULE = 16

_P = ctypes.c_void_p
_i32, _i64, _u64, _f32 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float


class BnStatsArgs(ctypes.Structure):
    _fields_ = [("x", _P), ("mean", _P), ("var", _P), ("N", _i32), ("C", _i32), ("HW", _i32),
                ("workspace", _P)]


class Upsample2xArgs(ctypes.Structure):
    _fields_ = [("x", _P), ("y", _P), ("P", _i32), ("H", _i32), ("W", _i32)]


class Maxpool3s2Args(ctypes.Structure):
    _fields_ = [("x", _P), ("y", _P), ("P", _i32), ("H", _i32), ("W", _i32)]


class Im2col3Args(ctypes.Structure):
    _fields_ = [("x", _P), ("col", _P), ("N", _i32), ("C", _i32), ("H", _i32), ("W", _i32)]


class Hist256Args(ctypes.Structure):
    _fields_ = [("x", _P), ("bins", _P), ("n", _i64)]


class PhiloxArgs(ctypes.Structure):
    _fields_ = [("out", _P), ("n", _i64), ("seed", _u64), ("first", _u64)]


class PolyArgs(ctypes.Structure):
    _fields_ = [("x", _P), ("y", _P), ("n", _i64), ("iters", _i32), ("coef", _f32 * 33)]


class Bf16AxpyArgs(ctypes.Structure):
    _fields_ = [("x", _P), ("y", _P), ("out", _P), ("n", _i64), ("alpha", _f32)]


class StreamTmplArgs(ctypes.Structure):
    _fields_ = [("x", _P), ("y", _P), ("n", _i64), ("k", _i32), ("n_barriers", _i32),
                ("smem_bytes", _i32), ("a", _f32), ("b", _f32)]


class HashScanArgs(ctypes.Structure):
    _fields_ = [("header", ctypes.c_uint8 * 80), ("first", ctypes.c_uint32),
                ("target", ctypes.c_uint32), ("n", _i64), ("digests", _P), ("hits", _P),
                ("hit_count", _P), ("hit_cap", _i32)]


ARGS_TYPES = [BnStatsArgs, Upsample2xArgs, Maxpool3s2Args, Im2col3Args, Hist256Args, PhiloxArgs,
              PolyArgs, Bf16AxpyArgs, StreamTmplArgs, HashScanArgs, HashScanArgs, HashScanArgs]


class KernelDesc(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("body_id", _i32), ("min_threads", _i32),
                ("max_threads", _i32), ("thread_granularity", _i32)]


class FusedInfo(ctypes.Structure):
    _fields_ = [("regs", _i32), ("spill_bytes", _i32), ("smem_bytes", _i32),
                ("block_threads", _i32), ("blocks_per_sm", _i32),
                ("max_threads_per_block", _i32), ("n_intervals", _i32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class DeviceLimits(ctypes.Structure):
    _fields_ = [("sm_count", _i32), ("regs_per_sm", _i32), ("smem_per_sm", _i32),
                ("threads_per_sm", _i32), ("smem_per_block_optin", _i32), ("l2_bytes", _i32),
                ("cc_major", _i32), ("cc_minor", _i32)]


class TunePoint(ctypes.Structure):
    _fields_ = [("split", _i32), ("regcap", _i32), ("blocks_per_sm", _i32), ("grid", _i32),
                ("time_us", _f32), ("p10_us", _f32), ("p90_us", _f32), ("regs", _i32),
                ("spill_bytes", _i32), ("status", _i32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class NwayPlan(ctypes.Structure):
    _fields_ = [("n_intervals", _i32), ("interval_of", _i32 * 16), ("interval_threads", _i32 * 15),
                ("regcap", _i32), ("grid", _i32), ("time_us", _f32), ("evals", _i32)]

    def as_dict(self):
        n = self.n_intervals
        return {"n_intervals": n, "interval_of": list(self.interval_of),
                "interval_threads": list(self.interval_threads[:n]), "regcap": self.regcap,
                "grid": self.grid, "time_us": self.time_us, "evals": self.evals}


# cost function of hf_nway_search_sim: (plan, interval finishing times out, user) -> time
PlanCostFn = ctypes.CFUNCTYPE(_f32, ctypes.POINTER(NwayPlan), ctypes.POINTER(_f32), _P)


class BodyWork(ctypes.Structure):
    _fields_ = [("bytes", ctypes.c_double), ("ffma", ctypes.c_double), ("imul", ctypes.c_double),
                ("smem_atomic", ctypes.c_double), ("ialu", ctypes.c_double), ("barriers", _i32),
                ("reserved", _i32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class PipePeaks(ctypes.Structure):
    _fields_ = [("hbm_gbs", ctypes.c_double), ("ffma_per_s", ctypes.c_double),
                ("imul_per_s", ctypes.c_double), ("smem_atomic_per_s", ctypes.c_double),
                ("ialu_per_s", ctypes.c_double)]


class HFError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__("%s -> %s: %s" % (fn, STATUS.get(status, status), msg))
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            "libhfuse.so is not built (expected at %s); run __graft_entry__.build() or "
            "python paper_2007_01277_gb300/build.py" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "hf_register_kernel": (_i32, [ctypes.POINTER(KernelDesc), ctypes.POINTER(_P)]),
        "hf_destroy_kernel": (None, [_P]),
        "hf_fuse": (_i32, [_P, _P, _i32, _i32, _i32, ctypes.POINTER(_P)]),
        "hf_fuse_checked": (_i32, [_P, _P, _i32, _i32, ctypes.POINTER(_P)]),
        "hf_fuse_n": (_i32, [ctypes.POINTER(_P), _i32, ctypes.POINTER(_i32),
                             ctypes.POINTER(_i32), _i32, _i32, ctypes.POINTER(_P)]),
        "hf_destroy_fused": (None, [_P]),
        "hf_launch": (_i32, [_P, ctypes.POINTER(_P), _i32, _P]),
        "hf_launch_single": (_i32, [_P, _P, _i32, _i32, _P]),
        "hf_query": (_i32, [_P, ctypes.POINTER(_P), ctypes.POINTER(FusedInfo)]),
        "hf_query_single": (_i32, [_P, _P, _i32, ctypes.POINTER(FusedInfo)]),
        "hf_workspace_size": (_i32, [_i32, _P, ctypes.POINTER(ctypes.c_size_t)]),
        "hf_regcaps": (_i32, [ctypes.POINTER(_i32), _i32]),
        "hf_device_info": (_i32, [ctypes.POINTER(DeviceLimits)]),
        "hf_register_bound": (_i32, [ctypes.POINTER(DeviceLimits), _i32, _i32, _i32, _i32, _i32,
                                     ctypes.POINTER(_i32)]),
        "hf_stream_wait": (_i32, [_P, _i32]),
        "hf_time_fused": (_i32, [_P, ctypes.POINTER(_P), _i32, _i32, _i32, _P,
                                 ctypes.POINTER(_f32), ctypes.POINTER(_f32), ctypes.POINTER(_f32)]),
        "hf_time_single": (_i32, [_P, _P, _i32, _i32, _i32, _i32, _P, ctypes.POINTER(_f32),
                                  ctypes.POINTER(_f32), ctypes.POINTER(_f32)]),
        "hf_profile_pair": (_i32, [_P, _P, ctypes.POINTER(_P), _i32, ctypes.POINTER(_i32), _i32,
                                   ctypes.POINTER(_i32), _i32, ctypes.POINTER(_i32), _i32, _i32,
                                   _i32, _P, ctypes.POINTER(TunePoint)]),
        "hf_search_alg2": (_i32, [_P, _P, ctypes.POINTER(_P), _i32, _i32, _i32, _i32, _P,
                                  ctypes.POINTER(TunePoint), ctypes.POINTER(TunePoint), _i32,
                                  ctypes.POINTER(_i32)]),
        "hf_bn_stats_noalloc": (_i32, [_P, _P, _P, _i32, _i32, _i32, _i32, _i32, _P]),
        "hf_autotune_nway": (_i32, [ctypes.POINTER(_P), _i32, ctypes.POINTER(_P), _i32, _i32, _i32,
                                    _P, ctypes.POINTER(NwayPlan), ctypes.POINTER(_f32)]),
        "hf_nway_search_sim": (_i32, [_i32, ctypes.POINTER(_f32), ctypes.POINTER(_f32), PlanCostFn, _P,
                                      _i32, ctypes.POINTER(NwayPlan)]),
        "hf_calibrate": (_i32, [_i32, _P, ctypes.POINTER(ctypes.c_double)]),
        "hf_src_fuse": (_i32, [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p, _i32,
                               _i32, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
        "hf_src_compile_check": (_i32, [ctypes.c_char_p, ctypes.c_char_p, _i32, ctypes.c_char_p,
                                        ctypes.c_size_t]),
        "hf_src_load": (_i32, [ctypes.c_char_p, ctypes.c_char_p, _i32, ctypes.POINTER(_P)]),
        "hf_src_fuse_load": (_i32, [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p,
                                    _i32, _i32, _i32, ctypes.POINTER(_P)]),
        "hf_src_launch": (_i32, [_P, ctypes.POINTER(_P), _i32, _i32, ctypes.c_size_t, _P]),
        "hf_src_launch_fused": (_i32, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_size_t,
                                       ctypes.c_size_t, _i32, _P]),
        "hf_src_query": (_i32, [_P, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                ctypes.POINTER(_i32)]),
        "hf_src_unload": (None, [_P]),
        "hf_check_device_error": (_i32, [ctypes.POINTER(ctypes.c_uint), _i32]),
        "hf_autotune": (_i32, [_P, _P, ctypes.POINTER(_P), _i32, _i32, _i32, _i32, _P,
                               ctypes.POINTER(TunePoint)]),
        "hf_selftest_wait_timeout": (_i32, [_i32, _P]),
        "hf_selftest_barrier": (_i32, [_i32, _i32, _i32, _i32, _P, _P]),
        "hf_ring_plan": (_i32, [_i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_uint),
                                _i32, ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(_i32),
                                ctypes.POINTER(_i32)]),
        "hf_tmpl_features": (_i32, [ctypes.POINTER(StreamTmplArgs), ctypes.POINTER(StreamTmplArgs),
                                    _i32, _i32, _i32, _i32, _i32, _i32, ctypes.c_double,
                                    ctypes.c_double, ctypes.POINTER(_f32)]),
        "hf_mlp_forward": (_i32, [_P, _P, _i32, _P, _P]),
        "hf_body_work_of": (_i32, [_i32, _P, ctypes.POINTER(BodyWork)]),
        "hf_pair_features": (_i32, [_P, _P, _P, _i32, _i32, _i32, _i32, _i32, _i32,
                                    ctypes.POINTER(PipePeaks), ctypes.POINTER(_f32)]),
        "hf_autotune_model": (_i32, [_P, _P, _P, _i32, _i32, _i32, _P, ctypes.POINTER(TunePoint),
                                     ctypes.POINTER(_i32)]),
        "hf_cost_model_set": (_i32, [_P, _i32, _f32, _f32, ctypes.POINTER(PipePeaks), _i32]),
        "hf_mlp_train": (_i32, [_P, _P, _P, _P, _P, _P, _i32, _i32, _f32, _f32, _f32, _f32, _i32,
                                _P, _P, _P]),
        "hf_mlp_nparams": (_i32, []),
        "hf_launch_traced": (_i32, [_P, ctypes.POINTER(_P), _i32, _P, _P]),
        "hf_graph_begin": (_i32, [_P]),
        "hf_graph_end": (_i32, [_P, ctypes.POINTER(_P)]),
        "hf_graph_launch": (_i32, [_P, _P]),
        "hf_graph_destroy": (None, [_P]),
        "hf_status_string": (ctypes.c_char_p, [_i32]),
        "hf_last_error": (ctypes.c_char_p, []),
        "hf_args_size": (ctypes.c_size_t, [_i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def _check(fn, status):
    if status != HF_OK:
        raise HFError(fn, status, lib.hf_last_error().decode())


def _stream_ptr(stream):
    """A torch.cuda.Stream, a raw cudaStream_t int, or None (current stream)."""
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ----------------------------------------------------------------- C entry points
def hf_register_kernel(body_id, min_threads=0, max_threads=0, granularity=0, name=None):
    d = KernelDesc(name.encode() if name else None, body_id, min_threads, max_threads, granularity)
    h = _P()
    _check("hf_register_kernel", lib.hf_register_kernel(ctypes.byref(d), ctypes.byref(h)))
    return h


def hf_fuse(a, b, split, d0, regcap=0):
    h = _P()
    _check("hf_fuse", lib.hf_fuse(a, b, split, d0, regcap, ctypes.byref(h)))
    return h


def hf_fuse_checked(a, b, split, d0):
    """hf_fuse from the checked build: interval barriers are bounded
    software barriers (an expired wait sets ERR_BARRIER_EXPIRED)."""
    h = _P()
    _check("hf_fuse_checked", lib.hf_fuse_checked(a, b, split, d0, ctypes.byref(h)))
    return h


def hf_fuse_n(kernels, interval_of, interval_threads, regcap=0):
    n, ni = len(kernels), len(interval_threads)
    ks = (_P * n)(*kernels)
    io = (_i32 * n)(*interval_of)
    it = (_i32 * ni)(*interval_threads)
    h = _P()
    _check("hf_fuse_n", lib.hf_fuse_n(ks, n, io, it, ni, regcap, ctypes.byref(h)))
    return h


def _argv(args):
    return (_P * len(args))(*[ctypes.cast(ctypes.pointer(a), _P) for a in args])


def hf_launch(f, args, grid=0, stream=None):
    _check("hf_launch", lib.hf_launch(f, _argv(args), grid, _stream_ptr(stream)))


def hf_launch_single(k, args, threads, grid=0, stream=None):
    _check("hf_launch_single", lib.hf_launch_single(k, ctypes.cast(ctypes.pointer(args), _P),
                                                    threads, grid, _stream_ptr(stream)))


def hf_query(f, args):
    info = FusedInfo()
    _check("hf_query", lib.hf_query(f, _argv(args), ctypes.byref(info)))
    return info.as_dict()


def hf_query_single(k, args, threads):
    info = FusedInfo()
    _check("hf_query_single", lib.hf_query_single(k, ctypes.cast(ctypes.pointer(args), _P),
                                                  threads, ctypes.byref(info)))
    return info.as_dict()


def hf_workspace_size(body_id, args):
    n = ctypes.c_size_t()
    _check("hf_workspace_size", lib.hf_workspace_size(body_id, ctypes.cast(ctypes.pointer(args), _P),
                                                      ctypes.byref(n)))
    return n.value


def hf_regcaps():
    buf = (_i32 * 32)()
    n = lib.hf_regcaps(buf, 32)
    return list(buf[:n])


def hf_device_info():
    lim = DeviceLimits()
    _check("hf_device_info", lib.hf_device_info(ctypes.byref(lim)))
    return lim


def hf_register_bound(lim, d1, nregs1, d2, nregs2, smem_fused):
    r = _i32()
    _check("hf_register_bound", lib.hf_register_bound(ctypes.byref(lim), d1, nregs1, d2, nregs2,
                                                      smem_fused, ctypes.byref(r)))
    return r.value


def hf_stream_wait(stream=None, timeout_ms=10000):
    _check("hf_stream_wait", lib.hf_stream_wait(_stream_ptr(stream), timeout_ms))


def hf_destroy_fused(f):
    lib.hf_destroy_fused(f)


def hf_destroy_kernel(k):
    lib.hf_destroy_kernel(k)


# ----------------------------------------------------------------- argument blocks
# An argument block holds raw device addresses; it also keeps a reference to
# the tensors behind them (attribute _keep), so that memory cannot be freed
# and reused while the block can still be launched.
def _ptr(t):
    return t.data_ptr() if t is not None else None


def _keep(block, *tensors):
    block._keep = tensors
    return block


def bn_stats_args(x, mean, var, workspace=None):
    N, C, H, W = x.shape
    a = BnStatsArgs(_ptr(x), _ptr(mean), _ptr(var), N, C, H * W, None)
    if workspace is not None:
        a.workspace = _ptr(workspace)
    return _keep(a, x, mean, var, workspace)


def bn_stats_workspace(x):
    """Zero-filled device workspace for bn_stats on x (counters must start
    at zero; every launch leaves them zero)."""
    import torch
    n = hf_workspace_size(BN_STATS, bn_stats_args(x, None, None))
    return torch.zeros(max(n, 16), dtype=torch.uint8, device=x.device)


def upsample2x_args(x, y):
    H, W = x.shape[-2:]
    return _keep(Upsample2xArgs(_ptr(x), _ptr(y), x.numel() // (H * W), H, W), x, y)


def maxpool3s2_args(x, y):
    H, W = x.shape[-2:]
    return _keep(Maxpool3s2Args(_ptr(x), _ptr(y), x.numel() // (H * W), H, W), x, y)


def im2col3_args(x, col):
    N, C, H, W = x.shape
    return _keep(Im2col3Args(_ptr(x), _ptr(col), N, C, H, W), x, col)


def hist256_args(x, bins):
    return _keep(Hist256Args(_ptr(x), _ptr(bins), x.numel()), x, bins)


def philox_args(out, seed, first=0):
    return _keep(PhiloxArgs(_ptr(out), out.numel() // 4, seed, first), out)


def poly_args(x, y, coef, iters=64):
    c = (_f32 * 33)(*[float(v) for v in coef])
    return _keep(PolyArgs(_ptr(x), _ptr(y), x.numel(), iters, c), x, y)


def bf16_axpy_args(x, y, out, alpha=0.5):
    return _keep(Bf16AxpyArgs(_ptr(x), _ptr(y), _ptr(out), x.numel(), alpha), x, y, out)


def stream_tmpl_args(x, y, k, n_barriers=0, smem_bytes=0, a=0.999, b=0.001):
    return _keep(StreamTmplArgs(_ptr(x), _ptr(y), x.numel(), k, n_barriers, smem_bytes, a, b), x, y)


def hash_scan_args(header, n, first=0, target=0, digests=None, hits=None, hit_count=None):
    """Argument block of the three hash scans (same layout for each).
    header: 80 bytes; digests: None or a uint8 tensor of n*32 bytes; hits:
    None or an int32 tensor (its length is the capacity); hit_count: None or
    a zeroed int32 tensor of one element."""
    h = bytes(header)
    if len(h) != 80:
        raise ValueError("the header is 80 bytes")
    a = HashScanArgs((ctypes.c_uint8 * 80)(*h), first & 0xFFFFFFFF, target & 0xFFFFFFFF, n,
                     _ptr(digests), _ptr(hits), _ptr(hit_count),
                     0 if hits is None else hits.numel())
    return _keep(a, digests, hits, hit_count)


# ----------------------------------------------------------------- profiling search
def hf_time_fused(f, args, grid=0, reps=10, flush_l2=True, stream=None):
    m, lo, hi = _f32(), _f32(), _f32()
    _check("hf_time_fused", lib.hf_time_fused(f, _argv(args), grid, reps, int(flush_l2),
                                              _stream_ptr(stream), ctypes.byref(m), ctypes.byref(lo),
                                              ctypes.byref(hi)))
    return m.value, lo.value, hi.value


def hf_time_single(k, args, threads, grid=0, reps=10, flush_l2=True, stream=None):
    m, lo, hi = _f32(), _f32(), _f32()
    _check("hf_time_single", lib.hf_time_single(k, ctypes.cast(ctypes.pointer(args), _P), threads,
                                                grid, reps, int(flush_l2), _stream_ptr(stream),
                                                ctypes.byref(m), ctypes.byref(lo), ctypes.byref(hi)))
    return m.value, lo.value, hi.value


def hf_profile_pair(a, b, args, d0, splits, regcaps, bps, reps=5, flush_l2=True, stream=None):
    n = len(splits) * len(regcaps) * len(bps)
    table = (TunePoint * n)()
    _check("hf_profile_pair", lib.hf_profile_pair(
        a, b, _argv(args), d0, (_i32 * len(splits))(*splits), len(splits),
        (_i32 * len(regcaps))(*regcaps), len(regcaps), (_i32 * len(bps))(*bps), len(bps), reps,
        int(flush_l2), _stream_ptr(stream), table))
    return [p.as_dict() for p in table]


def hf_search_alg2(a, b, args, d0, step=128, reps=5, flush_l2=True, stream=None):
    best = TunePoint()
    trace = (TunePoint * 64)()
    nt = _i32()
    _check("hf_search_alg2", lib.hf_search_alg2(a, b, _argv(args), d0, step, reps, int(flush_l2),
                                                _stream_ptr(stream), ctypes.byref(best), trace, 64,
                                                ctypes.byref(nt)))
    return best.as_dict(), [trace[i].as_dict() for i in range(min(nt.value, 64))]


# ----------------------------------------------------------------- allocation-free entry point
def hf_bn_stats_noalloc(x, mean, var, threads=256, grid=0, stream=None):
    """Batch-norm statistics through the entry point that allocates nothing
    (its scratch is a fixed device array inside the library)."""
    N, C, Hh, Ww = x.shape
    _check("hf_bn_stats_noalloc", lib.hf_bn_stats_noalloc(
        _ptr(x), _ptr(mean), _ptr(var), N, C, Hh * Ww, threads, grid, _stream_ptr(stream)))


# ----------------------------------------------------------------- N-way autotuner, calibration, graphs
def hf_autotune_nway(kernels, args, max_evals=200, reps=5, flush_l2=False, stream=None):
    n = len(kernels)
    plan = NwayPlan()
    single = (_f32 * n)()
    _check("hf_autotune_nway", lib.hf_autotune_nway((_P * n)(*kernels), n, _argv(args), max_evals,
                                                    reps, int(flush_l2), _stream_ptr(stream),
                                                    ctypes.byref(plan), single))
    d = plan.as_dict()
    d["interval_of"] = d["interval_of"][:n]
    return d, list(single)


def hf_nway_search_sim(standalone_us, cost, max_evals=200, issue_us=None):
    """The N-way search against cost(plan_dict) -> (time, [finish per
    interval]) instead of the GPU; issue_us (optional) are the kernels'
    busiest-pipe times; returns the plan dict (with "evals")."""
    n = len(standalone_us)

    def cb(plan_p, fin_p, _user):
        q = plan_p.contents.as_dict()
        q["interval_of"] = q["interval_of"][:n]
        t, fin = cost(q)
        for i, v in enumerate(fin[:q["n_intervals"]]):
            fin_p[i] = v
        return t

    fn = PlanCostFn(cb)
    plan = NwayPlan()
    iss = (_f32 * n)(*issue_us) if issue_us is not None else None
    _check("hf_nway_search_sim", lib.hf_nway_search_sim(n, (_f32 * n)(*standalone_us), iss, fn, None,
                                                        max_evals, ctypes.byref(plan)))
    d = plan.as_dict()
    d["interval_of"] = d["interval_of"][:n]
    return d


CAL_FFMA, CAL_IMUL, CAL_SMEM_ATOMIC, CAL_IALU = 0, 1, 2, 3


def hf_calibrate(what, stream=None):
    v = ctypes.c_double()
    _check("hf_calibrate", lib.hf_calibrate(what, _stream_ptr(stream), ctypes.byref(v)))
    return v.value


def hf_graph_begin(stream):
    _check("hf_graph_begin", lib.hf_graph_begin(_stream_ptr(stream)))


def hf_graph_end(stream):
    g = _P()
    _check("hf_graph_end", lib.hf_graph_end(_stream_ptr(stream), ctypes.byref(g)))
    return g


def hf_graph_launch(g, stream=None):
    _check("hf_graph_launch", lib.hf_graph_launch(g, _stream_ptr(stream)))


def hf_graph_destroy(g):
    lib.hf_graph_destroy(g)


# ----------------------------------------------------------------- learned cost model
MLP_NPARAMS = 5825
MLP_FEATURES = 24


def hf_tmpl_features(a, b, split, d0, regcap, bps, fused_regs, spill_bytes, hbm_gbs, ffma_per_s):
    out = (_f32 * MLP_FEATURES)()
    _check("hf_tmpl_features", lib.hf_tmpl_features(ctypes.byref(a), ctypes.byref(b), split, d0,
                                                    regcap, bps, fused_regs, spill_bytes,
                                                    float(hbm_gbs), float(ffma_per_s), out))
    return list(out)


def hf_mlp_forward(params, X, y, stream=None):
    _check("hf_mlp_forward", lib.hf_mlp_forward(_ptr(params), _ptr(X), X.shape[0], _ptr(y),
                                                _stream_ptr(stream)))


def hf_mlp_train(params, m, v, X, Y, idx, steps, batch, lr=1e-3, beta1=0.9, beta2=0.999,
                 eps=1e-8, t0=0, loss_out=None, grad_out=None, stream=None):
    _check("hf_mlp_train", lib.hf_mlp_train(_ptr(params), _ptr(m), _ptr(v), _ptr(X), _ptr(Y),
                                            _ptr(idx), steps, batch, lr, beta1, beta2, eps, t0,
                                            _ptr(loss_out), _ptr(grad_out), _stream_ptr(stream)))


def hf_launch_traced(f, args, grid=0, stream=None):
    """hf_launch of an N-way fused kernel that returns per-interval
    (start, end) in nanoseconds of the global timer."""
    import torch
    n_int = 15
    tr = torch.zeros(2 * n_int, dtype=torch.int64, device="cuda")
    tr[0::2] = -1   # all ones: the unsigned maximum
    _check("hf_launch_traced", lib.hf_launch_traced(f, _argv(args), grid, _stream_ptr(stream),
                                                    tr.data_ptr()))
    torch.cuda.synchronize()
    h = tr.cpu().numpy().view("uint64")
    return [(int(h[2 * i]), int(h[2 * i + 1])) for i in range(n_int) if h[2 * i + 1] > 0]


# ----------------------------------------------------------------- source front-end
def _b(x):
    return None if x is None else (x.encode() if isinstance(x, str) else bytes(x))


def hf_src_fuse(src_a, name_a, src_b, name_b, split, d0):
    """The generated CUDA source of the fused kernel (Algorithm 1 on source)."""
    n = ctypes.c_size_t()
    _check("hf_src_fuse", lib.hf_src_fuse(_b(src_a), _b(name_a), _b(src_b), _b(name_b), split, d0,
                                          None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check("hf_src_fuse", lib.hf_src_fuse(_b(src_a), _b(name_a), _b(src_b), _b(name_b), split, d0,
                                          buf, n.value, ctypes.byref(n)))
    return buf.value.decode()


def hf_src_compile_check(src, name, regcap=0):
    """Compile with NVRTC (no GPU needed); returns the compiler log."""
    log = ctypes.create_string_buffer(1 << 16)
    _check("hf_src_compile_check", lib.hf_src_compile_check(_b(src), _b(name), regcap, log, len(log)))
    return log.value.decode(errors="replace")


def hf_src_load(src, name, regcap=0):
    h = _P()
    _check("hf_src_load", lib.hf_src_load(_b(src), _b(name), regcap, ctypes.byref(h)))
    return h


def hf_src_fuse_load(src_a, name_a, src_b, name_b, split, d0, regcap=0):
    h = _P()
    _check("hf_src_fuse_load", lib.hf_src_fuse_load(_b(src_a), _b(name_a), _b(src_b), _b(name_b), split,
                                                    d0, regcap, ctypes.byref(h)))
    return h


class KernelParams:
    """Parameter values of a source kernel in launch order: torch tensors
    pass their device pointer, ctypes values pass as they are, Python ints
    as C int and floats as C float.  Holds the values while it lives."""

    def __init__(self, *values):
        self.vals = []
        for v in values:
            if hasattr(v, "data_ptr"):
                self.vals.append(ctypes.c_void_p(v.data_ptr()))
            elif isinstance(v, ctypes._SimpleCData):
                self.vals.append(v)
            elif isinstance(v, bool) or not isinstance(v, (int, float)):
                raise TypeError("unsupported parameter value %r" % (v,))
            elif isinstance(v, int):
                self.vals.append(ctypes.c_int(v))
            else:
                self.vals.append(ctypes.c_float(v))
        self.keep = values
        self.array = (_P * max(1, len(self.vals)))(
            *[ctypes.cast(ctypes.pointer(v), _P) for v in self.vals])


def hf_src_launch(m, params, grid, block, dyn_smem=0, stream=None):
    _check("hf_src_launch", lib.hf_src_launch(m, params.array, grid, block, dyn_smem, _stream_ptr(stream)))


def hf_src_launch_fused(m, params_a, params_b, grid, dyn_smem_a=0, dyn_smem_b=0, stream=None):
    _check("hf_src_launch_fused", lib.hf_src_launch_fused(m, params_a.array, params_b.array, dyn_smem_a,
                                                          dyn_smem_b, grid, _stream_ptr(stream)))


def hf_src_query(m):
    r, l, s_, t = _i32(), _i32(), _i32(), _i32()
    _check("hf_src_query", lib.hf_src_query(m, ctypes.byref(r), ctypes.byref(l), ctypes.byref(s_),
                                            ctypes.byref(t)))
    return {"regs": r.value, "local_bytes": l.value, "static_smem": s_.value, "max_threads": t.value}


def hf_src_unload(m):
    lib.hf_src_unload(m)


# ----------------------------------------------------------------- device errors
ERR_WAIT_EXPIRED = 1
ERR_BARRIER_EXPIRED = 2


def hf_check_device_error(clear=False):
    """The device error word (read after the launches have finished)."""
    v = ctypes.c_uint()
    _check("hf_check_device_error", lib.hf_check_device_error(ctypes.byref(v), int(clear)))
    return v.value


def hf_selftest_wait_timeout(limit_us, stream=None):
    _check("hf_selftest_wait_timeout", lib.hf_selftest_wait_timeout(limit_us, _stream_ptr(stream)))


def hf_selftest_barrier(warps, missing, rounds, limit_us, completed=None, stream=None):
    """completed: an int32 device tensor of one element (or None)."""
    ptr = _ptr(completed) if completed is not None else None
    _check("hf_selftest_barrier", lib.hf_selftest_barrier(warps, missing, rounds, limit_us, ptr,
                                                          _stream_ptr(stream)))


TUNE_EXHAUSTIVE, TUNE_ALG2, TUNE_MODEL = 0, 1, 2


def hf_body_work_of(body_id, args):
    """Algorithmic bytes and operations per pipe of one launch (dict)."""
    w = BodyWork()
    _check("hf_body_work_of", lib.hf_body_work_of(body_id, ctypes.cast(ctypes.pointer(args), _P),
                                                  ctypes.byref(w)))
    return w.as_dict()


def pipe_peaks(hbm_gbs, ffma, imul, smem_atomic, ialu):
    return PipePeaks(float(hbm_gbs), float(ffma), float(imul), float(smem_atomic), float(ialu))


def hf_pair_features(a, b, args, split, d0, regcap, bps, fused_regs, spill_bytes, peaks):
    out = (_f32 * MLP_FEATURES)()
    _check("hf_pair_features", lib.hf_pair_features(a, b, _argv(args), split, d0, regcap, bps,
                                                    fused_regs, spill_bytes, ctypes.byref(peaks), out))
    return list(out)


def hf_autotune_model(a, b, args, d0=512, reps=5, flush_l2=False, stream=None):
    """hf_autotune(TUNE_MODEL) plus the number of candidates it timed:
    returns (point dict, n_timed)."""
    best = TunePoint()
    n = _i32()
    _check("hf_autotune_model", lib.hf_autotune_model(a, b, _argv(args), d0, reps, int(flush_l2),
                                                      _stream_ptr(stream), ctypes.byref(best),
                                                      ctypes.byref(n)))
    return best.as_dict(), n.value


def hf_cost_model_set(params, mu, sd, peaks, confirm=5):
    """Installs the trained perceptron(s) for hf_autotune(..., TUNE_MODEL):
    params is one float32 tensor of MLP_NPARAMS values or a list of them
    (an ensemble whose mean prediction ranks the candidates); copied."""
    if params is None:
        _check("hf_cost_model_set", lib.hf_cost_model_set(None, 0, 0.0, 1.0, None, 1))
        return
    import numpy as np
    sets = params if isinstance(params, (list, tuple)) else [params]
    host = np.ascontiguousarray(np.concatenate([
        np.asarray(p.detach().cpu() if hasattr(p, "detach") else p, dtype=np.float32).reshape(-1)
        for p in sets]))
    assert host.size == MLP_NPARAMS * len(sets)
    _check("hf_cost_model_set", lib.hf_cost_model_set(host.ctypes.data_as(_P), len(sets), float(mu),
                                                      float(sd), ctypes.byref(peaks), int(confirm)))


def hf_autotune(a, b, args, d0=512, mode=TUNE_EXHAUSTIVE, reps=5, flush_l2=False, stream=None):
    """The (split, regcap, blocks_per_sm) to launch the pair with, by the
    exhaustive profile or Algorithm 2; returns the timed point as a dict."""
    best = TunePoint()
    _check("hf_autotune", lib.hf_autotune(a, b, _argv(args), d0, mode, reps, int(flush_l2),
                                          _stream_ptr(stream), ctypes.byref(best)))
    return best.as_dict()


RING_NONE, RING_STREAM, RING_ITEM = 0, 1, 2


def hf_ring_plan(warps, ring, min_bytes, blocks_per_sm):
    """([stage bytes], [stages], [uses]) per interval of the launch planner's
    ring decision; ring[i] is RING_NONE, RING_STREAM or RING_ITEM."""
    n = len(warps)
    st, ns, uses = (ctypes.c_uint * n)(), (_i32 * n)(), (_i32 * n)()
    _check("hf_ring_plan", lib.hf_ring_plan(n, (_i32 * n)(*warps), (_i32 * n)(*[int(r) for r in ring]),
                                            (ctypes.c_uint * n)(*min_bytes), blocks_per_sm, st, ns, uses))
    return list(st), list(ns), list(uses)
