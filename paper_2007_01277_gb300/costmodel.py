"""Learned cost model for the fusion search.

Algorithm 2 (Sec. 3.2) profiles every candidate configuration of a pair.
Here the exhaustive profile of a corpus of generated pairs becomes training
data for a small perceptron that predicts log(fused time) from static
features; for a new pair the model scores every candidate with one inference
launch and the search keeps the predicted best (optionally confirming the
top few by timing).  The exhaustive search stays the fallback and the yardstick:
regret = t(model's pick) / t(exhaustive best) - 1, both read from the
exhaustive table of held-out pairs.

Pipeline (all numerical work in the library's kernels):
  corpus     600 pairs of the parametric stream kernel, seed 0: per kernel
             k in {0,1,2,4,...,256} FMAs per 16 B, 0-4 barriers, 0-48 KB
             of shared staging, 2^20..2^28 floats (log-uniform)
  profile    hf_profile_pair over splits 1:7..7:1 warps of a 256-thread
             block x register caps {none,32,40,48,64,96} x 1-4 blocks/SM,
             L2 flushed before every timed launch; one JSONL record per
             pair (resumable)
  features   hf_tmpl_features (24 per point)
  train      hf_mlp_train on 500 pairs, Adam, one kernel launch
  evaluate   hf_mlp_forward on the 100 held-out pairs -> regret
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np
import torch

from . import experiments as _E
from . import hfuse as H
from . import workloads as W

K_CHOICES = (0, 1, 2, 4, 8, 16, 32, 64, 128, 256)
SMEM_CHOICES = (0, 4096, 8192, 16384, 24576, 32768, 49152)
D0 = 256
SPLITS = tuple(range(32, 256, 32))
CAPS = (0, 32, 40, 48, 64, 96)
BPS = (1, 2, 3, 4)
MAX_N = 1 << 28


def make_corpus(n_pairs: int = 600, seed: int = 0, max_log2: int = 28):
    g = torch.Generator().manual_seed(seed)

    def one():
        k = K_CHOICES[int(torch.randint(len(K_CHOICES), (1,), generator=g))]
        nb = int(torch.randint(5, (1,), generator=g))
        sm = SMEM_CHOICES[int(torch.randint(len(SMEM_CHOICES), (1,), generator=g))]
        n = W.log_uniform_int(1 << 20, 1 << max_log2, g)
        return {"k": k, "n_barriers": nb, "smem_bytes": sm, "n": n}
    return [{"id": i, "a": one(), "b": one()} for i in range(n_pairs)]


class Pool:
    """Device buffers sized for the largest kernel; pairs use prefixes."""

    def __init__(self, dev, max_n=MAX_N):
        self.xa = W.template_input(max_n, seed=11).to(dev)
        self.xb = W.template_input(max_n, seed=12).to(dev)
        self.ya = torch.empty(max_n, device=dev)
        self.yb = torch.empty(max_n, device=dev)

    def args(self, pair):
        a, b = pair["a"], pair["b"]
        return [H.stream_tmpl_args(self.xa[:a["n"]], self.ya[:a["n"]], a["k"], a["n_barriers"],
                                   a["smem_bytes"]),
                H.stream_tmpl_args(self.xb[:b["n"]], self.yb[:b["n"]], b["k"], b["n_barriers"],
                                   b["smem_bytes"])]


def profile_corpus(pairs, db_path, pool, reps=3, flush=True, log=None):
    """Exhaustive profile of every pair not yet in the JSONL file."""
    done = set()
    if os.path.exists(db_path):
        for line in open(db_path):
            try:
                done.add(json.loads(line)["id"])
            except (ValueError, KeyError):
                continue
    ka = H.hf_register_kernel(H.STREAM_TMPL)
    kb = H.hf_register_kernel(H.STREAM_TMPL)
    t0 = time.time()
    with open(db_path, "a") as f:
        for p in pairs:
            if p["id"] in done:
                continue
            table = H.hf_profile_pair(ka, kb, pool.args(p), D0, list(SPLITS), list(CAPS), list(BPS),
                                      reps=reps, flush_l2=flush)
            rec = dict(p)
            rec["points"] = [[q["split"], q["regcap"], q["blocks_per_sm"], round(q["time_us"], 3),
                              q["regs"], q["spill_bytes"], q["status"]] for q in table]
            f.write(json.dumps(rec) + "\n")
            f.flush()
            if log and p["id"] % 50 == 0:
                log("profiled pair %d (%.0f s)" % (p["id"], time.time() - t0))
    return load_db(db_path)


def load_db(db_path):
    recs = {}
    for line in open(db_path):
        r = json.loads(line)
        recs[r["id"]] = r
    return [recs[i] for i in sorted(recs)]


def _targs(spec):
    return H.StreamTmplArgs(None, None, spec["n"], spec["k"], spec["n_barriers"], spec["smem_bytes"],
                            0.999, 0.001)


def featurize(recs, hbm_gbs, ffma_per_s):
    """Rows of (pair index, point index, features, log time) for valid points."""
    X, Y, owner = [], [], []
    for pi, r in enumerate(recs):
        a, b = _targs(r["a"]), _targs(r["b"])
        for qi, (split, cap, bps, t, regs, spill, st) in enumerate(r["points"]):
            if st != 0 or t <= 0:
                continue
            X.append(H.hf_tmpl_features(a, b, split, D0, cap, bps, regs, spill, hbm_gbs, ffma_per_s))
            Y.append(math.log(t))
            owner.append((pi, qi))
    return np.asarray(X, np.float32), np.asarray(Y, np.float32), owner


def xavier_params(seed=0):
    g = torch.Generator().manual_seed(seed)

    def u(fan_in, fan_out, shape):
        a = math.sqrt(6.0 / (fan_in + fan_out))
        return (torch.rand(shape, generator=g) * 2 - 1) * a
    parts = [u(24, 64, (64 * 24,)), torch.zeros(64), u(64, 64, (64 * 64,)), torch.zeros(64),
             u(64, 1, (64,)), torch.zeros(1)]
    return torch.cat(parts).float()


def train(X, Y, dev, steps=20000, batch=64, lr=1e-3, seed=0):
    """Standardises the target, trains on the device, returns (params, mu, sd, losses)."""
    mu, sd = float(Y.mean()), float(Y.std() + 1e-8)
    Xd = torch.from_numpy(X).to(dev)
    Yd = torch.from_numpy((Y - mu) / sd).to(dev)
    P = xavier_params(seed).to(dev)
    M = torch.zeros_like(P)
    V = torch.zeros_like(P)
    g = torch.Generator().manual_seed(seed + 1)
    idx = torch.randint(0, X.shape[0], (steps * batch,), generator=g, dtype=torch.int32).to(dev)
    loss = torch.empty(steps, device=dev)
    H.hf_mlp_train(P, M, V, Xd, Yd, idx, steps, batch, lr=lr, loss_out=loss)
    torch.cuda.synchronize()
    return P, mu, sd, loss.cpu().numpy()


def predict(P, X, mu, sd, dev):
    Xd = torch.from_numpy(X).to(dev)
    y = torch.empty(X.shape[0], device=dev)
    H.hf_mlp_forward(P, Xd, y)
    torch.cuda.synchronize()
    return y.cpu().numpy() * sd + mu


def regret(recs, owner, pred_log, confirm=1):
    """Per pair: time of the model's pick (best measured among its `confirm`
    lowest predictions) over the exhaustive best, minus one."""
    by_pair = {}
    for (pi, qi), p in zip(owner, pred_log):
        by_pair.setdefault(pi, []).append((p, qi))
    out = []
    for pi, cand in by_pair.items():
        pts = recs[pi]["points"]
        best = min(pts[qi][3] for _, qi in cand)
        cand.sort()
        pick = min(pts[qi][3] for _, qi in cand[:confirm])
        out.append(pick / best - 1.0)
    return np.asarray(out)


def summarize(r):
    return {"mean": float(r.mean()), "geomean": float(np.exp(np.log1p(r).mean()) - 1),
            "p90": float(np.quantile(r, 0.9)), "max": float(r.max()),
            "within_5pct": float((r <= 0.05).mean()), "pairs": int(r.size)}


def run(dev, db_path, n_pairs=600, n_train=500, steps=20000, reps=3, hbm_gbs=6785.9, log=print):
    pairs = make_corpus(n_pairs)
    pool = Pool(dev)
    t0 = time.time()
    recs = profile_corpus(pairs, db_path, pool, reps=reps, log=log)
    t_profile = time.time() - t0
    ffma = H.hf_calibrate(H.CAL_FFMA)
    train_recs = [r for r in recs if r["id"] < n_train]
    test_recs = [r for r in recs if r["id"] >= n_train]
    Xtr, Ytr, _ = featurize(train_recs, hbm_gbs, ffma)
    Xte, Yte, own_te = featurize(test_recs, hbm_gbs, ffma)
    t1 = time.time()
    P, mu, sd, losses = train(Xtr, Ytr, dev, steps=steps)
    t_train = time.time() - t1
    t2 = time.time()
    pred = predict(P, Xte, mu, sd, dev)
    t_infer = time.time() - t2
    pred_tr = predict(P, Xtr, mu, sd, dev)
    res = {
        "pairs": len(recs), "train_pairs": len(train_recs), "test_pairs": len(test_recs),
        "train_points": int(Xtr.shape[0]), "test_points": int(Xte.shape[0]),
        "profile_s": round(t_profile, 1), "train_s": round(t_train, 3), "infer_s": round(t_infer, 4),
        "train_loss_first_last": [float(losses[:100].mean()), float(losses[-100:].mean())],
        "rmse_log_test": float(np.sqrt(np.mean((pred - Yte) ** 2))),
        "rmse_log_train": float(np.sqrt(np.mean((pred_tr - Ytr) ** 2))),
        "regret": summarize(regret(test_recs, own_te, pred, 1)),
        "regret_top3_confirmed": summarize(regret(test_recs, own_te, pred, 3)),
        "points_per_pair_exhaustive": len(SPLITS) * len(CAPS) * len(BPS),
    }
    return res, P, (mu, sd)


# ------------------------------------------------------------------ built-in pairs
# The model also learns from the library's own bodies: every pair type the
# workloads fuse (batch-norm + polynomial, histogram + Philox, upsample +
# max pool) and the ten Table-2 pairs of the deep-learning kernels, each
# profiled exhaustively at sizes below its workload size.  The workload
# sizes themselves are held out: the model's pick there is judged against
# the exhaustive table of the same sizes.
BUILTIN_PAIRS = {
    "bn_poly": (("bn_small", "poly"), 512),
    "hist_philox": (("hist_big", "philox"), 256),
    "upsample_maxpool": (("upsample_big", "maxpool"), 512),
}
for _i, _a in enumerate(_E.DL_BODIES):
    for _b in _E.DL_BODIES[_i + 1:]:
        BUILTIN_PAIRS[_a + "_" + _b] = ((_a, _b), 512)
BUILTIN_TARGETS = ("bn_poly", "hist_philox", "upsample_maxpool")
# training sizes bracket the held-out workload size (scale 1)
TRAIN_SCALES = (1 / 16, 1 / 8, 1 / 4, 1 / 2, 2, 4)
BUILTIN_CAPS = (0, 32, 40, 48, 64, 96, 128)
ENSEMBLE_SEEDS = (0, 1, 2)

# Workload size of each kernel kind: (body, leading dimension or element
# count, the rest of the shape).  Scaled kernels take a prefix of it.
_KINDS = {
    "bn_small": ("bn", 8, (64, 32, 32)), "poly": ("poly", 1 << 20, ()),
    "hist_big": ("hist", 1 << 28, ()), "philox": ("philox", 1 << 26, ()),
    "upsample_big": ("upsample", 32, (64, 128, 128)), "bn": ("bn", 64, (256, 56, 56)),
    "hist": ("hist", 1 << 27, ()), "maxpool": ("maxpool", 32, (128, 112, 112)),
    "upsample": ("upsample", 16, (64, 128, 128)), "im2col": ("im2col", 32, (64, 56, 56)),
}


class CorpusPool:
    """Device buffers of every kernel kind at the largest scale, drawn on the
    device (the corpus is only timed, never compared with the oracle, so the
    values need the workloads' distributions but not their exact bytes);
    scaled kernels use prefixes along the leading dimension."""

    def __init__(self, dev, max_scale, seed=0):
        self.dev, self.max_scale, self.buf = dev, max_scale, {}
        self.g = torch.Generator(device=dev)
        self.g.manual_seed(seed)

    def _lead(self, kind, scale):
        _body, n, _rest = _KINDS[kind]
        return max(1, int(round(n * scale)))

    def _get(self, kind):
        if kind in self.buf:
            return self.buf[kind]
        body, _n, rest = _KINDS[kind]
        L = self._lead(kind, self.max_scale)
        dev, g = self.dev, self.g
        if body == "bn":
            b = {"x": torch.randn((L,) + rest, device=dev, generator=g)}
        elif body == "poly":
            b = {"x": torch.rand(L, device=dev, generator=g) * 2 - 1, "y": torch.empty(L, device=dev)}
        elif body == "hist":
            b = {"x": torch.randint(0, 256, (L,), device=dev, generator=g, dtype=torch.uint8)}
        elif body == "philox":
            b = {"y": torch.empty((L, 4), dtype=torch.int32, device=dev)}
        elif body == "upsample":
            b = {"x": torch.rand((L,) + rest, device=dev, generator=g),
                 "y": torch.empty((L, rest[0], 2 * rest[1], 2 * rest[2]), device=dev)}
        elif body == "maxpool":
            b = {"x": torch.randn((L,) + rest, device=dev, generator=g),
                 "y": torch.empty((L, rest[0], (rest[1] - 1) // 2 + 1, (rest[2] - 1) // 2 + 1), device=dev)}
        else:   # im2col
            b = {"x": torch.randn((L,) + rest, device=dev, generator=g),
                 "y": torch.empty((L, rest[0] * 9, rest[1] * rest[2]), device=dev)}
        self.buf[kind] = b
        return b

    def kernel(self, kind, scale):
        """(body id, argument block) of `kind` at `scale` x its workload size."""
        body, _n, rest = _KINDS[kind]
        L = self._lead(kind, scale)
        b = self._get(kind)
        if body == "bn":
            x = b["x"][:L]
            m, v = torch.empty(rest[0], device=self.dev), torch.empty(rest[0], device=self.dev)
            return H.BN_STATS, H.bn_stats_args(x, m, v, H.bn_stats_workspace(x))
        if body == "poly":
            return H.POLY, H.poly_args(b["x"][:L], b["y"][:L], W.poly_coefficients().tolist())
        if body == "hist":
            L16 = max(16, L // 16 * 16)
            return H.HIST256, H.hist256_args(b["x"][:L16], torch.zeros(256, dtype=torch.int32, device=self.dev))
        if body == "philox":
            return H.PHILOX, H.philox_args(b["y"][:L], 0)
        if body == "upsample":
            return H.UPSAMPLE2X, H.upsample2x_args(b["x"][:L], b["y"][:L])
        if body == "maxpool":
            return H.MAXPOOL3S2, H.maxpool3s2_args(b["x"][:L], b["y"][:L])
        return H.IM2COL3, H.im2col3_args(b["x"][:L], b["y"][:L])


def builtin_grid(d0):
    return list(range(32, d0, 32)), list(BUILTIN_CAPS), [1, 2, 3, 4]


def profile_builtin(name, scale, pool, peaks, reps=3, stream=None, keep=False):
    """Exhaustive profile of one built-in pair at one size: a record like
    the template corpus's (points = [split, cap, bps, time, regs, spill,
    status]) with the features (hf_pair_features) and log times of its valid
    points.  The device tensors are released unless `keep` (then the
    record holds the kernels and argument blocks for further launches)."""
    (ka_kind, kb_kind), d0 = BUILTIN_PAIRS[name]
    ba, aa = pool.kernel(ka_kind, scale)
    bb, ab = pool.kernel(kb_kind, scale)
    ka, kb = H.hf_register_kernel(ba), H.hf_register_kernel(bb)
    splits, caps, bps = builtin_grid(d0)
    table = H.hf_profile_pair(ka, kb, [aa, ab], d0, splits, caps, bps, reps=reps, flush_l2=False,
                              stream=stream)
    rec = {"name": name, "scale": scale, "d0": d0, "bodies": [ba, bb],
           "points": [[q["split"], q["regcap"], q["blocks_per_sm"], round(q["time_us"], 3), q["regs"],
                       q["spill_bytes"], q["status"]] for q in table]}
    # target: log of the time over the pair's ideal-overlap time (constant
    # per pair, so the ranking within a pair is that of the time itself)
    rec["log_ideal"] = math.log(ideal_us([ba, bb], [aa, ab], peaks))
    X, Y, qis = [], [], []
    for qi, (split, cap, b_, t, regs, spill, st) in enumerate(rec["points"]):
        if st != 0 or t <= 0:
            continue
        X.append(H.hf_pair_features(ka, kb, [aa, ab], split, d0, cap, b_, regs, spill, peaks))
        Y.append(math.log(t) - rec["log_ideal"])
        qis.append(qi)
    rec["X"], rec["Y"], rec["qi"] = X, Y, qis
    if keep:
        rec["_kernels"], rec["_args"] = (ka, kb), [aa, ab]
    else:
        H.hf_destroy_kernel(ka)
        H.hf_destroy_kernel(kb)
    return rec


def ideal_us(bodies, args, peaks):
    """Ideal-overlap time of kernels run together (us): max(total bytes /
    HBM bandwidth, each pipe's total operations / its rate)."""
    tot = {"bytes": 0.0, "ffma": 0.0, "imul": 0.0, "smem_atomic": 0.0, "ialu": 0.0}
    for b, a in zip(bodies, args):
        w = H.hf_body_work_of(b, a)
        for k in tot:
            tot[k] += w[k]
    rate = {"ffma": peaks.ffma_per_s, "imul": peaks.imul_per_s, "smem_atomic": peaks.smem_atomic_per_s,
            "ialu": peaks.ialu_per_s}
    t = tot["bytes"] / (peaks.hbm_gbs * 1e9)
    for k, r in rate.items():
        if r > 0:
            t = max(t, tot[k] / r)
    return t * 1e6


def featurize_builtin(recs):
    """Rows of (pair index, point index, features, log time) for the valid
    points of built-in pair records."""
    X, Y, owner = [], [], []
    for pi, r in enumerate(recs):
        X += r["X"]
        Y += r["Y"]
        owner += [(pi, qi) for qi in r["qi"]]
    return np.asarray(X, np.float32), np.asarray(Y, np.float32), owner


def device_peaks(hbm_gbs, stream=None):
    """Measured HBM bandwidth plus the calibrated pipe rates of the device."""
    return H.pipe_peaks(hbm_gbs, H.hf_calibrate(H.CAL_FFMA, stream), H.hf_calibrate(H.CAL_IMUL, stream),
                        H.hf_calibrate(H.CAL_SMEM_ATOMIC, stream), H.hf_calibrate(H.CAL_IALU, stream))


def run_builtin(dev, hbm_gbs=6785.9, steps=20000, reps=3, confirm=5, scales=TRAIN_SCALES,
                seeds=ENSEMBLE_SEEDS, names=None, targets=BUILTIN_TARGETS, log=None):
    """Trains an ensemble (one perceptron per seed) on the built-in pairs at
    sizes bracketing their workload sizes, installs it for
    hf_autotune(TUNE_MODEL), then judges it at the held-out workload sizes
    of `targets`: the regret of the model's top-1 and top-`confirm` picks
    read from the exhaustive table of that size, of the library's model mode
    (which times its `confirm` best-scored candidates and the neighbours of
    the fastest of them; its pick's time is read from the same table), of
    Algorithm 2 and of the naive even split."""
    names = list(names or BUILTIN_PAIRS)
    st = torch.cuda.Stream(device=dev)
    peaks = device_peaks(hbm_gbs, st)
    pool = CorpusPool(dev, max(max(scales), 1.0))
    t0 = time.time()
    train_recs = []
    for nm in names:
        for sc in scales:
            train_recs.append(profile_builtin(nm, sc, pool, peaks, reps=reps, stream=st))
        if log:
            log("profiled %s (%.0f s)" % (nm, time.time() - t0))
    t_profile = time.time() - t0
    Xtr, Ytr, _ = featurize_builtin(train_recs)
    t1 = time.time()
    models = [train(Xtr, Ytr, dev, steps=steps, seed=sd_) for sd_ in seeds]
    t_train = time.time() - t1
    mu, sd = models[0][1], models[0][2]   # the same standardisation for every seed
    H.hf_cost_model_set([m[0] for m in models], mu, sd, peaks, confirm)
    out = {"train_pairs": len(names), "train_sizes": [round(x, 4) for x in scales],
           "train_points": int(Xtr.shape[0]), "ensemble": len(models), "confirm": confirm,
           "profile_s": round(t_profile, 1), "train_s": round(t_train, 3),
           "train_loss_first_last": [float(models[0][3][:100].mean()), float(models[0][3][-100:].mean())],
           "pairs": {}}
    for nm in targets:
        rec = profile_builtin(nm, 1.0, pool, peaks, reps=reps, stream=st, keep=True)
        X, Y, own = featurize_builtin([rec])
        pred = np.mean([predict(m[0], X, mu, sd, dev) for m in models], axis=0)
        ok = [q for q in rec["points"] if q[6] == 0 and q[3] > 0]
        table = {(q[0], q[1], q[2]): q[3] for q in ok}
        best = min(ok, key=lambda q: q[3])
        ka, kb = rec["_kernels"]
        d0 = rec["d0"]
        tuned, n_timed = H.hf_autotune_model(ka, kb, rec["_args"], d0, reps=reps, stream=st)
        key = (tuned["split"], tuned["regcap"], tuned["blocks_per_sm"])
        a2, _trace = H.hf_search_alg2(ka, kb, rec["_args"], d0, step=128 if d0 >= 512 else 64, reps=reps,
                                      flush_l2=False, stream=st)
        a2_t = table.get((a2["split"], a2["regcap"], a2["blocks_per_sm"]))
        naive = [q for q in ok if q[0] == d0 // 2 and q[1] == 0]
        naive_t = min(naive, key=lambda q: -q[2])[3] if naive else None
        rel = lambda t: round(t / best[3] - 1.0, 4) if t else None
        out["pairs"][nm] = {
            "points": len(ok), "rmse_log": round(float(np.sqrt(np.mean((pred - Y) ** 2))), 4),
            "exhaustive_best": {"split": best[0], "regcap": best[1], "blocks_per_sm": best[2],
                                "time_us": best[3]},
            "model_regret_top1": round(float(regret([rec], own, pred, 1)[0]), 4),
            "model_regret_top%d" % confirm: round(float(regret([rec], own, pred, confirm)[0]), 4),
            "autotune_model": {"split": key[0], "regcap": key[1], "blocks_per_sm": key[2],
                               "measured_us": round(tuned["time_us"], 3), "table_us": table.get(key),
                               "regret": rel(table.get(key)), "timed_points": n_timed},
            "alg2": {"split": a2["split"], "regcap": a2["regcap"], "blocks_per_sm": a2["blocks_per_sm"],
                     "table_us": a2_t, "regret": rel(a2_t), "timed_points": len(_trace)},
            "naive_even_split_regret": rel(naive_t),
        }
        H.hf_destroy_kernel(ka)
        H.hf_destroy_kernel(kb)
        del rec
    del pool
    torch.cuda.empty_cache()
    return out
