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
