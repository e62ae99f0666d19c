"""The cost model's regret computation against the oracle's definition, on a
stored hand-built table (tests/golden/regret_table.json): regret =
t(model's pick)/t(exhaustive best) - 1, both from the same exhaustive table
(the yardstick of the learned model that replaces Algorithm 2's profiling
loop, Sec. 3.2).  CPU only."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2007_01277_gb300 import costmodel as CM

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "regret_table.json")


def _table():
    d = json.load(open(GOLDEN))
    recs, owner, pred = [], [], []
    for pi, p in enumerate(d["pairs"]):
        recs.append({"id": p["id"], "points": p["points"]})
        for qi, (pt, pl) in enumerate(zip(p["points"], p["pred_log"])):
            if pt[6] == 0 and pt[3] > 0:     # the points featurize() keeps
                owner.append((pi, qi))
                pred.append(pl)
    return d["pairs"], recs, owner, np.asarray(pred, np.float32)


def _oracle_regret(points, preds, confirm):
    """Brute force: candidates = points that ran; pick = fastest measured
    among the `confirm` lowest predictions (ties by point order)."""
    cand = [(pl, qi) for qi, (pt, pl) in enumerate(zip(points, preds)) if pt[6] == 0 and pt[3] > 0]
    best = min(points[qi][3] for _, qi in cand)
    ranked = sorted(cand)
    pick = min(points[qi][3] for _, qi in ranked[:confirm])
    return oracle.regret(pick, best)


@pytest.mark.parametrize("confirm,key", [(1, "regret_top1"), (3, "regret_top3")])
def test_costmodel_regret_matches_oracle_and_hand_values(confirm, key):
    pairs, recs, owner, pred = _table()
    got = CM.regret(recs, owner, pred, confirm)
    want = [_oracle_regret(p["points"], p["pred_log"], confirm) for p in pairs]
    hand = [p[key] for p in pairs]
    assert got.shape == (len(pairs),)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
    np.testing.assert_allclose(got, hand, rtol=0, atol=1e-12)


def test_summary_of_the_hand_table():
    _pairs, recs, owner, pred = _table()
    s = CM.summarize(CM.regret(recs, owner, pred, 1))
    assert s["pairs"] == 3
    assert s["mean"] == pytest.approx((1 / 3 + 7 / 18 + 0.0) / 3, abs=1e-12)
    assert s["max"] == pytest.approx(7 / 18, abs=1e-12)
    assert s["within_5pct"] == pytest.approx(1 / 3, abs=1e-12)
