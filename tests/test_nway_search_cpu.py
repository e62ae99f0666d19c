"""The N-way autotuner's search on the host (hf_nway_search_sim): the same
code as hf_autotune_nway after its standalone timings, asked for plan costs
from a Python function instead of timing launches on the GPU.

The first landscape is a makespan: interval i runs its kernels one after
another with w_i warps, each kernel's time its standalone time divided by
the interval's warps, so interval i finishes at L_i / w_i and the plan takes
the latest finish, times a small factor for a register cap.  Its optimum
over integer warps is known closely: sum(L) / 32 at 1024 threads without a
cap (every partition reaches it with warps in proportion to load).  The
second models bodies on bulk-copy rings (below)."""
import pytest

from paper_2007_01277_gb300 import hfuse as H

LOADS = [229.3, 129.1, 120.8, 47.1, 42.9, 43.0, 38.9, 30.7]   # the 8-way workload's kernels alone (us)
CAPS = (0, 40, 48, 64, 96)


def makespan(loads, seen=None):
    def cost(q):
        if seen is not None:
            seen.append(q)
        P = q["n_intervals"]
        w = [t // 32 for t in q["interval_threads"]]
        L = [0.0] * P
        for k, i in enumerate(q["interval_of"]):
            L[i] += loads[k]
        fin = [L[i] / w[i] for i in range(P)]
        return max(fin) * (1.0 if q["regcap"] == 0 else 1.02), fin
    return cost


def _valid(q, n):
    P = q["n_intervals"]
    assert 1 <= P <= H.MAX_INTERVALS
    assert len(q["interval_of"]) == n and all(0 <= i < P for i in q["interval_of"])
    assert set(q["interval_of"]) == set(range(P))          # no empty interval
    assert all(t >= 32 and t % 32 == 0 for t in q["interval_threads"])
    assert sum(q["interval_threads"]) in (512, 768, 1024)
    assert q["regcap"] in CAPS


def test_search_balances_the_makespan():
    best = H.hf_nway_search_sim(LOADS, makespan(LOADS), max_evals=3000)
    _valid(best, len(LOADS))
    bound = sum(LOADS) / 32
    assert best["regcap"] == 0 and sum(best["interval_threads"]) == 1024
    assert bound <= best["time_us"] <= 1.03 * bound, (best, bound)


def test_every_plan_asked_for_is_valid_and_the_budget_holds():
    for budget in (40, 300, 1500):
        seen = []
        best = H.hf_nway_search_sim(LOADS, makespan(LOADS, seen), max_evals=budget)
        for q in seen:
            _valid(q, len(LOADS))
        # the packing seeds (at most 30) and the ten finalists' re-timings
        # are always done; the budget bounds the phases between
        assert best["evals"] <= max(budget, 30) + 10, (budget, best["evals"])
        # the trace phase asks for interval finishing times too
        assert len(seen) >= best["evals"]


def test_search_is_repeatable_and_monotone_in_the_budget():
    a = H.hf_nway_search_sim(LOADS, makespan(LOADS), max_evals=800)
    b = H.hf_nway_search_sim(LOADS, makespan(LOADS), max_evals=800)
    assert a == b
    times = [H.hf_nway_search_sim(LOADS, makespan(LOADS), max_evals=e)["time_us"] for e in (60, 200, 800, 2400)]
    assert all(t1 >= t2 for t1, t2 in zip(times, times[1:])), times


def test_search_rejects_bad_arguments():
    with pytest.raises(H.HFError):
        H.hf_nway_search_sim([], makespan([]))
    with pytest.raises(H.HFError):
        H.hf_nway_search_sim([1.0] * (H.MAX_SCHEDULE + 1), makespan([1.0] * (H.MAX_SCHEDULE + 1)))
    with pytest.raises(H.HFError):
        H.hf_nway_search_sim([5.0, 0.0], makespan([5.0, 0.0]))
    # no plan has a cost
    with pytest.raises(H.HFError):
        H.hf_nway_search_sim([5.0, 3.0], lambda q: (0.0, [0.0] * q["n_intervals"]))


# A landscape closer to fused kernels with bulk-copy rings: kernel k spends
# a fraction f_k of its standalone time issuing instructions (that part
# scales with its interval's warps, full speed at 16 warps) and the rest
# moving bytes, which a ring delivers at full rate with any warps; the bytes
# of all intervals share one memory system, so the plan takes at least the
# sum of the memory parts (M); warps beyond 16 per block cost 1 % each.
FRAC = [1.0, 0.02, 0.06, 0.15, 0.3, 0.0, 0.1, 0.2]


def ring_model(q):
    P = q["n_intervals"]
    w = [t // 32 for t in q["interval_threads"]]
    fin = [0.0] * P
    for k, i in enumerate(q["interval_of"]):
        fin[i] += LOADS[k] * (FRAC[k] * 16.0 / w[i] + (1.0 - FRAC[k]))
    M = sum((1.0 - f) * t for f, t in zip(FRAC, LOADS))
    c = (1.0 + 0.01 * max(0, sum(w) - 16)) * (1.0 if q["regcap"] == 0 else 1.02)
    return max(max(fin), M) * c, fin


def test_issue_weighted_seeds_reach_the_memory_bound():
    """With each kernel's issue time given, the packed seeds give the
    issuing kernel the warps and the streaming kernels one or two: a plan at
    the memory bound comes out of the seeds' phase (the search without them
    needs thousands of evaluations on this landscape)."""
    M = sum((1.0 - f) * t for f, t in zip(FRAC, LOADS))
    issue = [f * t for f, t in zip(FRAC, LOADS)]
    best = H.hf_nway_search_sim(LOADS, ring_model, max_evals=60, issue_us=issue)
    _valid(best, len(LOADS))
    assert best["time_us"] <= 1.001 * M, (best, M)
    assert sum(best["interval_threads"]) == 512 and best["regcap"] == 0
    assert best["evals"] <= max(60, 45) + 10   # up to 45 seeds with issue times
    with pytest.raises(H.HFError):
        H.hf_nway_search_sim(LOADS, ring_model, issue_us=[-1.0] + issue[1:])
