// tune.cu -- profiling search over fusion configurations (Sec. 3.2).
//
// hf_time_fused / hf_time_single time one configuration with CUDA events on
// the caller's stream: two warm-up launches, then `reps` launches each
// preceded (optionally) by a write of a buffer twice the L2 size, median and
// 10th/90th percentiles.  hf_profile_pair times the whole grid of (split,
// register cap, blocks/SM) points -- the exhaustive search and the training
// data of the cost model.  hf_search_alg2 is Algorithm 2: d1 = step, 2 step,
// ... < d0, each profiled without a bound and with the bound r0 of the
// register-bound formula (snapped down to the nearest compiled cap), keeping
// the first strictly faster configuration.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <mutex>
#include <vector>

#include "kernels.cuh"

extern "C" {
hf_status hf_query_single(hf_kernel k, const void *args, int threads, hf_fused_info *info);
}

namespace hf {
int kernel_body_id(const hf_kernel_t *k);   // runtime.cu
}

// LPT plan of the N-way autotuner: kernels -> intervals, warps per interval.
struct NwayPlanC {
    int P;
    int io[HF_MAX_SCHEDULE];
    int warps[HF_MAX_INTERVALS];
    int cap;
};

namespace {

struct FlushBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};
std::mutex g_flush_mu;
FlushBuf g_flush;

hf_status flush_l2(cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_flush_mu);
    if (!g_flush.ptr) {
        int dev = 0, l2 = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return HF_ERR_CUDA;
        if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) return HF_ERR_CUDA;
        g_flush.bytes = 2 * (size_t)std::max(l2, 1 << 20);
        if (cudaMalloc(&g_flush.ptr, g_flush.bytes) != cudaSuccess) {
            g_flush.ptr = nullptr;
            return HF_ERR_CUDA;
        }
    }
    return cudaMemsetAsync(g_flush.ptr, 0, g_flush.bytes, s) == cudaSuccess ? HF_OK : HF_ERR_CUDA;
}

template <class F>
hf_status time_it(F launch, int reps, int flush, cudaStream_t s, float *med, float *p10, float *p90)
{
    if (reps < 1) return HF_ERR_INVALID;
    for (int w = 0; w < 2; ++w) {
        hf_status st = launch();
        if (st) return st;
    }
    std::vector<cudaEvent_t> ev(2 * reps);
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return HF_ERR_CUDA;
    hf_status st = HF_OK;
    for (int r = 0; r < reps && !st; ++r) {
        if (flush) st = flush_l2(s);
        if (st) break;
        cudaEventRecord(ev[2 * r], s);
        st = launch();
        cudaEventRecord(ev[2 * r + 1], s);
    }
    std::vector<float> t;
    if (!st && cudaStreamSynchronize(s) != cudaSuccess) st = HF_ERR_CUDA;
    if (!st)
        for (int r = 0; r < reps; ++r) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[2 * r], ev[2 * r + 1]);
            t.push_back(ms * 1000.f);
        }
    for (auto &e : ev) cudaEventDestroy(e);
    if (st) return st;
    std::sort(t.begin(), t.end());
    auto q = [&](double f) { return t[std::min((size_t)(f * (t.size() - 1) + 0.5), t.size() - 1)]; };
    if (med) *med = q(0.5);
    if (p10) *p10 = q(0.1);
    if (p90) *p90 = q(0.9);
    return HF_OK;
}

int snap_cap(int r0)
{
    int caps[32];
    const int n = hf_regcaps(caps, 32);
    int best = 0;
    for (int i = 0; i < n && i < 32; ++i)
        if (caps[i] <= r0) best = caps[i];
    return best;
}

} // namespace

extern "C" {

hf_status hf_time_fused(hf_fused f, const void *const *args, int grid, int reps, int flush_l2_,
                        void *stream, float *median_us, float *p10_us, float *p90_us)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return time_it([&] { return hf_launch(f, args, grid, stream); }, reps, flush_l2_, s, median_us,
                   p10_us, p90_us);
}

hf_status hf_time_single(hf_kernel k, const void *args, int threads, int grid, int reps,
                         int flush_l2_, void *stream, float *median_us, float *p10_us, float *p90_us)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return time_it([&] { return hf_launch_single(k, args, threads, grid, stream); }, reps, flush_l2_,
                   s, median_us, p10_us, p90_us);
}

hf_status hf_profile_pair(hf_kernel a, hf_kernel b, const void *const *args, int d0, const int *splits,
                          int n_splits, const int *regcaps, int n_regcaps, const int *bps, int n_bps,
                          int reps, int flush_l2_, void *stream, hf_tune_point *table)
{
    if (!a || !b || !args || !splits || !regcaps || !bps || !table || n_splits < 1 || n_regcaps < 1 ||
        n_bps < 1)
        return HF_ERR_INVALID;
    hf_device_limits lim;
    hf_status st = hf_device_info(&lim);
    if (st) return st;
    int idx = 0;
    for (int i = 0; i < n_splits; ++i)
        for (int j = 0; j < n_regcaps; ++j) {
            hf_fused f = nullptr;
            hf_status fs = hf_fuse(a, b, splits[i], d0, regcaps[j], &f);
            hf_fused_info info;
            std::memset(&info, 0, sizeof info);
            if (!fs) fs = hf_query(f, args, &info);
            for (int k = 0; k < n_bps; ++k, ++idx) {
                hf_tune_point &p = table[idx];
                std::memset(&p, 0, sizeof p);
                p.split = splits[i];
                p.regcap = regcaps[j];
                p.blocks_per_sm = bps[k];
                p.regs = info.regs;
                p.spill_bytes = info.spill_bytes;
                p.status = fs;
                p.time_us = -1.f;
                if (fs) continue;
                if (bps[k] < 1 || bps[k] > info.blocks_per_sm) {
                    p.status = HF_ERR_REGS;   // not resident at this many blocks per SM
                    continue;
                }
                p.grid = bps[k] * lim.sm_count;
                p.status = hf_time_fused(f, args, p.grid, reps, flush_l2_, stream, &p.time_us,
                                         &p.p10_us, &p.p90_us);
                if (p.status == HF_ERR_CUDA) {
                    hf_destroy_fused(f);
                    return HF_ERR_CUDA;
                }
            }
            if (f) hf_destroy_fused(f);
        }
    return HF_OK;
}

hf_status hf_search_alg2(hf_kernel a, hf_kernel b, const void *const *args, int d0, int step,
                         int reps, int flush_l2_, void *stream, hf_tune_point *best,
                         hf_tune_point *trace, int trace_cap, int *n_trace)
{
    if (!a || !b || !args || !best || step < 32 || step % 32) return HF_ERR_INVALID;
    hf_device_limits lim;
    hf_status st = hf_device_info(&lim);
    if (st) return st;
    std::memset(best, 0, sizeof *best);
    best->time_us = -1.f;
    int nt = 0;
    auto record = [&](const hf_tune_point &p) {
        if (trace && nt < trace_cap) trace[nt] = p;
        ++nt;
    };
    for (int d1 = step; d1 < d0; d1 += step) {
        const int d2 = d0 - d1;
        // NRegs(S1), NRegs(S2): the kernels compiled alone
        hf_fused_info ia, ib;
        if (hf_query_single(a, args[0], d1, &ia) || hf_query_single(b, args[1], d2, &ib)) continue;
        for (int pass = 0; pass < 2; ++pass) {
            hf_fused f = nullptr;
            int cap = 0;
            hf_fused_info info;
            if (pass == 1) {
                // ShMem(F) of the unbounded instance, then the bound r0
                hf_fused f0 = nullptr;
                if (hf_fuse(a, b, d1, d0, 0, &f0)) continue;
                hf_status qs = hf_query(f0, args, &info);
                hf_destroy_fused(f0);
                if (qs) continue;
                int r0 = 0;
                hf_register_bound(&lim, d1, ia.regs, d2, ib.regs, info.smem_bytes, &r0);
                cap = snap_cap(r0);
                if (cap == 0) continue;   // no compiled cap at or below r0
            }
            if (hf_fuse(a, b, d1, d0, cap, &f)) continue;
            hf_tune_point p;
            std::memset(&p, 0, sizeof p);
            p.split = d1;
            p.regcap = cap;
            p.status = hf_query(f, args, &info);
            if (!p.status) {
                p.regs = info.regs;
                p.spill_bytes = info.spill_bytes;
                p.blocks_per_sm = info.blocks_per_sm;
                p.grid = info.blocks_per_sm * lim.sm_count;
                p.status = hf_time_fused(f, args, p.grid, reps, flush_l2_, stream, &p.time_us,
                                         &p.p10_us, &p.p90_us);
            }
            hf_destroy_fused(f);
            if (p.status == HF_ERR_CUDA) return HF_ERR_CUDA;
            record(p);
            if (!p.status && (best->time_us < 0.f || p.time_us < best->time_us)) *best = p;
        }
    }
    if (n_trace) *n_trace = nt;
    return best->time_us < 0.f ? HF_ERR_INVALID : HF_OK;
}


} // extern "C"

namespace {

// The measurements the N-way search asks for.  The same search runs on the
// GPU (hf_autotune_nway: each plan built, queried and timed) and against a
// cost function the caller gives (hf_nway_search_sim: the search itself
// tested on the host).
struct NwayMeasure {
    // time plan p: HF_OK with *us > 0 and the grid used, another status when
    // the plan cannot be built or is not resident (skipped); HF_ERR_CUDA ends
    // the search
    std::function<hf_status(const NwayPlanC &, float *, int *)> time;
    // each interval's finishing time of plan p launched on `grid` blocks,
    // relative to the earliest start (any unit)
    std::function<hf_status(const NwayPlanC &, int, double *)> finish;
    // time plan p again with three times the repetitions
    std::function<hf_status(const NwayPlanC &, int, float *)> retime;
};

// The search of hf_autotune_nway over plans for n kernels whose standalone
// times (phase 1, measured by the caller) are t[0..n): phases 2-6 below.
// issue (may be NULL) estimates each kernel's busiest-pipe time; it adds
// seeds whose warps follow issue time instead of standalone time.
hf_status nway_search(int n, const float *t, const float *issue, int max_evals, const NwayMeasure &m,
                      hf_nway_plan *best)
{
    hf_status st = HF_OK;
    int evals = 0;
    float best_t = -1.f;
    NwayPlanC bp;
    std::memset(&bp, 0, sizeof bp);
    auto eval = [&](const NwayPlanC &p, float *us, int *grid) -> hf_status {
        ++evals;
        return m.time(p, us, grid);
    };
    struct Seed {
        float t;
        int grid;
        NwayPlanC p;
    };
    std::vector<Seed> seeds, seen;
    float last_t = -1.f;
    int last_grid = 0;
    auto consider = [&](const NwayPlanC &p) -> hf_status {
        float us = 0.f;
        int grid = 0;
        last_t = -1.f;
        hf_status s2 = eval(p, &us, &grid);
        if (s2 == HF_ERR_CUDA) return s2;
        if (s2) return HF_OK;   // not buildable / not resident: skip
        last_t = us;
        last_grid = grid;
        seen.push_back(Seed{us, grid, p});
        if (best_t < 0.f || us < best_t) {
            best_t = us;
            bp = p;
            best->grid = grid;
        }
        return HF_OK;
    };
    // 2. LPT packings over block sizes, caps and interval counts
    std::vector<int> order(n);
    for (int k = 0; k < n; ++k) order[k] = k;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return t[a] > t[b]; });
    const int d0s[] = {512, 768, 1024};
    const int caps[] = {0, 40, 48, 64, 96};
    double issue_tot = 0.0;
    for (int k = 0; issue && k < n; ++k) issue_tot += std::max(0.f, issue[k]);
    for (int d0 : d0s)
        for (int cap : caps)
            for (int P : {n, (n + 1) / 2})
                for (int by_issue = 0; by_issue < (issue_tot > 0.0 && P < n ? 2 : 1); ++by_issue) {
                    const int W = d0 / 32;
                    if (P > HF_MAX_INTERVALS || P > W || P < 1) continue;
                    NwayPlanC p;
                    std::memset(&p, 0, sizeof p);
                    p.P = P;
                    p.cap = cap;
                    // kernels packed by standalone time; warps by standalone
                    // or by issue time of each interval's kernels
                    std::vector<double> load(P, 0.0), wt(P, 0.0);
                    for (int k : order) {
                        int i = (int)(std::min_element(load.begin(), load.end()) - load.begin());
                        p.io[k] = i;
                        load[i] += t[k];
                        wt[i] += by_issue ? std::max(0.f, issue[k]) : t[k];
                    }
                    double tot = 0.0;
                    for (double l : wt) tot += l;
                    int used = 0;
                    for (int i = 0; i < P; ++i) {
                        p.warps[i] = 1 + (int)((W - P) * wt[i] / tot);
                        used += p.warps[i];
                    }
                    while (used < W) {   // leftover warps to the most loaded per warp
                        int bi = 0;
                        for (int i = 1; i < P; ++i)
                            if (wt[i] / p.warps[i] > wt[bi] / p.warps[bi]) bi = i;
                        ++p.warps[bi];
                        ++used;
                    }
                    st = consider(p);
                    if (st) return st;
                    if (last_t > 0.f) seeds.push_back(Seed{last_t, last_grid, p});
                }
    if (best_t < 0.f) return HF_ERR_INVALID;
    std::sort(seeds.begin(), seeds.end(), [](const Seed &a, const Seed &b) { return a.t < b.t; });
    if (seeds.size() > 12) seeds.resize(12);
    // 3. rebalance from measured interval finishing times: interval i gets
    //    warps in proportion to warps_i * finish_i, so that intervals that
    //    end early give warps to the ones that end late
    for (const Seed &sd : seeds) {
    NwayPlanC cur = sd.p;
    int cur_grid = sd.grid;
    float cur_t = sd.t;
    for (int round = 0; round < 6 && evals < max_evals; ++round) {
        const NwayPlanC base = cur;
        double fin[HF_MAX_INTERVALS];
        const hf_status s2 = m.finish(base, cur_grid, fin);
        if (s2 == HF_ERR_CUDA) return s2;
        if (s2) break;
        const int W = [&] { int w = 0; for (int i = 0; i < base.P; ++i) w += base.warps[i]; return w; }();
        double want[HF_MAX_INTERVALS], tot = 0.0;
        for (int i = 0; i < base.P; ++i) {
            want[i] = base.warps[i] * fin[i];
            tot += want[i];
        }
        if (tot <= 0.0) break;
        NwayPlanC p = base;
        int used = 0;
        for (int i = 0; i < base.P; ++i) {
            p.warps[i] = std::max(1, (int)(want[i] / tot * W));
            used += p.warps[i];
        }
        while (used < W) {   // hand out the remainder to the latest finishers
            int bi = 0;
            for (int i = 1; i < p.P; ++i)
                if (want[i] / p.warps[i] > want[bi] / p.warps[bi]) bi = i;
            ++p.warps[bi];
            ++used;
        }
        while (used > W) {
            int bi = -1;
            for (int i = 0; i < p.P; ++i)
                if (p.warps[i] > 1 && (bi < 0 || want[i] / p.warps[i] < want[bi] / p.warps[bi])) bi = i;
            if (bi < 0) break;
            --p.warps[bi];
            --used;
        }
        if (std::equal(p.warps, p.warps + p.P, base.warps)) break;
        st = consider(p);
        if (st) return st;
        if (!(last_t > 0.f && last_t < cur_t)) break;   // this seed stopped improving
        cur = p;
        cur_t = last_t;
        cur_grid = last_grid;
    }
    }
    // 4. local search from the fastest plan: move one warp between two
    //    intervals, move one kernel to another interval, or swap two kernels
    //    of different intervals; take the best neighbour while it helps
    auto used_all = [&](const NwayPlanC &p) {
        int cnt[HF_MAX_INTERVALS] = {0};
        for (int k = 0; k < n; ++k) ++cnt[p.io[k]];
        for (int i = 0; i < p.P; ++i)
            if (!cnt[i]) return false;
        return true;
    };
    // local search from each of the five fastest distinct plans seen so far
    std::sort(seen.begin(), seen.end(), [](const Seed &a, const Seed &b) { return a.t < b.t; });
    std::vector<NwayPlanC> starts;
    auto same = [&](const NwayPlanC &a, const NwayPlanC &b) {
        if (a.P != b.P || a.cap != b.cap) return false;
        for (int k = 0; k < n; ++k)
            if (a.io[k] != b.io[k]) return false;
        for (int i = 0; i < a.P; ++i)
            if (a.warps[i] != b.warps[i]) return false;
        return true;
    };
    for (const Seed &sd : seen) {
        bool dup = false;
        for (const NwayPlanC &q : starts) dup = dup || same(q, sd.p);
        if (!dup) starts.push_back(sd.p);
        if (starts.size() == 5) break;
    }
    // the neighbours of a plan: one or two warps moved between two
    // intervals, one kernel moved to another interval, two kernels of
    // different intervals swapped, or the same plan under another register
    // cap
    auto neighbours = [&](const NwayPlanC &base) {
        std::vector<NwayPlanC> nb;
        for (int w = 1; w <= 2; ++w)
            for (int i = 0; i < base.P; ++i)
                for (int j = 0; j < base.P; ++j) {
                    if (i == j || base.warps[i] <= w) continue;
                    NwayPlanC p = base;
                    p.warps[i] -= w;
                    p.warps[j] += w;
                    nb.push_back(p);
                }
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < base.P; ++j) {
                if (j == base.io[k]) continue;
                NwayPlanC p = base;
                p.io[k] = j;
                if (used_all(p)) nb.push_back(p);
            }
        for (int k = 0; k < n; ++k)
            for (int l = k + 1; l < n; ++l) {
                if (base.io[k] == base.io[l]) continue;
                NwayPlanC p = base;
                std::swap(p.io[k], p.io[l]);
                nb.push_back(p);
            }
        for (int cap : caps) {
            if (cap == base.cap) continue;
            NwayPlanC p = base;
            p.cap = cap;
            nb.push_back(p);
        }
        return nb;
    };
    // Random numbers of the restarts below: SplitMix64 from a fixed seed, so
    // the search depends only on the measured times.
    unsigned long long rs = 0x2007012770000001ull;
    auto rnd = [&](size_t m) {
        rs += 0x9E3779B97F4A7C15ull;
        unsigned long long z = rs;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return (size_t)((z ^ (z >> 31)) % m);
    };
    // Local search from `start` (measured at start_t, < 0 if not yet).
    // Steepest descent: take the best neighbour while it is faster by more
    // than 0.5 %.  First improvement (the restarts): visit the neighbours in
    // random order and move to the first one faster by more than 0.5 %, so
    // that a restart costs a few dozen evaluations rather than a few hundred.
    auto local_search = [&](const NwayPlanC &start, float start_t, bool first) -> hf_status {
        NwayPlanC cur = start;
        float cur_t = start_t;
        bool improved = true;
        while (improved && evals < max_evals) {
            improved = false;
            float step_t = cur_t;
            NwayPlanC step_p = cur;
            std::vector<NwayPlanC> nb = neighbours(cur);
            if (first)
                for (size_t i = nb.size(); i > 1; --i) std::swap(nb[i - 1], nb[rnd(i)]);
            for (const NwayPlanC &p : nb) {
                if (evals >= max_evals) break;
                const hf_status s2 = consider(p);
                if (s2) return s2;
                if (last_t > 0.f && (step_t < 0.f || last_t < step_t)) {
                    step_t = last_t;
                    step_p = p;
                    if (first && cur_t > 0.f && step_t < cur_t * 0.995f) break;
                }
            }
            if (step_t > 0.f && (cur_t < 0.f || step_t < cur_t * 0.995f)) {
                cur = step_p;
                cur_t = step_t;
                improved = true;
            }
        }
        return HF_OK;
    };
    for (const NwayPlanC &start : starts) {
        float t0 = -1.f;
        for (const Seed &sd : seen)
            if (same(sd.p, start)) {
                t0 = sd.t;
                break;
            }
        st = local_search(start, t0, false);
        if (st) return st;
    }
    // 5. iterated local search with what is left of the budget.  Restarts
    //    cycle over three kinds of starting plan: one of the three fastest
    //    plans so far; the fastest plan of one block size and register cap
    //    (the families in turn, fastest first), so that a family that
    //    started behind is still refined; and one of the packing seeds of
    //    phase 2.  Every other elite or family start has three or four warps
    //    moved between two intervals, elite and family starts then take two
    //    or three random moves (one after a warp shift), and each restart
    //    ends in a first-improvement local search.
    auto by_time = [&] {
        std::vector<Seed> v = seen;
        std::sort(v.begin(), v.end(), [](const Seed &a, const Seed &b) { return a.t < b.t; });
        return v;
    };
    // the three fastest distinct plans measured so far
    auto elites = [&] {
        std::vector<NwayPlanC> e;
        for (const Seed &sd : by_time()) {
            bool dup = false;
            for (const NwayPlanC &q : e) dup = dup || same(q, sd.p);
            if (!dup) e.push_back(sd.p);
            if (e.size() == 3) break;
        }
        return e;
    };
    // the fastest plan of each (warps per block, register cap), fastest first
    auto family_bests = [&] {
        std::vector<NwayPlanC> fb;
        for (const Seed &sd : by_time()) {
            int w = 0;
            for (int i = 0; i < sd.p.P; ++i) w += sd.p.warps[i];
            bool dup = false;
            for (const NwayPlanC &q : fb) {
                int wq = 0;
                for (int i = 0; i < q.P; ++i) wq += q.warps[i];
                dup = dup || (wq == w && q.cap == sd.p.cap);
            }
            if (!dup) fb.push_back(sd.p);
        }
        return fb;
    };
    for (int restart = 0; restart < 512 && evals + 8 < max_evals; ++restart) {
        const int kind = restart % 3, turn = restart / 3;
        NwayPlanC p = bp;
        bool shift = turn % 2 == 1;
        if (kind == 2 && !seeds.empty()) {
            p = seeds[rnd(seeds.size())].p;
            shift = true;
        } else if (kind == 1) {
            const std::vector<NwayPlanC> fb = family_bests();
            if (!fb.empty()) p = fb[(size_t)turn % fb.size()];
        } else {
            const std::vector<NwayPlanC> el = elites();
            if (!el.empty()) p = el[(size_t)turn % el.size()];
        }
        if (shift && p.P > 1) {
            const int w = 3 + (int)rnd(2), i = (int)rnd(p.P), j = (i + 1 + (int)rnd(p.P - 1)) % p.P;
            if (p.warps[i] > w) {
                p.warps[i] -= w;
                p.warps[j] += w;
            }
        }
        const int moves = kind == 2 ? 0 : 2 + (int)rnd(2) - (shift ? 1 : 0);
        for (int m = 0; m < moves; ++m) {
            const std::vector<NwayPlanC> nb = neighbours(p);
            if (nb.empty()) break;
            p = nb[rnd(nb.size())];
        }
        st = consider(p);
        if (st) return st;
        if (last_t <= 0.f) continue;
        st = local_search(p, last_t, true);
        if (st) return st;
    }
    // 6. the ten fastest distinct plans again with three times the
    //    repetitions: a single noisy timing should not pick the winner
    std::sort(seen.begin(), seen.end(), [](const Seed &a, const Seed &b) { return a.t < b.t; });
    std::vector<Seed> finalists;
    for (const Seed &sd : seen) {
        bool dup = false;
        for (const Seed &q : finalists) dup = dup || same(q.p, sd.p);
        if (!dup) finalists.push_back(sd);
        if (finalists.size() == 10) break;
    }
    if (finalists.size() > 1) {
        float best_conf = -1.f;
        for (const Seed &sd : finalists) {
            float us = 0.f;
            const hf_status s2 = m.retime(sd.p, sd.grid, &us);
            ++evals;
            if (s2 == HF_ERR_CUDA) return s2;
            if (s2) continue;
            if (best_conf < 0.f || us < best_conf) {
                best_conf = us;
                bp = sd.p;
                best->grid = sd.grid;
                best_t = us;
            }
        }
    }
    const int grid = best->grid;
    std::memset(best, 0, sizeof *best);
    best->n_intervals = bp.P;
    for (int k = 0; k < n; ++k) best->interval_of[k] = bp.io[k];
    for (int i = 0; i < bp.P; ++i) best->interval_threads[i] = 32 * bp.warps[i];
    best->regcap = bp.cap;
    best->grid = grid;
    best->time_us = best_t;
    best->evals = evals;
    return HF_OK;
}

} // namespace

extern "C" {

hf_status hf_autotune_nway(const hf_kernel *ks, int n, const void *const *args, int max_evals,
                           int reps, int flush_l2_, void *stream, hf_nway_plan *best,
                           float *standalone_us)
{
    if (!ks || !args || !best || n < 1 || n > HF_MAX_SCHEDULE || reps < 1) return HF_ERR_INVALID;
    hf_device_limits lim;
    hf_status st = hf_device_info(&lim);
    if (st) return st;
    // each kernel alone (256 threads, resident grid): its load
    std::vector<float> t(n);
    for (int k = 0; k < n; ++k) {
        st = hf_time_single(ks[k], args[k], 256, 0, reps, flush_l2_, stream, &t[k], nullptr, nullptr);
        if (st) return st;
        if (standalone_us) standalone_us[k] = t[k];
    }
    unsigned long long *d_trace = nullptr;
    if (cudaMalloc(&d_trace, 2 * HF_MAX_INTERVALS * sizeof(unsigned long long)) != cudaSuccess)
        return HF_ERR_CUDA;
    auto build = [&](const NwayPlanC &p, hf_fused *f) {
        int thr[HF_MAX_INTERVALS];
        for (int i = 0; i < p.P; ++i) thr[i] = 32 * p.warps[i];
        return hf_fuse_n(ks, n, p.io, thr, p.P, p.cap, f);
    };
    NwayMeasure m;
    m.time = [&](const NwayPlanC &p, float *us, int *grid) -> hf_status {
        hf_fused f = nullptr;
        hf_status s2 = build(p, &f);
        if (s2) return s2;
        hf_fused_info info;
        s2 = hf_query(f, args, &info);
        if (!s2) {
            *grid = info.blocks_per_sm * lim.sm_count;
            s2 = hf_time_fused(f, args, *grid, reps, flush_l2_, stream, us, nullptr, nullptr);
        }
        hf_destroy_fused(f);
        return s2;
    };
    m.finish = [&](const NwayPlanC &p, int grid, double *fin) -> hf_status {
        hf_fused f = nullptr;
        if (build(p, &f)) return HF_ERR_INVALID;
        unsigned long long h[2 * HF_MAX_INTERVALS];
        for (int i = 0; i < p.P; ++i) h[2 * i] = ~0ull, h[2 * i + 1] = 0ull;
        cudaStream_t cs = static_cast<cudaStream_t>(stream);
        const bool ok = cudaMemcpyAsync(d_trace, h, sizeof h, cudaMemcpyHostToDevice, cs) == cudaSuccess &&
                        hf_launch_traced(f, args, grid, stream, d_trace) == HF_OK &&
                        cudaMemcpyAsync(h, d_trace, sizeof h, cudaMemcpyDeviceToHost, cs) == cudaSuccess &&
                        cudaStreamSynchronize(cs) == cudaSuccess;
        hf_destroy_fused(f);
        if (!ok) return HF_ERR_CUDA;
        unsigned long long t0 = ~0ull;
        for (int i = 0; i < p.P; ++i) t0 = std::min(t0, h[2 * i]);
        for (int i = 0; i < p.P; ++i) fin[i] = (double)(h[2 * i + 1] - t0);
        return HF_OK;
    };
    m.retime = [&](const NwayPlanC &p, int grid, float *us) -> hf_status {
        hf_fused f = nullptr;
        if (build(p, &f)) return HF_ERR_INVALID;
        const hf_status s2 = hf_time_fused(f, args, grid, 3 * reps, flush_l2_, stream, us, nullptr, nullptr);
        hf_destroy_fused(f);
        return s2;
    };
    // each kernel's busiest-pipe time from its algorithmic work, at the pipe
    // rates measured on GB300 (FFMA 3.80e13/s, 32-bit multiply 1.75e13/s,
    // add/XOR/rotate 2.99e13/s, shared atomics 9.66e12/s); only the ratios
    // matter: they shape the issue-weighted seeds
    std::vector<float> issue(n, 0.f);
    for (int k = 0; k < n; ++k) {
        hf_body_work w;
        if (hf_body_work_of(hf::kernel_body_id(ks[k]), args[k], &w)) continue;
        const double us = 1e6 * std::max(std::max(w.ffma / 3.80e13, w.imul / 1.75e13),
                                          std::max(w.ialu / 2.99e13, w.smem_atomic / 9.66e12));
        issue[k] = (float)us;
    }
    st = nway_search(n, t.data(), issue.data(), max_evals, m, best);
    cudaFree(d_trace);
    return st;
}

hf_status hf_nway_search_sim(int n, const float *standalone_us, const float *issue_us, hf_plan_cost_fn cost,
                             void *user, int max_evals, hf_nway_plan *best)
{
    if (!standalone_us || !cost || !best || n < 1 || n > HF_MAX_SCHEDULE) return HF_ERR_INVALID;
    for (int k = 0; k < n; ++k)
        if (!(standalone_us[k] > 0.f) || (issue_us && !(issue_us[k] >= 0.f))) return HF_ERR_INVALID;
    auto ask = [&](const NwayPlanC &p, float *fin) -> float {
        hf_nway_plan q;
        std::memset(&q, 0, sizeof q);
        q.n_intervals = p.P;
        for (int k = 0; k < n; ++k) q.interval_of[k] = p.io[k];
        for (int i = 0; i < p.P; ++i) q.interval_threads[i] = 32 * p.warps[i];
        q.regcap = p.cap;
        return cost(&q, fin, user);
    };
    NwayMeasure m;
    m.time = [&](const NwayPlanC &p, float *us, int *grid) -> hf_status {
        float fin[HF_MAX_INTERVALS] = {0.f};
        const float v = ask(p, fin);
        if (!(v > 0.f)) return HF_ERR_INVALID;
        *us = v;
        *grid = 0;
        return HF_OK;
    };
    m.finish = [&](const NwayPlanC &p, int, double *fin) -> hf_status {
        float f[HF_MAX_INTERVALS] = {0.f};
        if (!(ask(p, f) > 0.f)) return HF_ERR_INVALID;
        for (int i = 0; i < p.P; ++i) fin[i] = f[i];
        return HF_OK;
    };
    m.retime = [&](const NwayPlanC &p, int, float *us) -> hf_status {
        int grid = 0;
        return m.time(p, us, &grid);
    };
    return nway_search(n, standalone_us, issue_us, max_evals, m, best);
}

} // extern "C"

// ------------------------------------------------------------------ cost model
// The learned replacement of Algorithm 2's profiling loop: every candidate
// (split, register cap, blocks/SM) is built and queried on the host, scored
// by the perceptron in one launch, and only the best-scored few are timed.
namespace {
struct CostModel {
    std::vector<float> params;   // n_models parameter sets, back to back
    int n_models = 0;
    float mu = 0.f, sd = 1.f;
    hf_pipe_peaks peaks{};
    int confirm = 1;
};
std::mutex g_cm_mu;
CostModel g_cm;
bool g_cm_set = false;

hf_status autotune_model_impl(hf_kernel a, hf_kernel b, const void *const *args, int d0, int reps,
                              int flush_l2_, void *stream, hf_tune_point *best, int *n_timed)
{
    CostModel cm;
    {
        std::lock_guard<std::mutex> lk(g_cm_mu);
        if (!g_cm_set) return HF_ERR_INVALID;
        cm = g_cm;
    }
    if (d0 < 64 || d0 > 1024 || d0 % 32) return HF_ERR_INVALID;
    hf_device_limits lim;
    hf_status st = hf_device_info(&lim);
    if (st) return st;
    std::vector<int> caps = {0};
    const int nc = hf_regcaps(nullptr, 0);
    std::vector<int> compiled(nc > 0 ? nc : 0);
    if (nc > 0) hf_regcaps(compiled.data(), nc);
    caps.insert(caps.end(), compiled.begin(), compiled.end());
    std::vector<hf_tune_point> cand;
    std::vector<float> X;
    for (int split = 32; split < d0; split += 32)
        for (int cap : caps) {
            hf_fused f = nullptr;
            if (hf_fuse(a, b, split, d0, cap, &f)) continue;   // outside a kernel's range, ...
            hf_fused_info info;
            const hf_status qs = hf_query(f, args, &info);
            hf_destroy_fused(f);
            if (qs) continue;
            for (int bps = 1; bps <= std::min(4, info.blocks_per_sm); ++bps) {
                float feat[HF_MLP_FEATURES];
                if (hf_pair_features(a, b, args, split, d0, cap, bps, info.regs, info.spill_bytes,
                                     &cm.peaks, feat))
                    continue;
                hf_tune_point p;
                std::memset(&p, 0, sizeof p);
                p.split = split;
                p.regcap = cap;
                p.blocks_per_sm = bps;
                p.grid = bps * lim.sm_count;
                p.regs = info.regs;
                p.spill_bytes = info.spill_bytes;
                cand.push_back(p);
                X.insert(X.end(), feat, feat + HF_MLP_FEATURES);
            }
        }
    const int n = (int)cand.size();
    if (n == 0) return HF_ERR_INVALID;
    // one inference launch over every candidate
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float *dX = nullptr, *dy = nullptr, *dP = nullptr;
    const int m = cm.n_models;
    std::vector<float> ym((size_t)m * n), y(n, 0.f);
    bool ok = cudaMalloc(&dX, X.size() * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&dy, (size_t)m * n * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&dP, cm.params.size() * sizeof(float)) == cudaSuccess &&
              cudaMemcpyAsync(dX, X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice, s) ==
                  cudaSuccess &&
              cudaMemcpyAsync(dP, cm.params.data(), cm.params.size() * sizeof(float),
                              cudaMemcpyHostToDevice, s) == cudaSuccess;
    for (int k = 0; ok && k < m && st == HF_OK; ++k)
        st = hf_mlp_forward(dP + (size_t)k * HF_MLP_NPARAMS, dX, n, dy + (size_t)k * n, stream);
    ok = ok && st == HF_OK &&
         cudaMemcpyAsync(ym.data(), dy, ym.size() * sizeof(float), cudaMemcpyDeviceToHost, s) ==
             cudaSuccess &&
         cudaStreamSynchronize(s) == cudaSuccess;
    cudaFree(dX);
    cudaFree(dy);
    cudaFree(dP);
    if (!ok) return st ? st : HF_ERR_CUDA;
    for (int k = 0; k < m; ++k)   // the ensemble's mean prediction
        for (int i = 0; i < n; ++i) y[i] += ym[(size_t)k * n + i] / (float)m;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int i, int j) { return y[i] < y[j]; });
    // time the model's best few, then the untimed neighbours of the fastest
    // of them (other blocks/SM or register cap at its split, the splits one
    // warp either side at its cap and blocks/SM); the fastest measured wins
    best->time_us = -1.f;
    std::vector<char> timed(n, 0);
    int count = 0;
    auto time_one = [&](int i) -> hf_status {
        if (timed[i]) return HF_OK;
        timed[i] = 1;
        hf_tune_point p = cand[i];
        hf_fused f = nullptr;
        if (hf_fuse(a, b, p.split, d0, p.regcap, &f)) return HF_OK;
        p.status = hf_time_fused(f, args, p.grid, reps, flush_l2_, stream, &p.time_us, &p.p10_us,
                                 &p.p90_us);
        hf_destroy_fused(f);
        ++count;
        if (p.status == HF_ERR_CUDA) return HF_ERR_CUDA;
        if (!p.status && (best->time_us < 0.f || p.time_us < best->time_us)) *best = p;
        return HF_OK;
    };
    // the best-scored candidate at each blocks/SM (the coordinate the model
    // ranks least reliably), then the `confirm` best-scored candidates with
    // distinct (split, blocks/SM): candidates that differ only in the
    // register cap score alike and are covered by the neighbour step
    for (int b = 1; b <= 4; ++b)
        for (int r = 0; r < n; ++r)
            if (cand[order[r]].blocks_per_sm == b) {
                if (time_one(order[r]) == HF_ERR_CUDA) return HF_ERR_CUDA;
                break;
            }
    int confirmed = 0;
    for (int r = 0; r < n && confirmed < cm.confirm; ++r) {
        const hf_tune_point &q = cand[order[r]];
        bool seen = false;
        for (int i = 0; i < n && !seen; ++i)
            seen = timed[i] && cand[i].split == q.split && cand[i].blocks_per_sm == q.blocks_per_sm;
        if (seen) continue;
        if (time_one(order[r]) == HF_ERR_CUDA) return HF_ERR_CUDA;
        ++confirmed;
    }
    // neighbour steps from the fastest so far, while they find a faster one
    for (int round = 0; round < 3 && best->time_us >= 0.f; ++round) {
        const hf_tune_point c = *best;
        for (int i = 0; i < n; ++i) {
            const hf_tune_point &q = cand[i];
            const bool same_split = q.split == c.split;
            const bool nb = (same_split && q.regcap == c.regcap && q.blocks_per_sm != c.blocks_per_sm) ||
                            (same_split && q.blocks_per_sm == c.blocks_per_sm && q.regcap != c.regcap) ||
                            (std::abs(q.split - c.split) == 32 && q.regcap == c.regcap &&
                             q.blocks_per_sm == c.blocks_per_sm);
            if (nb && time_one(i) == HF_ERR_CUDA) return HF_ERR_CUDA;
        }
        if (best->split == c.split && best->regcap == c.regcap && best->blocks_per_sm == c.blocks_per_sm)
            break;
    }
    if (n_timed) *n_timed = count;
    return best->time_us < 0.f ? HF_ERR_INVALID : HF_OK;
}
} // namespace

extern "C" hf_status hf_autotune_model(hf_kernel a, hf_kernel b, const void *const *args, int d0, int reps,
                                       int flush_l2_, void *stream, hf_tune_point *best, int *n_timed)
{
    if (!a || !b || !args || !best || reps < 1) return HF_ERR_INVALID;
    return autotune_model_impl(a, b, args, d0, reps, flush_l2_, stream, best, n_timed);
}

extern "C" hf_status hf_cost_model_set(const float *params, int n_models, float mu, float sd,
                                       const hf_pipe_peaks *peaks, int confirm)
{
    std::lock_guard<std::mutex> lk(g_cm_mu);
    if (!params) {
        g_cm_set = false;
        return HF_OK;
    }
    if (n_models < 1 || n_models > 16 || !peaks || confirm < 1 || !(sd > 0.f) || peaks->hbm_gbs <= 0 ||
        peaks->ffma_per_s <= 0)
        return HF_ERR_INVALID;
    g_cm.params.assign(params, params + (size_t)n_models * HF_MLP_NPARAMS);
    g_cm.n_models = n_models;
    g_cm.mu = mu;
    g_cm.sd = sd;
    g_cm.peaks = *peaks;
    g_cm.confirm = confirm;
    g_cm_set = true;
    return HF_OK;
}

extern "C" hf_status hf_autotune(hf_kernel a, hf_kernel b, const void *const *args, int d0, int mode,
                                 int reps, int flush_l2_, void *stream, hf_tune_point *best)
{
    if (!a || !b || !args || !best || reps < 1) return HF_ERR_INVALID;
    if (mode == HF_TUNE_MODEL)
        return autotune_model_impl(a, b, args, d0, reps, flush_l2_, stream, best, nullptr);
    if (mode == HF_TUNE_ALG2)
        return hf_search_alg2(a, b, args, d0, d0 >= 512 ? 128 : 64, reps, flush_l2_, stream, best,
                              nullptr, 0, nullptr);
    if (mode != HF_TUNE_EXHAUSTIVE || d0 < 64 || d0 > 1024 || d0 % 32) return HF_ERR_INVALID;
    std::vector<int> splits, caps = {0}, bps = {1, 2, 3, 4};
    for (int s = 32; s < d0; s += 32) splits.push_back(s);
    int nc = hf_regcaps(nullptr, 0);
    std::vector<int> compiled(nc > 0 ? nc : 0);
    if (nc > 0) hf_regcaps(compiled.data(), nc);
    caps.insert(caps.end(), compiled.begin(), compiled.end());
    std::vector<hf_tune_point> table(splits.size() * caps.size() * bps.size());
    hf_status st = hf_profile_pair(a, b, args, d0, splits.data(), (int)splits.size(), caps.data(),
                                   (int)caps.size(), bps.data(), (int)bps.size(), reps, flush_l2_, stream,
                                   table.data());
    if (st) return st;
    const hf_tune_point *pick = nullptr;
    for (const hf_tune_point &p : table)
        if (p.status == HF_OK && (!pick || p.time_us < pick->time_us)) pick = &p;
    if (!pick) return HF_ERR_INVALID;
    *best = *pick;
    return HF_OK;
}
