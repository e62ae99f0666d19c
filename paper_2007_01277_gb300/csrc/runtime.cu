// runtime.cu -- the C ABI declared in include/hfuse.h: kernel registration,
// 2-way and N-way fusion, validation, launch, resource queries and the
// register bound of Algorithm 2 (Sec. 3.2).
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "kernels.cuh"

using namespace hf;

// ------------------------------------------------------------------ errors
namespace {
thread_local std::string g_last_error;

hf_status fail(hf_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

#define HF_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return fail(HF_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// ------------------------------------------------------------------ body table
struct BodyOps {
    size_t args_size;
    hf_status (*validate)(const void *);
    size_t (*smem)(int, const void *);
    size_t (*workspace)(const void *);
    int barriers;
    int (*ring)(const void *);    // ring kind for these arguments (RingKind below)
    unsigned ring_min;            // stream ring: least bytes in flight per warp worth a ring;
                                  // item ring: the stage size (one work item)
    const char *name;
};

// How a body uses a bulk-copy ring: not at all; streaming whole tiles of a
// flat array (any stage size, a share of the SM's bytes in flight); or one
// work item per stage (a fixed stage of ring_min bytes, two per warp).
enum RingKind { kRingNone = 0, kRingStream = 1, kRingItem = 2 };

// Bodies with a ring path declare `static bool uses_ring(const Args &)`;
// those that take one work item per stage also declare kRingItem = true.
template <class B, class = void>
struct RingItem {
    static constexpr bool value = false;
};
template <class B>
struct RingItem<B, std::void_t<decltype(B::kRingItem)>> {
    static constexpr bool value = B::kRingItem;
};
template <class B, class = void>
struct RingTrait {
    static int uses(const void *) { return kRingNone; }
};
template <class B>
struct RingTrait<B, std::void_t<decltype(B::uses_ring(std::declval<const typename B::Args &>()))>> {
    static int uses(const void *p)
    {
        if (!B::uses_ring(*static_cast<const typename B::Args *>(p))) return kRingNone;
        return RingItem<B>::value ? kRingItem : kRingStream;
    }
};
template <class B, class = void>
struct RingMin {
    static constexpr unsigned value = 1024;
};
template <class B>
struct RingMin<B, std::void_t<decltype(B::kRingMinBytes)>> {
    static constexpr unsigned value = B::kRingMinBytes;
};

template <class B>
BodyOps ops(const char *name)
{
    using A = typename B::Args;
    return BodyOps{sizeof(A),
                   [](const void *p) { return B::validate(*static_cast<const A *>(p)); },
                   [](int n, const void *p) { return B::smem_bytes(n, *static_cast<const A *>(p)); },
                   [](const void *p) { return B::workspace_bytes(*static_cast<const A *>(p)); },
                   B::kBarriers, &RingTrait<B>::uses, RingMin<B>::value, name};
}

const BodyOps &body_ops(int id)
{
    static const BodyOps kOps[HF_BODY_COUNT] = {
        ops<BodyBn>("bn_stats"),     ops<BodyUpsample>("upsample2x"),
        ops<BodyMaxpool>("maxpool3s2"), ops<BodyIm2col>("im2col3"),
        ops<BodyHist>("hist256"),    ops<BodyPhilox>("philox"),
        ops<BodyPoly>("poly"),       ops<BodyBf16Axpy>("bf16_axpy"),
        ops<BodyStreamTmpl>("stream_tmpl"), ops<BodySha256d>("sha256d"),
        ops<BodyBlake256>("blake256"), ops<BodyBlake2b>("blake2b")};
    return kOps[id];
}

bool valid_body(int id) { return id >= 0 && id < HF_BODY_COUNT; }

size_t align128(size_t v) { return (v + 127) / 128 * 128; }

// ------------------------------------------------------------------ registry
struct Registry {
    std::vector<Instance> pairs, nway;
    std::vector<Instance> checked;   // pairs compiled with bounded software barriers
    std::vector<SingleEntry> singles;
    std::vector<int> caps;
};

const Registry &registry()
{
    static Registry r;
    static std::once_flag once;
    std::call_once(once, [] {
        const Instance *(*tabs[])(int *) = {pair_table_0, pair_table_1, pair_table_2, pair_table_3,
                                                   pair_table_4};
        for (auto t : tabs) {
            int n = 0;
            const Instance *p = t(&n);
            r.pairs.insert(r.pairs.end(), p, p + n);
        }
        int n = 0;
        const Instance *p = nway_table(&n);
        r.nway.assign(p, p + n);
        p = hfl::checked_pair_table(&n);
        r.checked.assign(p, p + n);
        const SingleEntry *s = single_table(&n);
        r.singles.assign(s, s + n);
        for (auto &i : r.nway)
            if (i.regcap) r.caps.push_back(i.regcap);
        std::sort(r.caps.begin(), r.caps.end());
    });
    return r;
}

bool cap_ok(int regcap)
{
    if (regcap == 0) return true;
    for (int c : registry().caps)
        if (c == regcap) return true;
    return false;
}

const Instance *find_nway(int regcap)
{
    for (auto &i : registry().nway)
        if (i.regcap == regcap) return &i;
    return nullptr;
}

const SingleEntry *find_single(int body)
{
    for (auto &s : registry().singles)
        if (s.body == body) return &s;
    return nullptr;
}

// ------------------------------------------------------------------ per-function state
struct FuncInfo {
    int regs = 0, local = 0, max_threads = 0;
    size_t smem_set = 48 * 1024;
};
std::mutex g_mu;
std::unordered_map<const void *, FuncInfo> g_funcs;   // keyed by symbol (one device)

hf_status func_info(const void *f, FuncInfo *out)
{
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_funcs.find(f);
        if (it != g_funcs.end()) {
            *out = it->second;
            return HF_OK;
        }
    }
    cudaFuncAttributes a;
    HF_CUDA(cudaFuncGetAttributes(&a, f));
    FuncInfo fi;
    fi.regs = a.numRegs;
    fi.local = (int)a.localSizeBytes;
    fi.max_threads = a.maxThreadsPerBlock;
    std::lock_guard<std::mutex> lk(g_mu);
    g_funcs.emplace(f, fi);
    *out = fi;
    return HF_OK;
}

hf_status ensure_smem(const void *f, size_t smem)
{
    std::lock_guard<std::mutex> lk(g_mu);
    FuncInfo &fi = g_funcs[f];
    if (smem <= fi.smem_set) return HF_OK;
    HF_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    fi.smem_set = smem;
    return HF_OK;
}

hf_status limits(hf_device_limits *lim)
{
    int dev = 0;
    HF_CUDA(cudaGetDevice(&dev));
    static std::mutex mu;
    static std::unordered_map<int, hf_device_limits> cache;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(dev);
        if (it != cache.end()) {
            *lim = it->second;
            return HF_OK;
        }
    }
    cudaDeviceProp p;
    HF_CUDA(cudaGetDeviceProperties(&p, dev));
    hf_device_limits l;
    l.sm_count = p.multiProcessorCount;
    l.regs_per_sm = p.regsPerMultiprocessor;
    l.smem_per_sm = (int)p.sharedMemPerMultiprocessor;
    l.threads_per_sm = p.maxThreadsPerMultiProcessor;
    l.smem_per_block_optin = (int)p.sharedMemPerBlockOptin;
    l.l2_bytes = p.l2CacheSize;
    l.cc_major = p.major;
    l.cc_minor = p.minor;
    std::lock_guard<std::mutex> lk(mu);
    cache[dev] = l;
    *lim = l;
    return HF_OK;
}

hf_status check_threads(const hf_kernel_t *k, int t);

} // namespace

// ------------------------------------------------------------------ handles
struct hf_kernel_t {
    int body;
    int tmin, tmax, gran;
    std::string name;
};

// Static facts of a body for the cost model's features (costmodel.cu).
namespace hf {
int kernel_body_id(const hf_kernel_t *k) { return k ? k->body : -1; }
size_t body_smem_bytes(int id, int threads, const void *args)
{
    return valid_body(id) ? body_ops(id).smem(threads, args) : 0;
}
int body_barriers(int id) { return valid_body(id) ? body_ops(id).barriers : 0; }
hf_status body_validate(int id, const void *args)
{
    return valid_body(id) ? body_ops(id).validate(args) : HF_ERR_INVALID;
}
} // namespace hf

struct hf_fused_t {
    bool nway;
    int regcap;
    int d0;
    // pair
    int body_low, body_high, n_low, n_high;
    const Instance *inst;
    int low_is_a;   // instance body A runs on the low interval
    // N-way
    int n;
    int sched_body[HF_MAX_SCHEDULE];
    int sched_int[HF_MAX_SCHEDULE];
    int n_int;
    int int_threads[HF_MAX_INTERVALS];
};

namespace {
hf_status check_threads(const hf_kernel_t *k, int t)
{
    if (t % 32 || t < k->tmin || t > k->tmax || t % k->gran)
        return fail(HF_ERR_SPLIT, "%d threads outside kernel '%s' range [%d, %d] step %d", t,
                    k->name.c_str(), k->tmin, k->tmax, k->gran);
    return HF_OK;
}

// Resident blocks of `func` at d0 threads and `smem` bytes (cached, so that
// a launch recorded into a graph makes no occupancy query).
hf_status occ_blocks(const void *func, int d0, size_t smem, int *b)
{
    hf_status s = ensure_smem(func, smem);
    if (s) return s;
    static std::mutex occ_mu;
    static std::unordered_map<std::string, int> occ;
    char key[96];
    snprintf(key, sizeof key, "%p/%d/%zu", func, d0, smem);
    {
        std::lock_guard<std::mutex> lk(occ_mu);
        auto it = occ.find(key);
        if (it != occ.end()) {
            *b = it->second;
            return HF_OK;
        }
    }
    HF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, func, d0, smem));
    std::lock_guard<std::mutex> lk(occ_mu);
    occ[key] = *b;
    return HF_OK;
}

// Bulk-copy ring geometry for F bytes in flight per warp (about 40 KB per
// SM over the SM's ring warps, where HBM bandwidth peaks; more in flight
// costs bandwidth): stages of 1, 2 or 4 KB, 2 to 4 per warp.  Below 1 KB
// per warp register loads do as well: no ring.
void ring_geom(double F, unsigned *stage, int *stages)
{
    *stage = 0;
    *stages = 0;
    if (F < 1024.0) return;
    unsigned B = 1024;
    while (B < 4096 && 2.0 * B <= F) B *= 2;
    *stage = B;
    *stages = std::min(4, std::max(2, 1 + (int)(F / B + 0.5)));
}

// The ring decision for `b` resident blocks of a block whose intervals have
// warps[i] warps, ring kind kind[i] and ring_min[i].  Item rings (where
// item_ok[i], or everywhere when item_ok is NULL) get their fixed geometry: stages of ring_min[i] bytes, two per
// warp.  Stream rings share about 40 KB in flight per SM over their warps
// (the bf16 stream's optimum); intervals whose minimum the SM's share misses
// drop their ring and the share is recomputed over the rest.  Returns which
// intervals keep a ring and each one's stage bytes and stages.
constexpr int kItemStages = 2;
void ring_choice(int n, const int *warps, const int *kind, const unsigned *ring_min, int b,
                 const bool *item_ok, bool *use, unsigned *stage, int *stages)
{
    for (int i = 0; i < n; ++i) {
        use[i] = b > 0 && (kind[i] == kRingStream || (kind[i] == kRingItem && (!item_ok || item_ok[i])));
        stage[i] = 0;
        stages[i] = 0;
    }
    double F = 0.0;
    for (bool changed = true; changed;) {
        changed = false;
        int w = 0;
        for (int i = 0; i < n; ++i)
            if (use[i] && kind[i] == kRingStream) w += warps[i];
        F = w > 0 ? 40960.0 / ((double)b * w) : 0.0;
        for (int i = 0; i < n; ++i)
            if (use[i] && kind[i] == kRingStream && F < ring_min[i]) use[i] = false, changed = true;
    }
    unsigned sB = 0;
    int sS = 0;
    ring_geom(F, &sB, &sS);
    for (int i = 0; i < n; ++i) {
        if (!use[i]) continue;
        if (kind[i] == kRingItem) {
            stage[i] = (ring_min[i] + 127u) / 128u * 128u;
            stages[i] = kItemStages;
        } else if (sS > 0) {
            stage[i] = sB;
            stages[i] = sS;
        } else {
            use[i] = false;
        }
    }
}

// Shared-memory layout, ring geometry and grid of one launch.
struct LaunchPlan {
    unsigned off[HF_MAX_INTERVALS];          // slice offsets
    unsigned ring_stage[HF_MAX_INTERVALS];   // per interval, 0 = no ring
    int ring_stages[HF_MAX_INTERVALS];
    unsigned smem;                           // total dynamic shared memory
    int grid, bps;
};

// Plans a launch of `func` with d0 threads cut into n intervals of
// threads[i] whose kernels need base[i] bytes of shared memory and, where
// ring[i], a bulk-copy ring after it.  The blocks per SM are the most that
// stay resident once the rings are sized for that many blocks (or, with an
// explicit grid `want`, no more than it spreads over the SMs); the grid is
// `want` or blocks per SM x SMs.
hf_status plan_launch(const void *func, int d0, int n, const int *threads, const size_t *base,
                      const int *ring, const unsigned *ring_min, int want, LaunchPlan *out)
{
    hf_device_limits lim;
    hf_status s = limits(&lim);
    if (s) return s;
    size_t base_total = 0;
    int ring_w = 0;
    for (int i = 0; i < n; ++i) {
        base_total += align128(base[i]);
        if (ring[i]) ring_w += threads[i] / 32;
    }
    if (base_total > (size_t)lim.smem_per_block_optin)
        return fail(HF_ERR_SMEM, "combined shared memory %zu B above the %d B per-block limit", base_total,
                    lim.smem_per_block_optin);
    int bmax = 0;
    s = occ_blocks(func, d0, base_total, &bmax);
    if (s) return s;
    if (bmax <= 0)
        return fail(HF_ERR_REGS, "block of %d threads with %zu B shared memory cannot be resident", d0,
                    base_total);
    if (want > 0) bmax = std::max(1, std::min(bmax, (want + lim.sm_count - 1) / lim.sm_count));
    // item intervals, largest ring first: the order in which they give up
    // their ring when shared memory runs out
    int drop[HF_MAX_INTERVALS], n_item = 0;
    for (int i = 0; i < n; ++i)
        if (ring[i] == kRingItem) drop[n_item++] = i;
    std::sort(drop, drop + n_item, [&](int x, int y) {
        return (size_t)threads[x] * ring_min[x] > (size_t)threads[y] * ring_min[y];
    });
    for (int b = bmax; b >= 0; --b)
        for (int k = 0; k <= n_item; ++k) {
            // b == 0: the last resort, no rings at the largest block count.
            // Item rings that do not fit go, largest first, before the block
            // count drops; stream intervals whose body wants more in flight
            // per warp than the SM's share gives drop their ring (register
            // loads).
            bool use[HF_MAX_INTERVALS], item_ok[HF_MAX_INTERVALS];
            int warps[HF_MAX_INTERVALS], stages[HF_MAX_INTERVALS];
            unsigned stage[HF_MAX_INTERVALS];
            for (int i = 0; i < n; ++i) warps[i] = threads[i] / 32, item_ok[i] = true;
            for (int j = 0; j < k; ++j) item_ok[drop[j]] = false;
            ring_choice(n, warps, ring, ring_min, b, item_ok, use, stage, stages);
            size_t off = 0;
            for (int i = 0; i < n; ++i) {
                out->off[i] = (unsigned)off;
                const bool r = use[i] && stages[i] > 0;
                out->ring_stage[i] = r ? stage[i] : 0;
                out->ring_stages[i] = r ? stages[i] : 0;
                off += align128(align128(base[i]) + (r ? ring_bytes(threads[i], stage[i], stages[i]) : 0));
            }
            if (off > (size_t)lim.smem_per_block_optin) continue;
            int got = 0;
            s = occ_blocks(func, d0, off, &got);
            if (s) return s;
            if (got >= std::max(b, 1)) {
                out->smem = (unsigned)off;
                out->bps = b > 0 ? b : bmax;
                out->grid = want > 0 ? want : out->bps * lim.sm_count;
                return HF_OK;
            }
        }
    return fail(HF_ERR_REGS, "no resident configuration for a block of %d threads", d0);
}

} // namespace

// Shared memory of each interval of a two-interval block at b blocks per SM
// as the launch planner gives it: the body's slice plus the bulk-copy ring
// the ring planner hands it at that occupancy (host arithmetic, no device
// query; the cost model's features).
namespace hf {
void interval_smem_at(const int *ids, const void *const *args, const int *threads, int b, double *out)
{
    bool use[2];
    unsigned mins[2], stage[2];
    int kind[2], warps[2], stages[2];
    for (int i = 0; i < 2; ++i) {
        kind[i] = valid_body(ids[i]) ? body_ops(ids[i]).ring(args[i]) : kRingNone;
        mins[i] = valid_body(ids[i]) ? body_ops(ids[i]).ring_min : 0u;
        warps[i] = threads[i] / 32;
    }
    ring_choice(2, warps, kind, mins, b, nullptr, use, stage, stages);
    for (int i = 0; i < 2; ++i) {
        const double base = valid_body(ids[i]) ? (double)body_ops(ids[i]).smem(threads[i], args[i]) : 0.0;
        out[i] = base + (use[i] && stages[i] > 0 ? (double)ring_bytes(threads[i], stage[i], stages[i]) : 0.0);
    }
}
} // namespace hf

namespace {
hf_status single_plan(const hf_kernel_t *k, const void *args, int threads, int want, LaunchPlan *plan)
{
    const SingleEntry *e = find_single(k->body);
    const size_t base = body_ops(k->body).smem(threads, args);
    const int ring = body_ops(k->body).ring(args);
    const unsigned ring_min = body_ops(k->body).ring_min;
    return plan_launch(e->func, threads, 1, &threads, &base, &ring, &ring_min, want, plan);
}

hf_status validate_args(int body, const void *a, int which)
{
    if (!a) return fail(HF_ERR_INVALID, "argument block %d is NULL", which);
    hf_status s = body_ops(body).validate(a);
    if (s) return fail(s, "argument block %d (%s) rejected", which, body_ops(body).name);
    return HF_OK;
}

// Builds the N-way parameter block; also used for pairs without a compiled
// pair instance.
hf_status nway_params(const hf_fused_t *f, const void *const *args, int want, NwayParams *p,
                      LaunchPlan *plan)
{
    std::memset(p, 0, sizeof *p);
    p->n_int = f->n_int;
    int w = 0;
    size_t base[HF_MAX_INTERVALS];
    int ring[HF_MAX_INTERVALS];
    unsigned ring_min[HF_MAX_INTERVALS];
    for (int i = 0; i < f->n_int; ++i) {
        p->warp_begin[i] = w;
        w += f->int_threads[i] / 32;
        base[i] = 0;
        ring[i] = kRingNone;
        ring_min[i] = 0;
        // kernels sharing an interval share its ring: item geometry (the
        // largest item) when any of them takes items, a stream share else
        unsigned item_min = 0, stream_min = 0;
        for (int j = 0; j < f->n; ++j)
            if (f->sched_int[j] == i) {
                const BodyOps &o = body_ops(f->sched_body[j]);
                base[i] = std::max(base[i], o.smem(f->int_threads[i], args[j]));
                const int k = o.ring(args[j]);
                if (k == kRingItem) item_min = std::max(item_min, o.ring_min);
                if (k == kRingStream) stream_min = std::max(stream_min, o.ring_min);
            }
        if (item_min) ring[i] = kRingItem, ring_min[i] = item_min;
        else if (stream_min) ring[i] = kRingStream, ring_min[i] = stream_min;
    }
    p->warp_begin[f->n_int] = w;
    for (int i = 0; i < f->n_int; ++i)
        for (int k = p->warp_begin[i]; k < p->warp_begin[i + 1]; ++k) p->warp_int[k] = (unsigned char)i;
    // slots sorted by interval; kernels sharing an interval keep the
    // caller's order
    size_t boff = 0;
    int slot = 0;
    p->poly_slot = -1;
    for (int i = 0; i < f->n_int; ++i) {
        p->int_first[i] = slot;
        for (int j = 0; j < f->n; ++j) {
            if (f->sched_int[j] != i) continue;
            const size_t sz = body_ops(f->sched_body[j]).args_size;
            boff = (boff + 15) / 16 * 16;
            if (boff + sz > (size_t)kNwayBlob)
                return fail(HF_ERR_INVALID, "argument blocks exceed %d B", kNwayBlob);
            std::memcpy(p->blob + boff, args[j], sz);
            if (f->sched_body[j] == HF_BODY_POLY && p->poly_slot < 0) {
                p->poly_slot = slot;
                std::memcpy(&p->poly, args[j], sizeof p->poly);
            }
            p->sched_body[slot] = f->sched_body[j];
            p->args_off[slot] = (unsigned)boff;
            boff += sz;
            ++slot;
        }
    }
    p->int_first[f->n_int] = slot;
    hf_status s = plan_launch(f->inst->func, f->d0, f->n_int, f->int_threads, base, ring, ring_min, want,
                              plan);
    if (s) return s;
    for (int i = 0; i < f->n_int; ++i) {
        p->smem_off[i] = plan->off[i];
        p->ring_stage[i] = plan->ring_stage[i];
        p->ring_stages[i] = plan->ring_stages[i];
    }
    return HF_OK;
}

// Plans a 2-way fused launch.
hf_status pair_plan(const hf_fused_t *f, const void *const *uargs, int want, LaunchPlan *plan)
{
    const int threads[2] = {f->n_low, f->n_high};
    const size_t base[2] = {body_ops(f->body_low).smem(f->n_low, uargs[0]),
                            body_ops(f->body_high).smem(f->n_high, uargs[1])};
    const int ring[2] = {body_ops(f->body_low).ring(uargs[0]), body_ops(f->body_high).ring(uargs[1])};
    const unsigned ring_min[2] = {body_ops(f->body_low).ring_min, body_ops(f->body_high).ring_min};
    return plan_launch(f->inst->func, f->d0, 2, threads, base, ring, ring_min, want, plan);
}
} // namespace

// Records a one-line error for hf_last_error() from other translation units.
namespace hf {
hf_status set_last_error(hf_status s, const char *msg) { return fail(s, "%s", msg); }

// The device error word: a file-scope device variable (no allocation),
// its address looked up once per device.
static __device__ unsigned g_hf_error_word;

unsigned *error_word()
{
    static std::mutex mu;
    static unsigned *addr[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_hf_error_word) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        addr[dev] = static_cast<unsigned *>(p);
    }
    return addr[dev];
}
} // namespace hf

// ------------------------------------------------------------------ C ABI
extern "C" {

hf_status hf_ring_plan(int n, const int *warps, const int *ring, const unsigned *min_bytes,
                       int blocks_per_sm, unsigned *stage, int *stages, int *uses)
{
    if (n < 1 || n > HF_MAX_INTERVALS || !warps || !ring || !min_bytes || !stage || !stages || !uses ||
        blocks_per_sm < 1)
        return fail(HF_ERR_INVALID, "bad ring-plan arguments");
    int kind[HF_MAX_INTERVALS];
    bool use[HF_MAX_INTERVALS];
    for (int i = 0; i < n; ++i) {
        if (ring[i] < kRingNone || ring[i] > kRingItem) return fail(HF_ERR_INVALID, "bad ring kind");
        kind[i] = ring[i];
    }
    ring_choice(n, warps, kind, min_bytes, blocks_per_sm, nullptr, use, stage, stages);
    for (int i = 0; i < n; ++i) uses[i] = use[i] ? 1 : 0;
    return HF_OK;
}

hf_status hf_check_device_error(unsigned *flags, int clear)
{
    if (!flags) return fail(HF_ERR_INVALID, "NULL flags");
    HF_CUDA(cudaMemcpyFromSymbol(flags, hf::g_hf_error_word, sizeof(unsigned)));
    if (clear && *flags) {
        const unsigned z = 0;
        HF_CUDA(cudaMemcpyToSymbol(hf::g_hf_error_word, &z, sizeof z));
    }
    return HF_OK;
}

const char *hf_status_string(hf_status s)
{
    switch (s) {
    case HF_OK: return "ok";
    case HF_ERR_INVALID: return "invalid argument";
    case HF_ERR_SPLIT: return "invalid thread split";
    case HF_ERR_BARRIER: return "too many barrier intervals";
    case HF_ERR_SMEM: return "shared memory limit exceeded";
    case HF_ERR_REGS: return "block too large for the register use";
    case HF_ERR_UNSUPPORTED: return "configuration not compiled";
    case HF_ERR_CUDA: return "CUDA runtime error";
    case HF_ERR_TIMEOUT: return "timeout";
    }
    return "unknown status";
}

const char *hf_last_error(void) { return g_last_error.c_str(); }

size_t hf_args_size(int body_id) { return valid_body(body_id) ? body_ops(body_id).args_size : 0; }

int hf_regcaps(int *caps, int cap)
{
    const auto &c = registry().caps;
    for (int i = 0; i < (int)c.size() && i < cap; ++i) caps[i] = c[i];
    return (int)c.size();
}

hf_status hf_register_kernel(const hf_kernel_desc *d, hf_kernel *out)
{
    if (!d || !out) return fail(HF_ERR_INVALID, "NULL descriptor or output");
    if (!valid_body(d->body_id)) return fail(HF_ERR_INVALID, "unknown body id %d", d->body_id);
    const int tmin = d->min_threads ? d->min_threads : 32;
    const int tmax = d->max_threads ? d->max_threads : 1024;
    const int gran = d->thread_granularity ? d->thread_granularity : 32;
    if (tmin % 32 || tmax % 32 || gran % 32 || tmin < 32 || tmax > 1024 || tmin > tmax || gran <= 0)
        return fail(HF_ERR_INVALID, "thread range [%d, %d] step %d not warp aligned", tmin, tmax, gran);
    hf_kernel_t *k = new hf_kernel_t{d->body_id, tmin, tmax, gran,
                                     d->name ? d->name : body_ops(d->body_id).name};
    *out = k;
    return HF_OK;
}

void hf_destroy_kernel(hf_kernel k) { delete k; }

namespace {
// Algorithm 1 for two registered kernels: validation, then the compiled
// instance for (body pair, register cap) -- from the production instances,
// or from the checked-barrier ones when `checked` is set (which have no
// N-way fallback).
hf_status fuse_pair(hf_kernel a, hf_kernel b, int split, int d0, int regcap, bool checked,
                    hf_fused *out)
{
    if (!a || !b || !out) return fail(HF_ERR_INVALID, "NULL kernel or output");
    if (d0 % 32 || split % 32 || split <= 0 || split >= d0 || d0 > 1024)
        return fail(HF_ERR_SPLIT, "split %d of block %d: need multiples of 32, 0 < split < d0 <= 1024", split, d0);
    hf_status s = check_threads(a, split);
    if (s) return s;
    s = check_threads(b, d0 - split);
    if (s) return s;
    if (!cap_ok(regcap)) return fail(HF_ERR_UNSUPPORTED, "register cap %d not compiled", regcap);
    hf_fused_t *f = new hf_fused_t();
    f->regcap = regcap;
    f->d0 = d0;
    f->body_low = a->body;
    f->body_high = b->body;
    f->n_low = split;
    f->n_high = d0 - split;
    f->inst = nullptr;
    for (auto &i : checked ? registry().checked : registry().pairs) {
        if (i.regcap != regcap) continue;
        if (i.body_a == a->body && i.body_b == b->body) {
            f->inst = &i;
            f->low_is_a = 1;
            break;
        }
        if (i.body_a == b->body && i.body_b == a->body) {
            f->inst = &i;
            f->low_is_a = 0;
            break;
        }
    }
    if (!f->inst && checked) {
        delete f;
        return fail(HF_ERR_UNSUPPORTED, "no checked-barrier instance of this body pair");
    }
    if (!f->inst) {   // no compiled pair: the generic N-way kernel with two intervals
        f->nway = true;
        f->inst = find_nway(regcap);
        f->n = 2;
        f->n_int = 2;
        f->sched_body[0] = a->body;
        f->sched_body[1] = b->body;
        f->sched_int[0] = 0;
        f->sched_int[1] = 1;
        f->int_threads[0] = split;
        f->int_threads[1] = d0 - split;
    }
    FuncInfo fi;
    s = func_info(f->inst->func, &fi);
    if (s) {
        delete f;
        return s;
    }
    if (fi.max_threads < d0) {
        delete f;
        return fail(HF_ERR_REGS, "fused instance uses %d registers: at most %d threads per block, asked %d",
                    fi.regs, fi.max_threads, d0);
    }
    *out = f;
    return HF_OK;
}
} // namespace

hf_status hf_fuse(hf_kernel a, hf_kernel b, int split, int d0, int regcap, hf_fused *out)
{
    return fuse_pair(a, b, split, d0, regcap, false, out);
}

hf_status hf_fuse_checked(hf_kernel a, hf_kernel b, int split, int d0, hf_fused *out)
{
    return fuse_pair(a, b, split, d0, 0, true, out);
}

hf_status hf_fuse_n(const hf_kernel *ks, int n, const int *interval_of, const int *interval_threads,
                    int n_intervals, int regcap, hf_fused *out)
{
    if (!ks || !interval_of || !interval_threads || !out) return fail(HF_ERR_INVALID, "NULL argument");
    if (n < 1 || n > HF_MAX_SCHEDULE) return fail(HF_ERR_INVALID, "%d kernels (1..%d)", n, HF_MAX_SCHEDULE);
    if (n_intervals < 1) return fail(HF_ERR_INVALID, "no intervals");
    if (n_intervals > HF_MAX_INTERVALS)
        return fail(HF_ERR_BARRIER, "%d intervals: only %d named barrier ids", n_intervals, HF_MAX_INTERVALS);
    int d0 = 0;
    for (int i = 0; i < n_intervals; ++i) {
        if (interval_threads[i] <= 0 || interval_threads[i] % 32)
            return fail(HF_ERR_SPLIT, "interval %d has %d threads", i, interval_threads[i]);
        d0 += interval_threads[i];
    }
    if (d0 > 1024) return fail(HF_ERR_SPLIT, "block of %d threads", d0);
    std::vector<int> used(n_intervals, 0);
    for (int j = 0; j < n; ++j) {
        if (!ks[j]) return fail(HF_ERR_INVALID, "kernel %d is NULL", j);
        if (interval_of[j] < 0 || interval_of[j] >= n_intervals)
            return fail(HF_ERR_INVALID, "kernel %d on interval %d", j, interval_of[j]);
        hf_status s = check_threads(ks[j], interval_threads[interval_of[j]]);
        if (s) return s;
        used[interval_of[j]] = 1;
    }
    for (int i = 0; i < n_intervals; ++i)
        if (!used[i]) return fail(HF_ERR_INVALID, "interval %d runs no kernel", i);
    if (!cap_ok(regcap)) return fail(HF_ERR_UNSUPPORTED, "register cap %d not compiled", regcap);
    hf_fused_t *f = new hf_fused_t();
    f->nway = true;
    f->regcap = regcap;
    f->d0 = d0;
    f->inst = find_nway(regcap);
    f->n = n;
    f->n_int = n_intervals;
    for (int j = 0; j < n; ++j) {
        f->sched_body[j] = ks[j]->body;
        f->sched_int[j] = interval_of[j];
    }
    for (int i = 0; i < n_intervals; ++i) f->int_threads[i] = interval_threads[i];
    FuncInfo fi;
    hf_status s = func_info(f->inst->func, &fi);
    if (s) {
        delete f;
        return s;
    }
    if (fi.max_threads < d0) {
        delete f;
        return fail(HF_ERR_REGS, "N-way instance uses %d registers: at most %d threads per block", fi.regs,
                    fi.max_threads);
    }
    *out = f;
    return HF_OK;
}

void hf_destroy_fused(hf_fused f) { delete f; }

static hf_status launch_impl(hf_fused f, const void *const *args, int grid, void *stream,
                             unsigned long long *trace);

hf_status hf_launch(hf_fused f, const void *const *args, int grid, void *stream)
{
    return launch_impl(f, args, grid, stream, nullptr);
}

hf_status hf_launch_traced(hf_fused f, const void *const *args, int grid, void *stream,
                           unsigned long long *trace)
{
    if (!trace) return fail(HF_ERR_INVALID, "NULL trace buffer");
    if (f && !f->nway) return fail(HF_ERR_UNSUPPORTED, "interval tracing needs an N-way fused kernel");
    return launch_impl(f, args, grid, stream, trace);
}

static hf_status launch_impl(hf_fused f, const void *const *args, int grid, void *stream,
                             unsigned long long *trace)
{
    if (!f || !args) return fail(HF_ERR_INVALID, "NULL fused kernel or argument list");
    if (grid < 0) return fail(HF_ERR_INVALID, "grid %d", grid);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!f->nway) {
        hf_status s = validate_args(f->body_low, args[0], 0);
        if (s) return s;
        s = validate_args(f->body_high, args[1], 1);
        if (s) return s;
        const void *iargs[2] = {f->low_is_a ? args[0] : args[1], f->low_is_a ? args[1] : args[0]};
        LaunchPlan plan;
        s = pair_plan(f, iargs, grid, &plan);
        if (s) return s;
        PairLaunch L{iargs, f->n_low / 32, f->n_low, f->n_high, plan.off[1], plan.smem, f->low_is_a,
                     plan.grid, f->d0, hf::error_word(), {plan.ring_stage[0], plan.ring_stage[1]},
                     {plan.ring_stages[0], plan.ring_stages[1]}};
        HF_CUDA(f->inst->launch_pair(L, st));
        return HF_OK;
    }
    for (int j = 0; j < f->n; ++j) {
        hf_status s = validate_args(f->sched_body[j], args[j], j);
        if (s) return s;
    }
    static thread_local NwayParams p;
    LaunchPlan plan;
    hf_status s = nway_params(f, args, grid, &p, &plan);
    if (s) return s;
    p.trace = trace;
    p.err = hf::error_word();
    void *kargs[] = {&p};
    HF_CUDA(cudaLaunchKernel(f->inst->func, dim3(plan.grid), dim3(f->d0), kargs, plan.smem, st));
    return HF_OK;
}

hf_status hf_launch_single(hf_kernel k, const void *args, int threads, int grid, void *stream)
{
    if (!k) return fail(HF_ERR_INVALID, "NULL kernel");
    if (grid < 0) return fail(HF_ERR_INVALID, "grid %d", grid);
    hf_status s = check_threads(k, threads);
    if (s) return s;
    s = validate_args(k->body, args, 0);
    if (s) return s;
    const SingleEntry *e = find_single(k->body);
    FuncInfo fi;
    s = func_info(e->func, &fi);
    if (s) return s;
    if (fi.max_threads < threads)
        return fail(HF_ERR_REGS, "kernel uses %d registers: at most %d threads", fi.regs, fi.max_threads);
    LaunchPlan plan;
    s = single_plan(k, args, threads, grid, &plan);
    if (s) return s;
    HF_CUDA(e->launch(args, threads, plan.grid, plan.smem, hf::error_word(), plan.ring_stage[0],
                      plan.ring_stages[0], static_cast<cudaStream_t>(stream)));
    return HF_OK;
}

hf_status hf_query(hf_fused f, const void *const *args, hf_fused_info *info)
{
    if (!f || !args || !info) return fail(HF_ERR_INVALID, "NULL argument");
    LaunchPlan plan;
    if (!f->nway) {
        const void *iargs[2] = {f->low_is_a ? args[0] : args[1], f->low_is_a ? args[1] : args[0]};
        hf_status s = pair_plan(f, iargs, 0, &plan);
        if (s) return s;
    } else {
        static thread_local NwayParams p;
        hf_status s = nway_params(f, args, 0, &p, &plan);
        if (s) return s;
    }
    FuncInfo fi;
    hf_status s = func_info(f->inst->func, &fi);
    if (s) return s;
    const unsigned smem = plan.smem;
    const int bps = plan.bps;
    info->regs = fi.regs;
    info->spill_bytes = fi.local;
    info->smem_bytes = (int)smem;
    info->block_threads = f->d0;
    info->blocks_per_sm = bps;
    info->max_threads_per_block = fi.max_threads;
    info->n_intervals = f->nway ? f->n_int : 2;
    return HF_OK;
}

hf_status hf_query_single(hf_kernel k, const void *args, int threads, hf_fused_info *info)
{
    if (!k || !args || !info) return fail(HF_ERR_INVALID, "NULL argument");
    hf_status s = check_threads(k, threads);
    if (s) return s;
    const SingleEntry *e = find_single(k->body);
    FuncInfo fi;
    s = func_info(e->func, &fi);
    if (s) return s;
    LaunchPlan plan;
    s = single_plan(k, args, threads, 0, &plan);
    if (s) return s;
    const size_t smem = plan.smem;
    const int bps = plan.bps;
    info->regs = fi.regs;
    info->spill_bytes = fi.local;
    info->smem_bytes = (int)smem;
    info->block_threads = threads;
    info->blocks_per_sm = bps;
    info->max_threads_per_block = fi.max_threads;
    info->n_intervals = 1;
    return HF_OK;
}

hf_status hf_workspace_size(int body_id, const void *args, size_t *bytes)
{
    if (!valid_body(body_id) || !args || !bytes) return fail(HF_ERR_INVALID, "bad body id or NULL");
    *bytes = body_ops(body_id).workspace(args);
    return HF_OK;
}

hf_status hf_device_info(hf_device_limits *lim)
{
    if (!lim) return fail(HF_ERR_INVALID, "NULL output");
    return limits(lim);
}

hf_status hf_register_bound(const hf_device_limits *lim, int d1, int nregs1, int d2, int nregs2,
                            int smem_fused, int *r0)
{
    if (!lim || !r0 || d1 <= 0 || d2 <= 0 || nregs1 <= 0 || nregs2 <= 0 || smem_fused < 0)
        return fail(HF_ERR_INVALID, "bad register-bound input");
    const int d0 = d1 + d2;
    // resident blocks the two original kernels reach on their registers
    int b0 = std::min(lim->regs_per_sm / (d1 * nregs1), lim->regs_per_sm / (d2 * nregs2));
    if (smem_fused > 0) b0 = std::min(b0, lim->smem_per_sm / smem_fused);
    b0 = std::min(b0, lim->threads_per_sm / d0);
    *r0 = b0 > 0 ? lim->regs_per_sm / (b0 * d0) : 0;
    return HF_OK;
}

hf_status hf_stream_wait(void *stream, int timeout_ms)
{
    if (timeout_ms < 0) return fail(HF_ERR_INVALID, "negative timeout");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(st);
        if (e == cudaSuccess) return HF_OK;
        if (e != cudaErrorNotReady) return fail(HF_ERR_CUDA, "cudaStreamQuery: %s", cudaGetErrorString(e));
        const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                            std::chrono::steady_clock::now() - t0).count();
        if (ms >= timeout_ms) return fail(HF_ERR_TIMEOUT, "stream not done after %d ms", timeout_ms);
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

} // extern "C"
