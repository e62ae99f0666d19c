// costmodel.cu -- static features of a fused pair for the learned cost
// model (host arithmetic only).
//
// The model predicts log(fused time) of two parametric stream kernels fused
// in one block from features that need no profiling: for each kernel its
// size, FMAs per 16 bytes, barriers, shared memory, an HBM/FP32 roofline
// estimate of its time alone, how compute-bound that estimate is, its share
// of the block's threads, its resident warps per SM and its share of the
// pair's estimated work; and for the configuration the register cap,
// blocks per SM, thread occupancy, the fused instance's registers and spill
// bytes, and the shared-memory occupancy.  All features are scaled to about
// [0, 1].
#include <cmath>

#include "kernels.cuh"

namespace hf {
hf_status set_last_error(hf_status s, const char *msg);   // runtime.cu
}

extern "C" hf_status hf_tmpl_features(const hf_stream_tmpl_args *a, const hf_stream_tmpl_args *b,
                                      int split, int d0, int regcap, int blocks_per_sm,
                                      int fused_regs, int spill_bytes, double hbm_gbs,
                                      double ffma_per_s, float *out)
{
    if (!a || !b || !out || split <= 0 || split >= d0 || blocks_per_sm < 1 || hbm_gbs <= 0 ||
        ffma_per_s <= 0)
        return hf::set_last_error(HF_ERR_INVALID, "bad feature arguments");
    const hf_stream_tmpl_args *ks[2] = {a, b};
    const int thr[2] = {split, d0 - split};
    double est[2], comp[2];
    for (int i = 0; i < 2; ++i) {
        const double n = (double)ks[i]->n;
        const double t_mem = 8.0 * n / (hbm_gbs * 1e9);
        const double t_fma = (double)ks[i]->k * n / 4.0 / ffma_per_s;
        est[i] = std::max(t_mem, t_fma) * 1e6;
        comp[i] = t_fma / std::max(t_mem + t_fma, 1e-30);
    }
    const double tot = est[0] + est[1];
    int f = 0;
    for (int i = 0; i < 2; ++i) {
        const hf_stream_tmpl_args *k = ks[i];
        out[f++] = (float)(std::log2((double)std::max<int64_t>(k->n, 1)) / 28.0);
        out[f++] = (float)(std::log2(1.0 + k->k) / 8.0);
        out[f++] = (float)(k->n_barriers / 4.0);
        out[f++] = (float)(k->smem_bytes / 49152.0);
        out[f++] = (float)(std::log2(1.0 + est[i]) / 12.0);
        out[f++] = (float)comp[i];
        out[f++] = (float)((double)thr[i] / d0);
        out[f++] = (float)(thr[i] / 32.0 * blocks_per_sm / 64.0);
        out[f++] = (float)(est[i] / std::max(tot, 1e-30));
    }
    out[f++] = (float)((regcap ? regcap : 255) / 255.0);
    out[f++] = (float)(blocks_per_sm / 4.0);
    out[f++] = (float)(blocks_per_sm * (double)d0 / 2048.0);
    out[f++] = (float)(fused_regs / 255.0);
    out[f++] = (float)(std::log2(1.0 + spill_bytes) / 10.0);
    out[f++] = (float)((double)(a->smem_bytes + b->smem_bytes) * blocks_per_sm / 233472.0);
    return HF_OK;
}

// ------------------------------------------------------------------------
// Features of any pair of registered kernels.  Each body's algorithmic work
// (bytes and operations per pipe) comes from its arguments; the features
// are those of the stream template with the template's quantities replaced
// by their general counterparts: size = HBM bytes / 8 (a template float
// moves 8 bytes), FMAs per 16 B loaded = the busiest pipe's operations in
// FMA time per 32 bytes moved, the roofline estimate = max(HBM time,
// busiest pipe time).  For two stream templates every feature is computed
// from the same numbers as in hf_tmpl_features, so the two agree.
namespace hf {
int kernel_body_id(const hf_kernel_t *k);   // runtime.cu
size_t body_smem_bytes(int id, int threads, const void *args);
int body_barriers(int id);
hf_status body_validate(int id, const void *args);
void interval_smem_at(const int *ids, const void *const *args, const int *threads, int b, double *out);
}

namespace {

// 32-bit operations per item of the hash scans, as their definitions count
// them (a three-input add or XOR once, a rotate once, a 64-bit operation
// twice): SHA-256d two compressions of 64 x 14 + 48 x 10; BLAKE-256 14
// rounds x 8 G x 14; BLAKE2b 12 rounds x 8 G x 22.
constexpr double kOpsSha256d = 2.0 * 1376.0, kOpsBlake256 = 14.0 * 8 * 14, kOpsBlake2b = 12.0 * 8 * 22;

struct Terms {
    double bytes, t_mem, t_c, fma_equiv;
};

Terms terms_of(const hf_body_work &w, const hf_pipe_peaks &pk)
{
    Terms t;
    t.bytes = w.bytes;
    t.t_mem = w.bytes / (pk.hbm_gbs * 1e9);
    // the busiest pipe, expressed as FP32 FMAs (the FMA pipe itself unscaled)
    double eq = w.ffma;
    if (w.imul > 0 && pk.imul_per_s > 0) eq = std::max(eq, w.imul * (pk.ffma_per_s / pk.imul_per_s));
    if (w.smem_atomic > 0 && pk.smem_atomic_per_s > 0)
        eq = std::max(eq, w.smem_atomic * (pk.ffma_per_s / pk.smem_atomic_per_s));
    if (w.ialu > 0 && pk.ialu_per_s > 0) eq = std::max(eq, w.ialu * (pk.ffma_per_s / pk.ialu_per_s));
    t.fma_equiv = eq;
    t.t_c = eq / pk.ffma_per_s;
    return t;
}

} // namespace

extern "C" hf_status hf_body_work_of(int body, const void *args, hf_body_work *out)
{
    if (!args || !out) return hf::set_last_error(HF_ERR_INVALID, "NULL argument");
    if (body < 0 || body >= HF_BODY_COUNT) return hf::set_last_error(HF_ERR_INVALID, "unknown body");
    hf_body_work w{};
    w.barriers = hf::body_barriers(body);
    switch (body) {
    case HF_BODY_BN_STATS: {
        const auto &a = *static_cast<const hf_bn_stats_args *>(args);
        const double n = (double)a.N * a.C * a.HW;
        w.bytes = 4.0 * n + 8.0 * a.C;
        w.ffma = 2.0 * n;   // shifted sum and sum of squares
        break;
    }
    case HF_BODY_UPSAMPLE2X: {
        const auto &a = *static_cast<const hf_upsample2x_args *>(args);
        const double n = (double)a.P * a.H * a.W;
        w.bytes = 4.0 * n + 16.0 * n;
        w.ffma = 16.0 * n;   // two blends (multiply + FMA) per output, four outputs per input
        break;
    }
    case HF_BODY_MAXPOOL3S2: {
        const auto &a = *static_cast<const hf_maxpool3s2_args *>(args);
        const double n = (double)a.P * a.H * a.W;
        const double o = (double)a.P * ((a.H - 1) / 2 + 1) * ((a.W - 1) / 2 + 1);
        w.bytes = 4.0 * n + 4.0 * o;
        w.ffma = 8.0 * o;   // eight comparisons per output
        break;
    }
    case HF_BODY_IM2COL3: {
        const auto &a = *static_cast<const hf_im2col3_args *>(args);
        const double n = (double)a.N * a.C * a.H * a.W;
        w.bytes = 4.0 * n + 36.0 * n;
        break;
    }
    case HF_BODY_HIST256: {
        const auto &a = *static_cast<const hf_hist256_args *>(args);
        w.bytes = (double)a.n + 1024.0;
        w.smem_atomic = (double)a.n;
        break;
    }
    case HF_BODY_PHILOX: {
        const auto &a = *static_cast<const hf_philox_args *>(args);
        w.bytes = 16.0 * (double)a.n;
        w.imul = 40.0 * (double)a.n;   // 10 rounds x 2 products x (high + low half)
        break;
    }
    case HF_BODY_POLY: {
        const auto &a = *static_cast<const hf_poly_args *>(args);
        w.bytes = 8.0 * (double)a.n;
        w.ffma = (double)a.n * a.iters * HF_POLY_NCOEF;
        break;
    }
    case HF_BODY_BF16_AXPY: {
        const auto &a = *static_cast<const hf_bf16_axpy_args *>(args);
        w.bytes = 6.0 * (double)a.n;
        w.ffma = (double)a.n;
        break;
    }
    case HF_BODY_STREAM_TMPL: {
        const auto &a = *static_cast<const hf_stream_tmpl_args *>(args);
        w.bytes = 8.0 * (double)a.n;
        w.ffma = (double)a.k * (double)a.n / 4.0;
        w.barriers = a.n_barriers;
        break;
    }
    case HF_BODY_SHA256D:
    case HF_BODY_BLAKE256:
    case HF_BODY_BLAKE2B: {
        const auto &a = *static_cast<const hf_hash_scan_args *>(args);
        const double per = body == HF_BODY_SHA256D ? kOpsSha256d
                           : body == HF_BODY_BLAKE256 ? kOpsBlake256 : kOpsBlake2b;
        w.bytes = 0.0;
        w.ialu = per * (double)a.n;
        break;
    }
    default: break;
    }
    *out = w;
    return HF_OK;
}

extern "C" hf_status hf_pair_features(hf_kernel ka, hf_kernel kb, const void *const *args, int split,
                                      int d0, int regcap, int blocks_per_sm, int fused_regs,
                                      int spill_bytes, const hf_pipe_peaks *pk, float *out)
{
    if (!ka || !kb || !args || !args[0] || !args[1] || !pk || !out || split <= 0 || split >= d0 ||
        blocks_per_sm < 1 || pk->hbm_gbs <= 0 || pk->ffma_per_s <= 0)
        return hf::set_last_error(HF_ERR_INVALID, "bad feature arguments");
    const int id[2] = {hf::kernel_body_id(ka), hf::kernel_body_id(kb)};
    const int thr[2] = {split, d0 - split};
    Terms t[2];
    int bar[2];
    double smem[2];
    for (int i = 0; i < 2; ++i) {
        hf_body_work w;
        hf_status s = hf_body_work_of(id[i], args[i], &w);
        if (s) return s;
        t[i] = terms_of(w, *pk);
        bar[i] = w.barriers;
    }
    // each interval's shared memory as launched: slice + bulk-copy ring
    hf::interval_smem_at(id, args, thr, blocks_per_sm, smem);
    double est[2], comp[2];
    for (int i = 0; i < 2; ++i) {
        est[i] = std::max(t[i].t_mem, t[i].t_c) * 1e6;
        comp[i] = t[i].t_c / std::max(t[i].t_mem + t[i].t_c, 1e-30);
    }
    const double tot = est[0] + est[1];
    int f = 0;
    for (int i = 0; i < 2; ++i) {
        const double n = t[i].bytes / 8.0;
        const double k = t[i].fma_equiv * 32.0 / std::max(t[i].bytes, 32.0);
        out[f++] = (float)(std::log2(std::max(n, 1.0)) / 28.0);
        out[f++] = (float)(std::log2(1.0 + k) / 8.0);
        out[f++] = (float)(bar[i] / 4.0);
        out[f++] = (float)(smem[i] / 49152.0);
        out[f++] = (float)(std::log2(1.0 + est[i]) / 12.0);
        out[f++] = (float)comp[i];
        out[f++] = (float)((double)thr[i] / d0);
        out[f++] = (float)(thr[i] / 32.0 * blocks_per_sm / 64.0);
        out[f++] = (float)(est[i] / std::max(tot, 1e-30));
    }
    out[f++] = (float)((regcap ? regcap : 255) / 255.0);
    out[f++] = (float)(blocks_per_sm / 4.0);
    out[f++] = (float)(blocks_per_sm * (double)d0 / 2048.0);
    out[f++] = (float)(fused_regs / 255.0);
    out[f++] = (float)(std::log2(1.0 + spill_bytes) / 10.0);
    out[f++] = (float)((smem[0] + smem[1]) * blocks_per_sm / 233472.0);
    return HF_OK;
}
