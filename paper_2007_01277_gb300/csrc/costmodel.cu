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
