/*
 * hf_oracle.c -- plain CPU oracle for the horizontal-fusion hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this code.  The product path
 * (the CUDA library and its Python binding) never calls it and shares no
 * code, header, table or constant with it.
 *
 * What is computed here.  Horizontal fusion (Sec. 1.1, Sec. 3.1) produces a
 * kernel that is functionally equivalent to the kernels it fuses, so the
 * oracle of a fused launch is simply the plain definition of every
 * constituent kernel, evaluated independently.  Floating point work is done
 * in double precision from the float32 inputs; integer and copy work is
 * exact.  Loops are the textbook ones: no blocking, no reordering.
 *
 * Constituents (Sec. 4.1 names the deep-learning ones; the rest are the
 * project's own workload kernels):
 *   or_bn_stats       per-channel mean and biased variance (two passes)
 *   or_upsample2x     bilinear x2 upsampling, half-pixel centres
 *   or_maxpool3s2p1   3x3 stride-2 pad-1 max pooling
 *   or_im2col3        3x3 stride-1 pad-1 patch-to-column rearrangement
 *   or_hist256        256-bin histogram of bytes
 *   or_philox4x32_10  Philox4x32-10 counter-based generator
 *                     (Salmon, Moraes, Dror, Shaw, SC'11)
 *   or_poly           64-step repeated degree-32 Horner recurrence
 *   or_bf16_axpy      out = bf16_rne(alpha*x + y)
 *   or_stream_tmpl    affine FMA chain applied per 16-byte group
 *   or_mlp_*          3-layer perceptron forward/backward and Adam step
 *                     (Kingma & Ba, ICLR 2015)
 *   or_register_bound the register bound of Algorithm 2 (Sec. 3.2)
 *   or_blocks_per_sm  the resident-block count of Sec. 2.1
 *
 * Every function is pinned by tests outside this file against closed forms,
 * hand-worked grids, library routines or the paper's worked numbers.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Batch-norm statistics (Sec. 2.3, the batch_norm_collect_statistics kernel;
 * Sec. 4.1 "Batchnorm collects the batch mean and variance").
 * x is NCHW float32; channel c holds M = N*HW values.  mean_c = sum x / M,
 * var_c = sum (x - mean_c)^2 / M (biased), both in double, two passes.     */
void or_bn_stats(const float *x, int N, int C, int HW, double *mean,
                 double *var)
{
    for (int c = 0; c < C; ++c) {
        double s = 0.0;
        for (int n = 0; n < N; ++n)
            for (int i = 0; i < HW; ++i)
                s += (double)x[((long)n * C + c) * HW + i];
        double M = (double)N * (double)HW;
        double m = s / M;
        double q = 0.0;
        for (int n = 0; n < N; ++n)
            for (int i = 0; i < HW; ++i) {
                double d = (double)x[((long)n * C + c) * HW + i] - m;
                q += d * d;
            }
        mean[c] = m;
        var[c] = q / M;
    }
}

/* ------------------------------------------------------------------------ */
/* Bilinear upsampling by 2 with half-pixel centres (align_corners = false),
 * the Upsample kernel of Sec. 4.1.  For output coordinate o on an axis of
 * input length L: src = max(0, (o + 0.5) * L / (2L) - 0.5), i0 = floor(src),
 * i1 = min(i0 + 1, L - 1), lambda = src - i0, and the value is
 * (1-ly)[(1-lx) a + lx b] + ly[(1-lx) c + lx d].  P planes of H x W.     */
void or_upsample2x(const float *in, int P, int H, int W, double *out)
{
    int Ho = 2 * H, Wo = 2 * W;
    for (int p = 0; p < P; ++p) {
        const float *src = in + (long)p * H * W;
        double *dst = out + (long)p * Ho * Wo;
        for (int oy = 0; oy < Ho; ++oy) {
            double sy = ((double)oy + 0.5) * ((double)H / (double)Ho) - 0.5;
            if (sy < 0.0) sy = 0.0;
            int y0 = (int)floor(sy);
            int y1 = y0 + 1 < H ? y0 + 1 : H - 1;
            double ly = sy - (double)y0;
            for (int ox = 0; ox < Wo; ++ox) {
                double sx = ((double)ox + 0.5) * ((double)W / (double)Wo) - 0.5;
                if (sx < 0.0) sx = 0.0;
                int x0 = (int)floor(sx);
                int x1 = x0 + 1 < W ? x0 + 1 : W - 1;
                double lx = sx - (double)x0;
                double a = src[(long)y0 * W + x0], b = src[(long)y0 * W + x1];
                double c = src[(long)y1 * W + x0], d = src[(long)y1 * W + x1];
                dst[(long)oy * Wo + ox] =
                    (1.0 - ly) * ((1.0 - lx) * a + lx * b) +
                    ly * ((1.0 - lx) * c + lx * d);
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* 3x3 max pooling, stride 2, padding 1 (Sec. 4.1 "Maxpool applies a 2D
 * maxpooling").  Padding never wins: the maximum is over the in-bounds part
 * of the window.  Ho = (H + 2 - 3) / 2 + 1, likewise Wo.  Exact.          */
void or_maxpool3s2p1(const float *in, int P, int H, int W, float *out)
{
    int Ho = (H - 1) / 2 + 1, Wo = (W - 1) / 2 + 1;
    for (int p = 0; p < P; ++p)
        for (int oy = 0; oy < Ho; ++oy)
            for (int ox = 0; ox < Wo; ++ox) {
                float m = -INFINITY;
                for (int ky = 0; ky < 3; ++ky)
                    for (int kx = 0; kx < 3; ++kx) {
                        int iy = 2 * oy - 1 + ky, ix = 2 * ox - 1 + kx;
                        if (iy < 0 || iy >= H || ix < 0 || ix >= W) continue;
                        float v = in[((long)p * H + iy) * W + ix];
                        if (v > m) m = v;
                    }
                out[((long)p * Ho + oy) * Wo + ox] = m;
            }
}

/* ------------------------------------------------------------------------ */
/* im2col for a 3x3 window, stride 1, padding 1 (Sec. 4.1 "Im2Col rearranges
 * the input image blocks into columns").  Output row r = c*9 + ky*3 + kx of
 * image n has H*W columns; column oy*W + ox holds x[n][c][oy+ky-1][ox+kx-1]
 * or 0 outside the image.  Exact copy.                                    */
void or_im2col3(const float *in, int N, int C, int H, int W, float *out)
{
    long cols = (long)H * W;
    for (int n = 0; n < N; ++n)
        for (int c = 0; c < C; ++c)
            for (int ky = 0; ky < 3; ++ky)
                for (int kx = 0; kx < 3; ++kx) {
                    long row = ((long)n * C * 9) + c * 9 + ky * 3 + kx;
                    for (int oy = 0; oy < H; ++oy)
                        for (int ox = 0; ox < W; ++ox) {
                            int iy = oy + ky - 1, ix = ox + kx - 1;
                            float v = 0.0f;
                            if (iy >= 0 && iy < H && ix >= 0 && ix < W)
                                v = in[(((long)n * C + c) * H + iy) * W + ix];
                            out[row * cols + (long)oy * W + ox] = v;
                        }
                }
}

/* ------------------------------------------------------------------------ */
/* Histogram with 256 bins over bytes (Sec. 2.3, the kernelHistogram1D
 * kernel, specialised to one bin per byte value).  bins are overwritten.  */
void or_hist256(const uint8_t *x, long n, uint32_t *bins)
{
    for (int b = 0; b < 256; ++b) bins[b] = 0;
    for (long i = 0; i < n; ++i) bins[x[i]] += 1u;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 4.2 of that paper).  One round
 * maps counter (x0,x1,x2,x3) under round key (k0,k1) to
 *   (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0))
 * and the key is bumped by the Weyl constants (W0,W1) between rounds.
 * Output i is the block for counter (lo32(first+i), hi32(first+i), 0, 0)
 * under key (lo32(seed), hi32(seed)); out holds 4 words per output.       */
static const uint32_t OR_PHILOX_M0 = 0xD2511F53u;
static const uint32_t OR_PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t OR_PHILOX_W0 = 0x9E3779B9u; /* floor(2^32 (sqrt5-1)/2) */
static const uint32_t OR_PHILOX_W1 = 0xBB67AE85u; /* floor(2^32 (sqrt3-1))   */

void or_philox_round(uint32_t ctr[4], const uint32_t key[2])
{
    uint64_t p0 = (uint64_t)OR_PHILOX_M0 * (uint64_t)ctr[0];
    uint64_t p1 = (uint64_t)OR_PHILOX_M1 * (uint64_t)ctr[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ ctr[1] ^ key[0];
    uint32_t y2 = hi0 ^ ctr[3] ^ key[1];
    ctr[0] = y0;
    ctr[1] = lo1;
    ctr[2] = y2;
    ctr[3] = lo0;
}

void or_philox4x32_10(uint64_t seed, uint64_t first, long n, uint32_t *out)
{
    for (long i = 0; i < n; ++i) {
        uint64_t c = first + (uint64_t)i;
        uint32_t ctr[4] = {(uint32_t)c, (uint32_t)(c >> 32), 0u, 0u};
        uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        for (int r = 0; r < 10; ++r) {
            if (r > 0) {
                key[0] += OR_PHILOX_W0;
                key[1] += OR_PHILOX_W1;
            }
            or_philox_round(ctr, key);
        }
        memcpy(out + 4 * i, ctr, sizeof ctr);
    }
}

/* ------------------------------------------------------------------------ */
/* FMA-chain polynomial.  c[0..32] are the coefficients of
 * p(x) = sum_k c_k x^k (degree 32).  acc_0 = 0 and each of `iters` steps runs
 * one Horner evaluation seeded with the running value:
 *   h = acc; for k = 32 .. 0: h = h*x + c_k; acc = h,
 * i.e. acc_{t+1} = acc_t x^33 + p(x): 33 multiply-adds per step.
 * bound[i] (optional) receives the Horner conditioning scale
 * sum_t sum_k |c_k| |x|^(k + 33 t) that the tolerance is measured against. */
void or_poly(const float *x, long n, const float *c, int iters, double *out,
             double *bound)
{
    for (long i = 0; i < n; ++i) {
        double xv = (double)x[i];
        double acc = 0.0;
        for (int t = 0; t < iters; ++t) {
            double h = acc;
            for (int k = 32; k >= 0; --k) h = h * xv + (double)c[k];
            acc = h;
        }
        out[i] = acc;
        if (bound) {
            double ax = fabs(xv), pa = 0.0, geo = 0.0;
            for (int k = 32; k >= 0; --k) pa = pa * ax + fabs((double)c[k]);
            double x33 = pow(ax, 33.0), term = 1.0;
            for (int t = 0; t < iters; ++t) {
                geo += term;
                term *= x33;
            }
            bound[i] = pa * geo;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* bfloat16 helpers: a bf16 is the top 16 bits of an IEEE binary32.        */
static double or_bf16_to_double(uint16_t h)
{
    uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, sizeof f);
    return (double)f;
}

/* Round a double to the nearest bfloat16, ties to even, by exact integer
 * arithmetic on the significand (no intermediate float rounding).         */
uint16_t or_double_to_bf16(double v)
{
    if (isnan(v)) return (uint16_t)0x7FC0u;
    uint16_t sign = signbit(v) ? 0x8000u : 0u;
    double a = fabs(v);
    if (a == 0.0) return sign;
    if (isinf(a)) return (uint16_t)(sign | 0x7F80u);
    int e;
    double m = frexp(a, &e);           /* a = m * 2^e, m in [0.5, 1)     */
    int be = e - 1;                    /* a = (2m) * 2^be, 2m in [1, 2)  */
    if (be < -126) {
        /* subnormal: value = q * 2^-133, q < 128 */
        double q = ldexp(a, 133);
        double r = nearbyint(q);       /* default mode: ties to even     */
        return (uint16_t)(sign | (uint16_t)r);
    }
    double q = ldexp(2.0 * m, 7);      /* in [128, 256): 8 significant bits */
    double r = nearbyint(q);
    if (r == 256.0) {
        r = 128.0;
        be += 1;
    }
    if (be > 127) return (uint16_t)(sign | 0x7F80u);
    uint32_t mant = (uint32_t)r - 128u;
    return (uint16_t)(sign | ((uint32_t)(be + 127) << 7) | mant);
}

/* out_i = bf16_rne(alpha * x_i + y_i), evaluated exactly in double.       */
void or_bf16_axpy(const uint16_t *x, const uint16_t *y, double alpha, long n,
                  uint16_t *out)
{
    for (long i = 0; i < n; ++i)
        out[i] = or_double_to_bf16(alpha * or_bf16_to_double(x[i]) +
                                   or_bf16_to_double(y[i]));
}

/* ------------------------------------------------------------------------ */
/* Parametric stream template.  For every 16-byte group (4 floats) of the
 * input, k multiply-adds v <- v*a + b are applied, the j-th one (j = 0..k-1)
 * to component j mod 4; the group is then stored.  n is a multiple of 4.  */
void or_stream_tmpl(const float *in, long n, int k, float a, float b,
                    double *out)
{
    for (long g = 0; g < n / 4; ++g) {
        double v[4];
        for (int j = 0; j < 4; ++j) v[j] = (double)in[4 * g + j];
        for (int j = 0; j < k; ++j) v[j % 4] = v[j % 4] * (double)a + (double)b;
        for (int j = 0; j < 4; ++j) out[4 * g + j] = v[j];
    }
}

/* ------------------------------------------------------------------------ */
/* Three-layer perceptron 24 -> 64 -> ReLU -> 64 -> ReLU -> 1 on a batch of
 * B rows.  Parameters in one flat array, row-major:
 *   W1[64][24], b1[64], W2[64][64], b2[64], w3[64], b3[1]   (5825 values).
 * Loss = mean over the batch of (yhat - y)^2.                              */
#define OR_MLP_IN 24
#define OR_MLP_H 64
#define OR_MLP_NPARAM (OR_MLP_H * OR_MLP_IN + OR_MLP_H + OR_MLP_H * OR_MLP_H + \
                       OR_MLP_H + OR_MLP_H + 1)

int or_mlp_nparam(void) { return OR_MLP_NPARAM; }

static void or_mlp_row(const double *P, const double *xin, double *h1,
                       double *h2, double *yhat)
{
    const double *W1 = P, *b1 = W1 + OR_MLP_H * OR_MLP_IN;
    const double *W2 = b1 + OR_MLP_H, *b2 = W2 + OR_MLP_H * OR_MLP_H;
    const double *w3 = b2 + OR_MLP_H, *b3 = w3 + OR_MLP_H;
    for (int j = 0; j < OR_MLP_H; ++j) {
        double s = b1[j];
        for (int i = 0; i < OR_MLP_IN; ++i) s += W1[j * OR_MLP_IN + i] * xin[i];
        h1[j] = s > 0.0 ? s : 0.0;
    }
    for (int j = 0; j < OR_MLP_H; ++j) {
        double s = b2[j];
        for (int i = 0; i < OR_MLP_H; ++i) s += W2[j * OR_MLP_H + i] * h1[i];
        h2[j] = s > 0.0 ? s : 0.0;
    }
    double s = b3[0];
    for (int i = 0; i < OR_MLP_H; ++i) s += w3[i] * h2[i];
    *yhat = s;
}

void or_mlp_forward(const double *P, const float *X, int B, double *yhat)
{
    double xin[OR_MLP_IN], h1[OR_MLP_H], h2[OR_MLP_H];
    for (int r = 0; r < B; ++r) {
        for (int i = 0; i < OR_MLP_IN; ++i) xin[i] = X[(long)r * OR_MLP_IN + i];
        or_mlp_row(P, xin, h1, h2, &yhat[r]);
    }
}

/* Loss and its gradient with respect to all parameters (backpropagation of
 * the mean squared error).  Returns the loss; grad has OR_MLP_NPARAM slots. */
double or_mlp_loss_grad(const double *P, const float *X, const float *Y, int B,
                        double *grad)
{
    const double *W2 = P + OR_MLP_H * OR_MLP_IN + OR_MLP_H;
    const double *w3 = W2 + OR_MLP_H * OR_MLP_H + OR_MLP_H;
    double *gW1 = grad, *gb1 = gW1 + OR_MLP_H * OR_MLP_IN;
    double *gW2 = gb1 + OR_MLP_H, *gb2 = gW2 + OR_MLP_H * OR_MLP_H;
    double *gw3 = gb2 + OR_MLP_H, *gb3 = gw3 + OR_MLP_H;
    for (int i = 0; i < OR_MLP_NPARAM; ++i) grad[i] = 0.0;
    double xin[OR_MLP_IN], h1[OR_MLP_H], h2[OR_MLP_H], d2[OR_MLP_H],
        d1[OR_MLP_H], yhat, loss = 0.0;
    for (int r = 0; r < B; ++r) {
        for (int i = 0; i < OR_MLP_IN; ++i) xin[i] = X[(long)r * OR_MLP_IN + i];
        or_mlp_row(P, xin, h1, h2, &yhat);
        double e = yhat - (double)Y[r];
        loss += e * e / B;
        double dy = 2.0 * e / B;
        gb3[0] += dy;
        for (int i = 0; i < OR_MLP_H; ++i) {
            gw3[i] += dy * h2[i];
            d2[i] = h2[i] > 0.0 ? dy * w3[i] : 0.0;
        }
        for (int j = 0; j < OR_MLP_H; ++j) {
            gb2[j] += d2[j];
            for (int i = 0; i < OR_MLP_H; ++i) gW2[j * OR_MLP_H + i] += d2[j] * h1[i];
        }
        for (int i = 0; i < OR_MLP_H; ++i) {
            double s = 0.0;
            for (int j = 0; j < OR_MLP_H; ++j) s += W2[j * OR_MLP_H + i] * d2[j];
            d1[i] = h1[i] > 0.0 ? s : 0.0;
        }
        for (int j = 0; j < OR_MLP_H; ++j) {
            gb1[j] += d1[j];
            for (int i = 0; i < OR_MLP_IN; ++i) gW1[j * OR_MLP_IN + i] += d1[j] * xin[i];
        }
    }
    return loss;
}

/* One Adam step (Kingma & Ba, Algorithm 1) at step number t >= 1.          */
void or_adam_step(double *P, const double *g, double *m, double *v, int n,
                  int t, double lr, double beta1, double beta2, double eps)
{
    double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
    for (int i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        P[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* ------------------------------------------------------------------------ */
/* Resident blocks per SM (Sec. 2.1): the minimum of the register, shared
 * memory and thread limits, each a floor division.                         */
int or_blocks_per_sm(int sm_regs, int sm_smem, int sm_threads, int threads,
                     int regs_per_thread, int smem_per_block)
{
    int b = sm_threads / threads;
    if (regs_per_thread > 0) {
        int br = sm_regs / (threads * regs_per_thread);
        if (br < b) b = br;
    }
    if (smem_per_block > 0) {
        int bs = sm_smem / smem_per_block;
        if (bs < b) b = bs;
    }
    return b;
}

/* The register bound of Algorithm 2 (Sec. 3.2):
 *   b1 = SMNRegs / (d1 NRegs(S1)), b2 = SMNRegs / (d2 NRegs(S2)),
 *   b0 = min(b1, b2, SMShMem / ShMem(F), SMNThreads / d0),
 *   r0 = SMNRegs / (b0 d0),
 * with floor divisions; a zero ShMem(F) drops that term.  Returns r0, or 0
 * when b0 is 0 (the fused block does not fit).                             */
int or_register_bound(int sm_regs, int sm_smem, int sm_threads, int d1,
                      int nregs1, int d2, int nregs2, int smem_fused)
{
    int d0 = d1 + d2;
    int b1 = sm_regs / (d1 * nregs1);
    int b2 = sm_regs / (d2 * nregs2);
    int b0 = b1 < b2 ? b1 : b2;
    if (smem_fused > 0) {
        int bs = sm_smem / smem_fused;
        if (bs < b0) b0 = bs;
    }
    int bt = sm_threads / d0;
    if (bt < b0) b0 = bt;
    if (b0 <= 0) return 0;
    return sm_regs / (b0 * d0);
}
