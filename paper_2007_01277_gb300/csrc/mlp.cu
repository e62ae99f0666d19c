// mlp.cu -- the learned cost model's kernels: a 24 -> 64 -> ReLU -> 64 ->
// ReLU -> 1 perceptron in FP32 on the CUDA cores (it is far too small for
// the tensor cores to pay off).
//
// Parameters are one flat FP32 array, row-major:
//   W1[64][24] @0, b1[64] @1536, W2[64][64] @1600, b2[64] @5696,
//   w3[64] @5760, b3 @5824                                  (5825 values)
//
// k_mlp_forward scores samples grid-wide: one warp per sample, lane j owns
// hidden units j and j+32, the first layer's weights sit in registers, the
// second layer's (transposed) in shared memory, and the output is a warp
// butterfly sum.
//
// k_mlp_train runs a whole training run in ONE persistent block: for each
// step it gathers a minibatch (rows idx[step*B .. step*B+B)), runs the
// forward pass, back-propagates the mean squared error, and applies Adam
// (Kingma & Ba) to parameters held in shared memory.  Every activation and
// gradient lives in shared memory with padded rows (stride 65 / 25) so that
// lanes that walk samples hit distinct banks; every sum has a fixed order,
// so a run is deterministic.
#include <cmath>

#include "kernels.cuh"

namespace hf {
hf_status set_last_error(hf_status s, const char *msg);   // runtime.cu
}

namespace {

constexpr int IN = 24, HD = 64, NP = 5825;
constexpr int OW1 = 0, OB1 = 1536, OW2 = 1600, OB2 = 5696, OW3 = 5760, OB3 = 5824;
constexpr int kMaxBatch = 64;
constexpr int kTrainThreads = 512;
constexpr int SX = IN + 1, SH = HD + 1;   // padded row strides

__global__ void __launch_bounds__(256) k_mlp_forward(const float *__restrict__ P,
                                                     const float *__restrict__ X, int n,
                                                     float *__restrict__ y)
{
    __shared__ float w2t[HD][HD];   // w2t[i][j] = W2[j][i]
    __shared__ float b2s[HD], w3s[HD];
    for (int e = threadIdx.x; e < HD * HD; e += blockDim.x) {
        const int j = e / HD, i = e % HD;
        w2t[i][j] = P[OW2 + e];
    }
    for (int j = threadIdx.x; j < HD; j += blockDim.x) {
        b2s[j] = P[OB2 + j];
        w3s[j] = P[OW3 + j];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    float w1a[IN], w1b[IN];
#pragma unroll
    for (int k = 0; k < IN; ++k) {
        w1a[k] = P[OW1 + lane * IN + k];
        w1b[k] = P[OW1 + (lane + 32) * IN + k];
    }
    const float b1a = P[OB1 + lane], b1b = P[OB1 + lane + 32], b3 = P[OB3];
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < n; s += warps) {
        const float *xs = X + (int64_t)s * IN;
        float a0 = b1a, a1 = b1b;
#pragma unroll
        for (int k = 0; k < IN; ++k) {
            const float xk = __ldg(xs + k);
            a0 = __fmaf_rn(w1a[k], xk, a0);
            a1 = __fmaf_rn(w1b[k], xk, a1);
        }
        const float ha = fmaxf(a0, 0.f), hb = fmaxf(a1, 0.f);
        float c0 = b2s[lane], c1 = b2s[lane + 32];
#pragma unroll
        for (int i = 0; i < HD; ++i) {
            const float hi = __shfl_sync(0xffffffffu, i < 32 ? ha : hb, i & 31);
            c0 = __fmaf_rn(w2t[i][lane], hi, c0);
            c1 = __fmaf_rn(w2t[i][lane + 32], hi, c1);
        }
        float o = __fmaf_rn(w3s[lane], fmaxf(c0, 0.f), w3s[lane + 32] * fmaxf(c1, 0.f));
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) o += __shfl_xor_sync(0xffffffffu, o, m);
        if (lane == 0) y[s] = o + b3;
    }
}

struct TrainSmem {
    float P[NP], M[NP], V[NP], G[NP];
    float X[kMaxBatch * SX];
    float H1[kMaxBatch * SH];
    float H2[kMaxBatch * SH];   // becomes D2 after the output layer's gradient
    float D1[kMaxBatch * SH];
    float Y[kMaxBatch], dY[kMaxBatch];
};

__global__ void __launch_bounds__(kTrainThreads) k_mlp_train(
    float *__restrict__ Pg, float *__restrict__ Mg, float *__restrict__ Vg,
    const float *__restrict__ X, const float *__restrict__ Y, const int *__restrict__ idx,
    int steps, int B, float lr, float beta1, float beta2, float eps, int t0,
    float *__restrict__ loss_out, float *__restrict__ grad_out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem &S = *reinterpret_cast<TrainSmem *>(smem_raw);
    const int tid = threadIdx.x, T = blockDim.x;
    for (int p = tid; p < NP; p += T) {
        S.P[p] = Pg[p];
        S.M[p] = Mg[p];
        S.V[p] = Vg[p];
    }
    __syncthreads();
    const float invB = 1.0f / (float)B;
    for (int step = 0; step < steps; ++step) {
        // gather the minibatch
        const int *rows = idx + (int64_t)step * B;
        for (int e = tid; e < B * IN; e += T) {
            const int s = e / IN, k = e % IN;
            S.X[s * SX + k] = X[(int64_t)rows[s] * IN + k];
        }
        for (int s = tid; s < B; s += T) S.Y[s] = Y[rows[s]];
        __syncthreads();
        // H1 = relu(X W1^T + b1); lanes walk samples
        for (int o = tid; o < B * HD; o += T) {
            const int j = o / B, s = o % B;
            float a = S.P[OB1 + j];
            for (int k = 0; k < IN; ++k) a = __fmaf_rn(S.P[OW1 + j * IN + k], S.X[s * SX + k], a);
            S.H1[s * SH + j] = fmaxf(a, 0.f);
        }
        __syncthreads();
        // H2 = relu(H1 W2^T + b2)
        for (int o = tid; o < B * HD; o += T) {
            const int j = o / B, s = o % B;
            float a = S.P[OB2 + j];
            for (int i = 0; i < HD; ++i) a = __fmaf_rn(S.P[OW2 + j * HD + i], S.H1[s * SH + i], a);
            S.H2[s * SH + j] = fmaxf(a, 0.f);
        }
        __syncthreads();
        // output, error and dL/dy (mean squared error)
        for (int s = tid; s < B; s += T) {
            float a = S.P[OB3];
            for (int j = 0; j < HD; ++j) a = __fmaf_rn(S.P[OW3 + j], S.H2[s * SH + j], a);
            const float e = a - S.Y[s];
            S.dY[s] = 2.f * e * invB;
            S.D1[s] = e * e;   // scratch for the loss
        }
        __syncthreads();
        if (tid == 0 && loss_out) {
            float l = 0.f;
            for (int s = 0; s < B; ++s) l += S.D1[s];
            loss_out[step] = l * invB;
        }
        // gradients of the output layer
        for (int j = tid; j <= HD; j += T) {
            float g = 0.f;
            if (j < HD)
                for (int s = 0; s < B; ++s) g = __fmaf_rn(S.dY[s], S.H2[s * SH + j], g);
            else
                for (int s = 0; s < B; ++s) g += S.dY[s];
            S.G[j < HD ? OW3 + j : OB3] = g;
        }
        __syncthreads();
        // D2 = dY w3^T masked by the ReLU, in place of H2
        for (int o = tid; o < B * HD; o += T) {
            const int j = o / B, s = o % B;
            const float h = S.H2[s * SH + j];
            S.H2[s * SH + j] = h > 0.f ? S.dY[s] * S.P[OW3 + j] : 0.f;
        }
        __syncthreads();
        // gW2[j][i] = sum_s D2[s][j] H1[s][i]; gb2[j] = sum_s D2[s][j]
        for (int o = tid; o < HD * HD; o += T) {
            const int j = o / HD, i = o % HD;
            float g = 0.f;
            for (int s = 0; s < B; ++s) g = __fmaf_rn(S.H2[s * SH + j], S.H1[s * SH + i], g);
            S.G[OW2 + o] = g;
        }
        for (int j = tid; j < HD; j += T) {
            float g = 0.f;
            for (int s = 0; s < B; ++s) g += S.H2[s * SH + j];
            S.G[OB2 + j] = g;
        }
        // D1[s][i] = (sum_j D2[s][j] W2[j][i]) masked by the ReLU
        for (int o = tid; o < B * HD; o += T) {
            const int i = o / B, s = o % B;
            float a = 0.f;
            for (int j = 0; j < HD; ++j) a = __fmaf_rn(S.H2[s * SH + j], S.P[OW2 + j * HD + i], a);
            S.D1[s * SH + i] = S.H1[s * SH + i] > 0.f ? a : 0.f;
        }
        __syncthreads();
        // gW1[j][k] = sum_s D1[s][j] X[s][k]; gb1[j] = sum_s D1[s][j]
        for (int o = tid; o < HD * IN; o += T) {
            const int j = o / IN, k = o % IN;
            float g = 0.f;
            for (int s = 0; s < B; ++s) g = __fmaf_rn(S.D1[s * SH + j], S.X[s * SX + k], g);
            S.G[OW1 + o] = g;
        }
        for (int j = tid; j < HD; j += T) {
            float g = 0.f;
            for (int s = 0; s < B; ++s) g += S.D1[s * SH + j];
            S.G[OB1 + j] = g;
        }
        __syncthreads();
        if (grad_out && step == 0)
            for (int p = tid; p < NP; p += T) grad_out[p] = S.G[p];
        // Adam
        const int t = t0 + step + 1;
        const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
        for (int p = tid; p < NP; p += T) {
            const float g = S.G[p];
            const float m = beta1 * S.M[p] + (1.f - beta1) * g;
            const float v = beta2 * S.V[p] + (1.f - beta2) * g * g;
            S.M[p] = m;
            S.V[p] = v;
            S.P[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
        }
        __syncthreads();
    }
    for (int p = tid; p < NP; p += T) {
        Pg[p] = S.P[p];
        Mg[p] = S.M[p];
        Vg[p] = S.V[p];
    }
}

} // namespace

extern "C" {

hf_status hf_mlp_forward(const float *params, const float *X, int n, float *y, void *stream)
{
    if (n < 0 || (n > 0 && (!params || !X || !y))) return hf::set_last_error(HF_ERR_INVALID, "bad MLP forward arguments");
    if (n == 0) return HF_OK;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = std::min((n + 7) / 8, 4 * sms);   // 8 warps per block
    k_mlp_forward<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, X, n, y);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HF_OK : hf::set_last_error(HF_ERR_CUDA, cudaGetErrorString(e));
}

hf_status hf_mlp_train(float *params, float *adam_m, float *adam_v, const float *X, const float *Y,
                       const int *idx, int steps, int batch, float lr, float beta1, float beta2,
                       float eps, int t0, float *loss_out, float *grad_out, void *stream)
{
    if (!params || !adam_m || !adam_v || !X || !Y || !idx || steps < 0 || batch < 1 ||
        batch > kMaxBatch || t0 < 0)
        return hf::set_last_error(HF_ERR_INVALID, "bad MLP training arguments (batch 1..64)");
    if (steps == 0) return HF_OK;
    const size_t smem = sizeof(TrainSmem);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return hf::set_last_error(HF_ERR_CUDA, cudaGetErrorString(e));
    k_mlp_train<<<1, kTrainThreads, smem, static_cast<cudaStream_t>(stream)>>>(
        params, adam_m, adam_v, X, Y, idx, steps, batch, lr, beta1, beta2, eps, t0, loss_out, grad_out);
    e = cudaGetLastError();
    return e == cudaSuccess ? HF_OK : hf::set_last_error(HF_ERR_CUDA, cudaGetErrorString(e));
}

int hf_mlp_nparams(void) { return NP; }

} // extern "C"
