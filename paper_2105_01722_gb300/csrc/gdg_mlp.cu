// Learned initial guess for the element u_t solve: a three-layer perceptron
// (162 -> 64 -> 64 -> 81, tanh) with BF16 weights and FP32 accumulation,
// and its training kernels (a pattern layered on the element PCG of
// Section 7.1; the paper has no learned component).
//
// Parameter block (FP32 master copy, in this order):
//   W1 [64][162], b1 [64], W2 [64][64], b2 [64], W3 [81][64], b3 [81]
// BF16 working weights: W1, W2, W3 in the same order (biases stay FP32).
// Features of an element (162 FP32): c^2 / mean(c^2) at the 81 nodes, then
// r_u / ||r_u||; output: a guess of y / ||r_u|| for (S_c2 + w w^T) y = r_u.
//
// Kernels
//   k_mlp_forward   Y = net(X) for B samples (32 per CTA, weights in smem)
//   k_mlp_backward  per-CTA partial loss and gradients of the mean squared
//                   error, for the samples idx[0..B) of a dataset
//   k_mlp_reduce    fixed-order sum of the CTA partials (deterministic)
//   k_mlp_adam      Adam update of the master copy, refresh of the BF16 copy
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>

#include "gdg_internal.h"

namespace {

constexpr int IN = GDG_MLP_IN, HID = GDG_MLP_HID, OUT = GDG_MLP_OUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + HID * IN, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID;
constexpr int OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + OUT * HID, NPARAM = OFF_B3 + OUT;
constexpr int WB_W1 = 0, WB_W2 = HID * IN, WB_W3 = WB_W2 + HID * HID, NWEIGHT = WB_W3 + OUT * HID;
static_assert(NPARAM == GDG_MLP_NPARAM, "parameter count");
static_assert(NWEIGHT == GDG_MLP_NWEIGHT, "weight count");

constexpr int SPB = 32;        // samples per CTA
constexpr int THREADS = 256;

struct MlpSmem {
    float *W1, *W2, *W3, *b1, *b2, *b3, *x, *h1, *h2, *y;
    __device__ MlpSmem(float *base) {
        W1 = base; W2 = W1 + HID * IN; W3 = W2 + HID * HID;
        b1 = W3 + OUT * HID; b2 = b1 + HID; b3 = b2 + HID;
        x = b3 + OUT; h1 = x + SPB * IN; h2 = h1 + SPB * HID; y = h2 + SPB * HID;
    }
    __host__ __device__ static constexpr size_t floats() { return NWEIGHT + 2 * HID + OUT + SPB * (IN + 2 * HID + OUT); }
};

// weights BF16 -> FP32 into shared memory, biases from the master block
__device__ void load_net(const __nv_bfloat16 *wb, const float *params, MlpSmem &s) {
    for (int i = threadIdx.x; i < NWEIGHT; i += blockDim.x) s.W1[i] = __bfloat162float(wb[i]);
    for (int i = threadIdx.x; i < HID; i += blockDim.x) {
        s.b1[i] = params[OFF_B1 + i];
        s.b2[i] = params[OFF_B2 + i];
    }
    for (int i = threadIdx.x; i < OUT; i += blockDim.x) s.b3[i] = params[OFF_B3 + i];
}

// forward pass of the SPB samples in s.x (ns valid): h1, h2, y in shared memory
__device__ void forward_tile(MlpSmem &s, int ns) {
    for (int o = threadIdx.x; o < SPB * HID; o += blockDim.x) {
        const int n = o / HID, j = o - (o / HID) * HID;
        float a = s.b1[j];
        if (n < ns) {
            const float *w = s.W1 + j * IN, *x = s.x + n * IN;
#pragma unroll 6
            for (int k = 0; k < IN; ++k) a = fmaf(w[k], x[k], a);
        }
        s.h1[o] = tanhf(a);
    }
    __syncthreads();
    for (int o = threadIdx.x; o < SPB * HID; o += blockDim.x) {
        const int n = o / HID, j = o - (o / HID) * HID;
        float a = s.b2[j];
        const float *w = s.W2 + j * HID, *h = s.h1 + n * HID;
#pragma unroll 8
        for (int k = 0; k < HID; ++k) a = fmaf(w[k], h[k], a);
        s.h2[o] = tanhf(a);
    }
    __syncthreads();
    for (int o = threadIdx.x; o < SPB * OUT; o += blockDim.x) {
        const int n = o / OUT, j = o - (o / OUT) * OUT;
        float a = s.b3[j];
        const float *w = s.W3 + j * HID, *h = s.h2 + n * HID;
#pragma unroll 8
        for (int k = 0; k < HID; ++k) a = fmaf(w[k], h[k], a);
        s.y[o] = a;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(THREADS)
k_mlp_forward(const __nv_bfloat16 *wb, const float *params, const float *X, int B, float *Y) {
    extern __shared__ float smf[];
    MlpSmem s(smf);
    load_net(wb, params, s);
    const int n0 = blockIdx.x * SPB, ns = min(SPB, B - n0);
    for (int i = threadIdx.x; i < SPB * IN; i += blockDim.x)
        s.x[i] = (i / IN) < ns ? X[(size_t)n0 * IN + i] : 0.f;
    __syncthreads();
    forward_tile(s, ns);
    for (int i = threadIdx.x; i < ns * OUT; i += blockDim.x) Y[(size_t)n0 * OUT + i] = s.y[i];
}

// Per-CTA partials of loss = (1/B) sum ||yhat - t||^2 and of its gradient for
// the samples idx[blockIdx.x*SPB ...] (idx may be null: samples in order).
// partial: [gridDim.x][NPARAM + 1] (the last entry is the loss share).
__global__ void __launch_bounds__(THREADS)
k_mlp_backward(const __nv_bfloat16 *wb, const float *params, const float *X, const float *T, const int *idx,
               int B, float *partial) {
    extern __shared__ float smf[];
    MlpSmem s(smf);
    float *g3 = s.y;                    // reuses y after the loss
    float *g2 = s.y + SPB * OUT;        // SPB*HID
    float *g1 = g2 + SPB * HID;         // SPB*HID
    float *red = g1 + SPB * HID;        // THREADS
    load_net(wb, params, s);
    const int n0 = blockIdx.x * SPB, ns = min(SPB, B - n0);
    for (int i = threadIdx.x; i < SPB * IN; i += blockDim.x) {
        const int n = i / IN;
        s.x[i] = n < ns ? X[(size_t)(idx ? idx[n0 + n] : n0 + n) * IN + (i - n * IN)] : 0.f;
    }
    __syncthreads();
    forward_tile(s, ns);
    // g3 = 2 (yhat - t) / B, loss share
    float lsum = 0.f;
    for (int o = threadIdx.x; o < SPB * OUT; o += blockDim.x) {
        const int n = o / OUT;
        float g = 0.f;
        if (n < ns) {
            const float d = s.y[o] - T[(size_t)(idx ? idx[n0 + n] : n0 + n) * OUT + (o - n * OUT)];
            lsum += d * d;
            g = 2.f * d / (float)B;
        }
        g3[o] = g;
    }
    red[threadIdx.x] = lsum;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    float *out = partial + (size_t)blockIdx.x * (NPARAM + 1);
    if (threadIdx.x == 0) out[NPARAM] = red[0] / (float)B;
    // layer 3: dW3[o][j] = sum_n g3[n][o] h2[n][j], db3
    for (int p = threadIdx.x; p < OUT * HID; p += blockDim.x) {
        const int o = p / HID, j = p - (p / HID) * HID;
        float a = 0.f;
        for (int n = 0; n < SPB; ++n) a = fmaf(g3[n * OUT + o], s.h2[n * HID + j], a);
        out[OFF_W3 + p] = a;
    }
    for (int o = threadIdx.x; o < OUT; o += blockDim.x) {
        float a = 0.f;
        for (int n = 0; n < SPB; ++n) a += g3[n * OUT + o];
        out[OFF_B3 + o] = a;
    }
    // g2 = (g3 W3) * (1 - h2^2)
    for (int q = threadIdx.x; q < SPB * HID; q += blockDim.x) {
        const int n = q / HID, j = q - (q / HID) * HID;
        float a = 0.f;
        for (int o = 0; o < OUT; ++o) a = fmaf(g3[n * OUT + o], s.W3[o * HID + j], a);
        const float h = s.h2[q];
        g2[q] = a * (1.f - h * h);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < HID * HID; p += blockDim.x) {
        const int j = p / HID, k = p - (p / HID) * HID;
        float a = 0.f;
        for (int n = 0; n < SPB; ++n) a = fmaf(g2[n * HID + j], s.h1[n * HID + k], a);
        out[OFF_W2 + p] = a;
    }
    for (int j = threadIdx.x; j < HID; j += blockDim.x) {
        float a = 0.f;
        for (int n = 0; n < SPB; ++n) a += g2[n * HID + j];
        out[OFF_B2 + j] = a;
    }
    // g1 = (g2 W2) * (1 - h1^2)
    for (int q = threadIdx.x; q < SPB * HID; q += blockDim.x) {
        const int n = q / HID, j = q - (q / HID) * HID;
        float a = 0.f;
        for (int k = 0; k < HID; ++k) a = fmaf(g2[n * HID + k], s.W2[k * HID + j], a);
        const float h = s.h1[q];
        g1[q] = a * (1.f - h * h);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < HID * IN; p += blockDim.x) {
        const int j = p / IN, k = p - (p / IN) * IN;
        float a = 0.f;
        for (int n = 0; n < SPB; ++n) a = fmaf(g1[n * HID + j], s.x[n * IN + k], a);
        out[OFF_W1 + p] = a;
    }
    for (int j = threadIdx.x; j < HID; j += blockDim.x) {
        float a = 0.f;
        for (int n = 0; n < SPB; ++n) a += g1[n * HID + j];
        out[OFF_B1 + j] = a;
    }
}

// grad[p] = sum over CTAs (in order) of partial[c][p]; loss likewise
__global__ void k_mlp_reduce(const float *partial, int nblocks, float *grad, float *loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > NPARAM) return;
    float a = 0.f;
    for (int c = 0; c < nblocks; ++c) a += partial[(size_t)c * (NPARAM + 1) + p];
    if (p < NPARAM) grad[p] = a;
    else *loss = a;
}

__global__ void k_mlp_adam(float *params, float *m, float *v, const float *grad, float lr, float b1, float b2,
                           float eps, float c1, float c2, __nv_bfloat16 *wb) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    const float g = grad[p];
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float x = params[p] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    params[p] = x;
    // refresh the BF16 working copy of the weights
    int w = -1;
    if (p < OFF_B1) w = WB_W1 + (p - OFF_W1);
    else if (p >= OFF_W2 && p < OFF_B2) w = WB_W2 + (p - OFF_W2);
    else if (p >= OFF_W3 && p < OFF_B3) w = WB_W3 + (p - OFF_W3);
    if (w >= 0) wb[w] = __float2bfloat16_rn(x);
}

__global__ void k_mlp_to_bf16(const float *params, __nv_bfloat16 *wb) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    int w = -1;
    if (p < OFF_B1) w = WB_W1 + (p - OFF_W1);
    else if (p >= OFF_W2 && p < OFF_B2) w = WB_W2 + (p - OFF_W2);
    else if (p >= OFF_W3 && p < OFF_B3) w = WB_W3 + (p - OFF_W3);
    if (w >= 0) wb[w] = __float2bfloat16_rn(params[p]);
}

// Learned u_t guess for every element: x0 = ||r_u|| net([c2feat, r_u/||r_u||]).
__global__ void __launch_bounds__(THREADS)
k_mlp_guess(const __nv_bfloat16 *wb, const float *params, const float *c2feat, const double *ru, int ne,
            double *x0u) {
    extern __shared__ float smf[];
    MlpSmem s(smf);
    float *nrm = smf + MlpSmem::floats();     // [SPB]
    load_net(wb, params, s);
    const int n0 = blockIdx.x * SPB, ns = min(SPB, ne - n0);
    if (threadIdx.x < SPB) {
        double a = 0.0;
        if ((int)threadIdx.x < ns)
            for (int k = 0; k < OUT; ++k) {
                const double r = ru[(size_t)(n0 + threadIdx.x) * OUT + k];
                a += r * r;
            }
        nrm[threadIdx.x] = (float)sqrt(a);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SPB * IN; i += blockDim.x) {
        const int n = i / IN, k = i - (i / IN) * IN;
        float x = 0.f;
        if (n < ns) {
            if (k < OUT) x = c2feat[(size_t)(n0 + n) * OUT + k];
            else if (nrm[n] > 0.f) x = (float)(ru[(size_t)(n0 + n) * OUT + (k - OUT)] / (double)nrm[n]);
        }
        s.x[i] = x;
    }
    __syncthreads();
    forward_tile(s, ns);
    for (int i = threadIdx.x; i < ns * OUT; i += blockDim.x) x0u[(size_t)n0 * OUT + i] = (double)nrm[i / OUT] * s.y[i];
}

// training rows: X = [c2feat, r_u/||r_u||] (FP32) and, when y is given,
// T = y/||r_u|| (FP32); one thread per element
__global__ void k_mlp_rows(const float *c2feat, const double *ru, const double *y, int ne, float *X, float *T) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    double a = 0.0;
    for (int k = 0; k < OUT; ++k) {
        const double r = ru[(size_t)e * OUT + k];
        a += r * r;
    }
    const double n = sqrt(a), inv = n > 0.0 ? 1.0 / n : 0.0;
    for (int k = 0; k < OUT; ++k) {
        X[(size_t)e * IN + k] = c2feat[(size_t)e * OUT + k];
        X[(size_t)e * IN + OUT + k] = (float)(ru[(size_t)e * OUT + k] * inv);
        if (y && T) T[(size_t)e * OUT + k] = (float)(y[(size_t)e * OUT + k] * inv);
    }
}

size_t fwd_smem() { return MlpSmem::floats() * sizeof(float); }
size_t guess_smem() { return (MlpSmem::floats() + SPB) * sizeof(float); }
size_t bwd_smem() { return (MlpSmem::floats() + 2 * SPB * HID + THREADS) * sizeof(float); }

bool attrs_done = false;
int set_attrs() {
    if (attrs_done) return GDG_OK;
    if (cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem()) != cudaSuccess ||
        cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem()) != cudaSuccess ||
        cudaFuncSetAttribute(k_mlp_guess, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)guess_smem()) != cudaSuccess)
        return GDG_ECUDA;
    attrs_done = true;
    return GDG_OK;
}

}  // namespace

int gdg_mlp_guess_launch(const uint16_t *w_bf16, const float *params, const float *c2feat, const double *ru,
                         int ne, double *x0u, cudaStream_t s) {
    if (set_attrs()) return GDG_ECUDA;
    k_mlp_guess<<<(ne + SPB - 1) / SPB, THREADS, guess_smem(), s>>>(
        reinterpret_cast<const __nv_bfloat16 *>(w_bf16), params, c2feat, ru, ne, x0u);
    return GDG_OK;
}

int gdg_mlp_rows_launch(const float *c2feat, const double *ru, const double *y, int ne, float *X, float *T,
                        cudaStream_t s) {
    k_mlp_rows<<<(ne + 127) / 128, 128, 0, s>>>(c2feat, ru, y, ne, X, T);
    return GDG_OK;
}

extern "C" int gdg_mlp_forward(const uint16_t *w_bf16, const float *params, const float *X, int B, float *Y,
                               void *stream) {
    if (!w_bf16 || !params || !X || !Y || B < 0) return GDG_EINVAL;
    if (B == 0) return GDG_OK;
    if (set_attrs()) return GDG_ECUDA;
    const int grid = (B + SPB - 1) / SPB;
    k_mlp_forward<<<grid, THREADS, fwd_smem(), (cudaStream_t)stream>>>(
        reinterpret_cast<const __nv_bfloat16 *>(w_bf16), params, X, B, Y);
    return cudaGetLastError() == cudaSuccess ? GDG_OK : GDG_ECUDA;
}

extern "C" long long gdg_mlp_partial_len(int B) {
    return B <= 0 ? 0 : (long long)((B + SPB - 1) / SPB) * (NPARAM + 1);
}

extern "C" int gdg_mlp_backward(const uint16_t *w_bf16, const float *params, const float *X, const float *T,
                                const int *idx, int B, float *partial, float *grad, float *loss, void *stream) {
    if (!w_bf16 || !params || !X || !T || !partial || !grad || !loss || B <= 0) return GDG_EINVAL;
    if (set_attrs()) return GDG_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = (B + SPB - 1) / SPB;
    k_mlp_backward<<<grid, THREADS, bwd_smem(), s>>>(reinterpret_cast<const __nv_bfloat16 *>(w_bf16), params, X,
                                                     T, idx, B, partial);
    k_mlp_reduce<<<(NPARAM + 1 + 255) / 256, 256, 0, s>>>(partial, grid, grad, loss);
    return cudaGetLastError() == cudaSuccess ? GDG_OK : GDG_ECUDA;
}

extern "C" int gdg_mlp_adam(float *params, float *m, float *v, const float *grad, int step, float lr,
                            uint16_t *w_bf16, void *stream) {
    if (!params || !m || !v || !grad || !w_bf16 || step < 1 || !(lr > 0.f)) return GDG_EINVAL;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - std::pow(b1, (float)step), c2 = 1.f - std::pow(b2, (float)step);
    k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        params, m, v, grad, lr, b1, b2, eps, c1, c2, reinterpret_cast<__nv_bfloat16 *>(w_bf16));
    return cudaGetLastError() == cudaSuccess ? GDG_OK : GDG_ECUDA;
}

extern "C" int gdg_mlp_to_bf16(const float *params, uint16_t *w_bf16, void *stream) {
    if (!params || !w_bf16) return GDG_EINVAL;
    k_mlp_to_bf16<<<(NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        params, reinterpret_cast<__nv_bfloat16 *>(w_bf16));
    return cudaGetLastError() == cudaSuccess ? GDG_OK : GDG_ECUDA;
}
