// mlp.cu -- troubled-cell classifier: 44 -> 64 -> 64 -> 1, ReLU, sigmoid, FP32.
//
// Inference (k_mlp_forward): one thread per cell, weights staged in shared
// memory.  Training (k_mlp_grad): each block takes 64 samples, runs the forward
// and backward passes with the activations in shared memory, and forms its part
// of the weight gradients as small contractions over its samples before one
// atomic add per weight; k_mlp_adam applies the Adam update.  The loss is the
// mean binary cross-entropy, written from the logits.
//
// Parameter vector (7105 floats): W1[64][44], b1[64], W2[64][64], b2[64],
// w3[64], b3.
#include <cuda_runtime.h>
#include <math.h>

#include "../../include/crkdg.h"

namespace {

constexpr int NIN = CRKDG_MLP_NIN, NH = CRKDG_MLP_NH;
constexpr int OW1 = 0, OB1 = OW1 + NH * NIN, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NH, NP = OB3 + 1;
static_assert(NP == CRKDG_MLP_NPARAM, "parameter layout");

__device__ __forceinline__ float softplus(float z) { return fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z))); }
__device__ __forceinline__ float sigmoidf_(float z) {
    float e = expf(-fabsf(z));
    return z >= 0.0f ? 1.0f / (1.0f + e) : e / (1.0f + e);
}

__global__ void __launch_bounds__(256) k_mlp_forward(const float *__restrict__ theta, const float *__restrict__ X,
                                                     int n, float *__restrict__ prob) {
    __shared__ float w[NP];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = theta[i];
    __syncthreads();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float x[NIN], h1[NH];
#pragma unroll
    for (int k = 0; k < NIN; ++k) x[k] = X[(size_t)r * NIN + k];
#pragma unroll 4
    for (int j = 0; j < NH; ++j) {
        float a = w[OB1 + j];
#pragma unroll
        for (int k = 0; k < NIN; ++k) a = fmaf(w[OW1 + j * NIN + k], x[k], a);
        h1[j] = fmaxf(a, 0.0f);
    }
    float z = w[OB3];
    for (int j = 0; j < NH; ++j) {
        float a = w[OB2 + j];
#pragma unroll
        for (int i = 0; i < NH; ++i) a = fmaf(w[OW2 + j * NH + i], h1[i], a);
        z = fmaf(w[OW3 + j], fmaxf(a, 0.0f), z);
    }
    prob[r] = sigmoidf_(z);
}

constexpr int SB = 64;  // samples per block in the gradient kernel

__global__ void __launch_bounds__(SB) k_mlp_grad(const float *__restrict__ theta, const float *__restrict__ X,
                                                 const float *__restrict__ y, int n, float inv_total,
                                                 float *__restrict__ grad, float *__restrict__ loss) {
    extern __shared__ float sm[];
    float *w = sm;                  // NP
    float *sx = w + NP;             // SB x NIN
    float *sh1 = sx + SB * NIN;     // SB x NH  (h1)
    float *sd1 = sh1 + SB * NH;     // SB x NH  (d a1)
    float *sd2 = sd1 + SB * NH;     // SB x NH  (d a2)
    float *sdz = sd2 + SB * NH;     // SB
    float *sh2 = sdz + SB;          // SB x NH  (h2)
    for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = theta[i];
    const int t = threadIdx.x;
    const int r = blockIdx.x * SB + t;
    const bool valid = r < n;
    for (int k = 0; k < NIN; ++k) sx[t * NIN + k] = valid ? X[(size_t)r * NIN + k] : 0.0f;
    __syncthreads();
    // forward, one sample per thread
    float a1[NH];
    for (int j = 0; j < NH; ++j) {
        float a = w[OB1 + j];
        for (int k = 0; k < NIN; ++k) a = fmaf(w[OW1 + j * NIN + k], sx[t * NIN + k], a);
        a1[j] = a;
        sh1[t * NH + j] = fmaxf(a, 0.0f);
    }
    float z = w[OB3];
    for (int j = 0; j < NH; ++j) {
        float a = w[OB2 + j];
        for (int i = 0; i < NH; ++i) a = fmaf(w[OW2 + j * NH + i], sh1[t * NH + i], a);
        float h = fmaxf(a, 0.0f);
        sh2[t * NH + j] = h;
        sd2[t * NH + j] = a > 0.0f ? 1.0f : 0.0f;  // ReLU mask, scaled below
        z = fmaf(w[OW3 + j], h, z);
    }
    float yy = valid ? y[r] : 0.0f;
    float dz = valid ? (sigmoidf_(z) - yy) * inv_total : 0.0f;
    if (valid) atomicAdd(loss, (softplus(z) - yy * z) * inv_total);
    sdz[t] = dz;
    // backward through the layers of this sample
    for (int j = 0; j < NH; ++j) sd2[t * NH + j] *= dz * w[OW3 + j];
    for (int i = 0; i < NH; ++i) {
        float s = 0.0f;
        for (int j = 0; j < NH; ++j) s = fmaf(sd2[t * NH + j], w[OW2 + j * NH + i], s);
        sd1[t * NH + i] = a1[i] > 0.0f ? s : 0.0f;
    }
    __syncthreads();
    // weight gradients: contractions over the block's samples, one atomic per weight
    for (int e = t; e < NH * NIN; e += SB) {
        int j = e / NIN, k = e - j * NIN;
        float s = 0.0f;
        for (int q = 0; q < SB; ++q) s = fmaf(sd1[q * NH + j], sx[q * NIN + k], s);
        atomicAdd(&grad[OW1 + e], s);
    }
    for (int e = t; e < NH * NH; e += SB) {
        int j = e / NH, i = e - j * NH;
        float s = 0.0f;
        for (int q = 0; q < SB; ++q) s = fmaf(sd2[q * NH + j], sh1[q * NH + i], s);
        atomicAdd(&grad[OW2 + e], s);
    }
    if (t < NH) {
        float s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
        for (int q = 0; q < SB; ++q) {
            s1 += sd1[q * NH + t];
            s2 += sd2[q * NH + t];
            s3 = fmaf(sdz[q], sh2[q * NH + t], s3);
        }
        atomicAdd(&grad[OB1 + t], s1);
        atomicAdd(&grad[OB2 + t], s2);
        atomicAdd(&grad[OW3 + t], s3);
    }
    if (t == 0) {
        float s = 0.0f;
        for (int q = 0; q < SB; ++q) s += sdz[q];
        atomicAdd(&grad[OB3], s);
    }
}

__global__ void k_mlp_adam(float *theta, float *m, float *v, const float *grad, float lr, float c1, float c2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float g = grad[i];
    float mi = b1 * m[i] + (1.0f - b1) * g;
    float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

size_t grad_smem() { return sizeof(float) * (NP + SB * NIN + 4 * SB * NH + SB); }

}  // namespace

extern "C" {

crkdg_status crkdg_mlp_forward(const float *params, const float *X, int n, float *prob, void *stream) {
    if (!params || !X || !prob || n < 0) return CRKDG_E_ARG;
    if (n == 0) return CRKDG_OK;
    k_mlp_forward<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, X, n, prob);
    return cudaGetLastError() == cudaSuccess ? CRKDG_OK : CRKDG_E_CUDA;
}

crkdg_status crkdg_mlp_grad(const float *params, const float *X, const float *y, int n, float *grad, float *loss,
                            void *stream) {
    if (!params || !X || !y || !grad || !loss || n <= 0) return CRKDG_E_ARG;
    static bool configured = false;
    if (!configured) {
        if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem()) !=
            cudaSuccess)
            return CRKDG_E_CUDA;
        configured = true;
    }
    k_mlp_grad<<<(n + SB - 1) / SB, SB, grad_smem(), (cudaStream_t)stream>>>(params, X, y, n, 1.0f / (float)n, grad,
                                                                            loss);
    return cudaGetLastError() == cudaSuccess ? CRKDG_OK : CRKDG_E_CUDA;
}

crkdg_status crkdg_mlp_adam(float *params, float *m, float *v, const float *grad, int step, float lr, void *stream) {
    if (!params || !m || !v || !grad || step < 1 || !(lr > 0.0f)) return CRKDG_E_ARG;
    float c1 = 1.0f - powf(0.9f, (float)step), c2 = 1.0f - powf(0.999f, (float)step);
    k_mlp_adam<<<(NP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, m, v, grad, lr, c1, c2);
    return cudaGetLastError() == cudaSuccess ? CRKDG_OK : CRKDG_E_CUDA;
}

}  // extern "C"
