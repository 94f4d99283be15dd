// mlp.cu -- the Newton-seed MLP (not in the paper): a 2 -> 32 -> 32 -> 1 tanh
// network that maps (ln E, x = |M|/E) to where the root v lies between the
// p = e/3 root vc and x, giving the start of the Newton cons->prim solve for a
// tabulated EOS.  The 32x32 layer runs on
// the tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation);
// its inputs and the weights are rounded to BF16, everything else is FP32.
// Training (loss gradient + Adam) runs on the GPU with the same forward and
// an FP32 backward pass; the bf16 rounding is passed straight through.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <random>
#include <vector>

#include "../../include/hydro.h"
#include "common.h"
#include "kernels.h"
#include "mlp_device.cuh"

namespace hy {

// bf16 copy of the whole parameter vector (weights are read at their offsets)
__global__ void k_mlp_prepare(const float *__restrict__ p, __nv_bfloat16 *__restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < MLP_NPARAM) w[i] = __float2bfloat16_rn(p[i]);
}

// X [n][2] = (ln E, x); one warp per 32 samples
__global__ void k_mlp_forward(const float *__restrict__ F, const __nv_bfloat16 *__restrict__ Wb,
                              const float *__restrict__ X, int n, float *__restrict__ out) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int s = warp * 32 + lane;
    if (warp * 32 >= n) return;   // whole warp out of range
    const bool ok = s < n;
    const float lnE = ok ? X[2 * s] : 0.f, x = ok ? X[2 * s + 1] : 0.f;
    const float in0 = (lnE - __ldg(F + MLP_OFF_NORM)) / __ldg(F + MLP_OFF_NORM + 1);
    const float in1 = (x - __ldg(F + MLP_OFF_NORM + 2)) / __ldg(F + MLP_OFF_NORM + 3);
    float z;
    const float v = mlp_warp_forward<false>(F, Wb, in0, in1, x, nullptr, nullptr, 0, z);
    if (ok) out[s] = v;
}

// the bf16-rounded first-layer activations that k_mlp_forward feeds to the
// tensor cores, H1 [n][32] (same warp forward, its rows kept in shared memory)
constexpr int HID_WARPS = 4;
__global__ void __launch_bounds__(32 * HID_WARPS)
k_mlp_hidden(const float *__restrict__ F, const __nv_bfloat16 *__restrict__ Wb,
             const float *__restrict__ X, int n, float *__restrict__ H1out) {
    __shared__ float h1s[HID_WARPS][32 * (MLP_H + 1)];
    __shared__ float h2s[HID_WARPS][32 * (MLP_H + 1)];
    const int wl = threadIdx.x >> 5;
    const int warp = blockIdx.x * HID_WARPS + wl;
    const int lane = threadIdx.x & 31;
    const int s = warp * 32 + lane;
    if (warp * 32 >= n) return;   // whole warp out of range
    const bool ok = s < n;
    const float lnE = ok ? X[2 * s] : 0.f, x = ok ? X[2 * s + 1] : 0.f;
    const float in0 = (lnE - __ldg(F + MLP_OFF_NORM)) / __ldg(F + MLP_OFF_NORM + 1);
    const float in1 = (x - __ldg(F + MLP_OFF_NORM + 2)) / __ldg(F + MLP_OFF_NORM + 3);
    float z;
    mlp_warp_forward<true>(F, Wb, in0, in1, x, h1s[wl], h2s[wl], MLP_H + 1, z);
    __syncwarp();
    if (ok)
        for (int k = 0; k < MLP_H; ++k) H1out[(long long)s * MLP_H + k] = h1s[wl][lane * (MLP_H + 1) + k];
}

constexpr int TB = 256;          // samples per block in the gradient kernel
constexpr int LDH = MLP_H + 1;   // padded smem row

// loss and gradient over samples idx[first .. first+count) (idx may be null)
__global__ void __launch_bounds__(TB)
k_mlp_loss_grad(const float *__restrict__ F, const __nv_bfloat16 *__restrict__ Wb,
                const float *__restrict__ X, const float *__restrict__ Y,
                const int *__restrict__ idx, long long first, int count, float inv_n,
                float *__restrict__ grad, float *__restrict__ loss) {
    extern __shared__ float sm[];
    float *H1 = sm;
    float *H2 = H1 + TB * LDH;
    float *DA2 = H2 + TB * LDH;
    float *DA1 = DA2 + TB * LDH;
    float *DZ = DA1 + TB * LDH;
    float *IN0 = DZ + TB;
    float *IN1 = IN0 + TB;
    float *LS = IN1 + TB;
    const int t = threadIdx.x;
    const long long base = first + (long long)blockIdx.x * TB;
    const bool ok = (long long)blockIdx.x * TB + t < count;
    long long s = base + t;
    if (ok && idx) s = idx[s];
    const float lnE = ok ? X[2 * s] : 0.f, x = ok ? X[2 * s + 1] : 0.f;
    const float y = ok ? Y[s] : 0.f;
    const float in0 = (lnE - __ldg(F + MLP_OFF_NORM)) / __ldg(F + MLP_OFF_NORM + 1);
    const float in1 = (x - __ldg(F + MLP_OFF_NORM + 2)) / __ldg(F + MLP_OFF_NORM + 3);
    const int wbase = (t >> 5) * 32;
    float z;
    const float v0 = mlp_warp_forward<true>(F, Wb, in0, in1, x, H1 + wbase * LDH,
                                            H2 + wbase * LDH, LDH, z);
    const float r = 1.0f / (1.0f + __expf(-z));
    const float d = ok ? v0 - y : 0.f;
    const float vc = 3.0f * x / (2.0f + sqrtf(4.0f - 3.0f * x * x));
    DZ[t] = 2.0f * d * inv_n * (x - vc) * r * (1.0f - r);
    IN0[t] = in0;
    IN1[t] = in1;
    LS[t] = d * d;
    __syncwarp();
    // per-sample backward through layer 3 and layer 2
    {
        const float dz = DZ[t];
        const float *h2 = H2 + t * LDH;
        float *da2 = DA2 + t * LDH;
#pragma unroll 8
        for (int j = 0; j < MLP_H; ++j) {
            const float w3 = __bfloat162float(Wb[MLP_OFF_W3 + j]);
            da2[j] = dz * w3 * (1.0f - h2[j] * h2[j]);
        }
        const float *h1 = H1 + t * LDH;
        float *da1 = DA1 + t * LDH;
        for (int k = 0; k < MLP_H; ++k) {
            float acc = 0.f;
#pragma unroll 8
            for (int j = 0; j < MLP_H; ++j)
                acc = fmaf(__bfloat162float(Wb[MLP_OFF_W2 + j * MLP_H + k]), da2[j], acc);
            da1[k] = acc * (1.0f - h1[k] * h1[k]);
        }
    }
    __syncthreads();
    // weight gradients: sums over the block's samples
    for (int e = t; e < MLP_NPARAM - 4; e += TB) {
        float acc = 0.f;
        if (e < MLP_OFF_B1) {                       // W1[k][c]
            const int k = e >> 1, c = e & 1;
            const float *in = c ? IN1 : IN0;
            for (int q = 0; q < TB; ++q) acc = fmaf(DA1[q * LDH + k], in[q], acc);
        } else if (e < MLP_OFF_W2) {                // b1[k]
            const int k = e - MLP_OFF_B1;
            for (int q = 0; q < TB; ++q) acc += DA1[q * LDH + k];
        } else if (e < MLP_OFF_B2) {                // W2[j][k]
            const int j = (e - MLP_OFF_W2) / MLP_H, k = (e - MLP_OFF_W2) % MLP_H;
            for (int q = 0; q < TB; ++q) acc = fmaf(DA2[q * LDH + j], H1[q * LDH + k], acc);
        } else if (e < MLP_OFF_W3) {                // b2[j]
            const int j = e - MLP_OFF_B2;
            for (int q = 0; q < TB; ++q) acc += DA2[q * LDH + j];
        } else if (e < MLP_OFF_B3) {                // W3[j]
            const int j = e - MLP_OFF_W3;
            for (int q = 0; q < TB; ++q) acc = fmaf(DZ[q], H2[q * LDH + j], acc);
        } else {                                    // b3
            for (int q = 0; q < TB; ++q) acc += DZ[q];
        }
        atomicAdd(grad + e, acc);
    }
    if (t == 0) {
        float l = 0.f;
        for (int q = 0; q < TB; ++q) l += LS[q];
        atomicAdd(loss, l * inv_n);
    }
}

constexpr size_t LG_SMEM = (size_t)(4 * TB * LDH + 4 * TB) * sizeof(float);

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1t, float b2t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_NPARAM - 4) return;   // normalisation constants stay fixed
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / (1.f - b1t)) / (sqrtf(vi / (1.f - b2t)) + eps);
}

__global__ void k_accumulate(float *__restrict__ dst, const float *__restrict__ src) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst += *src;
}

cudaError_t launch_mlp_prepare(const float *params, void *w_bf16, cudaStream_t s) {
    k_mlp_prepare<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(params, (__nv_bfloat16 *)w_bf16);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float *params, const float *X, int n, float *out,
                               cudaStream_t s) {
    __nv_bfloat16 *w;
    cudaError_t e = cudaMallocAsync(&w, MLP_NPARAM * sizeof(__nv_bfloat16), s);
    if (e != cudaSuccess) return e;
    k_mlp_prepare<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(params, w);
    const int warps = (n + 31) / 32;
    if (warps > 0) k_mlp_forward<<<(warps + 3) / 4, 128, 0, s>>>(params, w, X, n, out);
    e = cudaGetLastError();
    cudaFreeAsync(w, s);
    return e;
}

cudaError_t launch_mlp_hidden(const float *params, const float *X, int n, float *H1,
                              cudaStream_t s) {
    __nv_bfloat16 *w;
    cudaError_t e = cudaMallocAsync(&w, MLP_NPARAM * sizeof(__nv_bfloat16), s);
    if (e != cudaSuccess) return e;
    k_mlp_prepare<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(params, w);
    const int warps = (n + 31) / 32;
    if (warps > 0)
        k_mlp_hidden<<<(warps + HID_WARPS - 1) / HID_WARPS, 32 * HID_WARPS, 0, s>>>(params, w, X,
                                                                                  n, H1);
    e = cudaGetLastError();
    cudaFreeAsync(w, s);
    return e;
}

static cudaError_t loss_grad_into(const float *params, const __nv_bfloat16 *w, const float *X,
                                  const float *Y, const int *idx, long long first, int count,
                                  float *grad, float *loss, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_loss_grad,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)LG_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int blocks = (count + TB - 1) / TB;
    k_mlp_loss_grad<<<blocks, TB, LG_SMEM, s>>>(params, w, X, Y, idx, first, count,
                                                1.0f / (float)count, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_mlp_loss_grad(const float *params, const float *X, const float *Y, int n,
                                 float *grad, float *loss, cudaStream_t s) {
    __nv_bfloat16 *w;
    cudaError_t e = cudaMallocAsync(&w, MLP_NPARAM * sizeof(__nv_bfloat16), s);
    if (e != cudaSuccess) return e;
    k_mlp_prepare<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(params, w);
    cudaMemsetAsync(grad, 0, MLP_NPARAM * sizeof(float), s);
    cudaMemsetAsync(loss, 0, sizeof(float), s);
    e = loss_grad_into(params, w, X, Y, nullptr, 0, n, grad, loss, s);
    cudaFreeAsync(w, s);
    return e;
}

}  // namespace hy

using namespace hy;

extern "C" hydro_status hydro_mlp_train(float *params, const float *X, const float *Y, int n,
                                        int batch, int epochs, float lr, unsigned long long seed,
                                        float *loss_hist, void *stream_) {
    if (!params || !X || !Y || n < 1 || batch < 1 || epochs < 1 || !(lr > 0.f))
        return HYDRO_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream_;
    batch = std::min(batch, n);
    float *g = nullptr, *m = nullptr, *v = nullptr, *lbuf = nullptr;
    int *idx = nullptr;
    __nv_bfloat16 *w = nullptr;
    cudaError_t e = cudaSuccess;
    auto cleanup = [&]() {
        cudaStreamSynchronize(s);
        cudaFree(g); cudaFree(m); cudaFree(v); cudaFree(lbuf); cudaFree(idx); cudaFree(w);
    };
    if ((e = cudaMalloc(&g, MLP_NPARAM * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&m, MLP_NPARAM * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&v, MLP_NPARAM * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&lbuf, sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&idx, (size_t)n * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&w, MLP_NPARAM * sizeof(__nv_bfloat16))) != cudaSuccess) {
        cleanup();
        return e == cudaErrorMemoryAllocation ? HYDRO_E_OOM : HYDRO_E_CUDA;
    }
    cudaMemsetAsync(m, 0, MLP_NPARAM * sizeof(float), s);
    cudaMemsetAsync(v, 0, MLP_NPARAM * sizeof(float), s);
    cudaMemsetAsync(loss_hist, 0, epochs * sizeof(float), s);
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    std::mt19937_64 rng(seed);
    double b1t = 1.0, b2t = 1.0;
    const int nb = n / batch;   // full minibatches per epoch
    const double total = double(nb) * epochs;
    long long step = 0;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        e = cudaMemcpyAsync(idx, perm.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);   // perm is reused next epoch
        for (int b = 0; b < nb && e == cudaSuccess; ++b) {
            b1t *= 0.9;
            b2t *= 0.999;
            k_mlp_prepare<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(params, w);
            cudaMemsetAsync(g, 0, MLP_NPARAM * sizeof(float), s);
            cudaMemsetAsync(lbuf, 0, sizeof(float), s);
            e = loss_grad_into(params, w, X, Y, idx, (long long)b * batch, batch, g, lbuf, s);
            if (e != cudaSuccess) break;
            // cosine decay of the learning rate over the whole run
            const float lr_t = (float)(0.5 * lr * (1.0 + cos(3.14159265358979 * double(step++) / total)));
            k_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(params, g, m, v, lr_t, (float)b1t,
                                                            (float)b2t);
            k_accumulate<<<1, 32, 0, s>>>(loss_hist + ep, lbuf);
            e = cudaGetLastError();
        }
    }
    cleanup();
    if (e != cudaSuccess) return HYDRO_E_CUDA;
    // loss_hist holds the sum of minibatch means; divide by the count on the host side
    std::vector<float> h(epochs);
    cudaMemcpy(h.data(), loss_hist, epochs * sizeof(float), cudaMemcpyDeviceToHost);
    for (float &x : h) x /= (float)std::max(nb, 1);
    cudaMemcpy(loss_hist, h.data(), epochs * sizeof(float), cudaMemcpyHostToDevice);
    return HYDRO_OK;
}
