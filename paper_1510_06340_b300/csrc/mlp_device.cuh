// mlp_device.cuh -- device evaluation of the Newton-seed MLP (inputs
// (ln E, |M|/E) standardised; tanh hidden layers of 32; output
// v0 = (|M|/E) sigmoid(z)).  BF16 weights and layer-2 inputs, FP32
// accumulation.  The warp form runs the 32x32 layer on the tensor cores
// (mma.sync m16n8k16) for the 32 samples of a converged warp; the scalar
// form is the same arithmetic for one thread.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.h"

namespace hy {

__device__ __forceinline__ float mlp_seed_scalar(const Scheme &sc, float lnE, float x) {
    const float *F = sc.mlp_f;
    const __nv_bfloat16 *Wb = static_cast<const __nv_bfloat16 *>(sc.mlp_w);
    const float in0 = (lnE - __ldg(F + MLP_OFF_NORM)) / __ldg(F + MLP_OFF_NORM + 1);
    const float in1 = (x - __ldg(F + MLP_OFF_NORM + 2)) / __ldg(F + MLP_OFF_NORM + 3);
    float h1[MLP_H];
#pragma unroll
    for (int j = 0; j < MLP_H; ++j) {
        const float a = fmaf(__bfloat162float(Wb[MLP_OFF_W1 + 2 * j + 1]), in1,
                             fmaf(__bfloat162float(Wb[MLP_OFF_W1 + 2 * j]), in0,
                                  __ldg(F + MLP_OFF_B1 + j)));
        h1[j] = __bfloat162float(__float2bfloat16_rn(tanhf(a)));
    }
    float z = __ldg(F + MLP_OFF_B3);
#pragma unroll 4
    for (int j = 0; j < MLP_H; ++j) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < MLP_H; ++k)
            s = fmaf(__bfloat162float(Wb[MLP_OFF_W2 + j * MLP_H + k]), h1[k], s);
        z = fmaf(__bfloat162float(Wb[MLP_OFF_W3 + j]), tanhf(s + __ldg(F + MLP_OFF_B2 + j)), z);
    }
    const float vc = 3.0f * x / (2.0f + sqrtf(4.0f - 3.0f * x * x));
    return vc + (x - vc) / (1.0f + __expf(-z));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x = lo (low half)
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Warp-level forward of 32 samples (two 16-row tiles).  Lane l supplies the
// inputs of sample l through in0/in1 (already standardised) and x = |M|/E;
// returns the seed of sample l.  Optionally stores h1 (bf16-rounded) and h2
// per sample into shared rows H1[l][.], H2[l][.] (stride ld).
// hardware tanh approximation (max relative error about 2^-11); used for the
// seed inside sweeps, where it only moves Newton's starting point
__device__ __forceinline__ float tanh_fast(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <bool FAST>
__device__ __forceinline__ float act_tanh(float x) {
    return FAST ? tanh_fast(x) : tanhf(x);
}

template <bool STORE, bool FAST = false>
__device__ __forceinline__ float mlp_warp_forward(const float *__restrict__ F,
                                                  const __nv_bfloat16 *__restrict__ Wb,
                                                  float in0, float in1, float x, float *H1,
                                                  float *H2, int ld, float &z_out) {
    const int lane = threadIdx.x & 31;
    const int gid = lane >> 2, tig = lane & 3;
    float zp[2][2];   // [tile][row half] partial of layer 3
#pragma unroll
    for (int tile = 0; tile < 2; ++tile) {
        const int r0 = tile * 16 + gid, r1 = r0 + 8;   // samples (lanes) of this thread's rows
        const float a0 = __shfl_sync(0xffffffffu, in0, r0), a1 = __shfl_sync(0xffffffffu, in1, r0);
        const float c0 = __shfl_sync(0xffffffffu, in0, r1), c1 = __shfl_sync(0xffffffffu, in1, r1);
        // layer 1 in A-fragment layout: cols k = ks*16 + tig*2 + {0,1} (+8)
        uint32_t A[2][4];
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int k0 = ks * 16 + half * 8 + tig * 2;
                float h[2][2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int k = k0 + q;
                    const float w0 = __bfloat162float(Wb[MLP_OFF_W1 + 2 * k]);
                    const float w1 = __bfloat162float(Wb[MLP_OFF_W1 + 2 * k + 1]);
                    const float b = __ldg(F + MLP_OFF_B1 + k);
                    h[0][q] = act_tanh<FAST>(fmaf(w1, a1, fmaf(w0, a0, b)));
                    h[1][q] = act_tanh<FAST>(fmaf(w1, c1, fmaf(w0, c0, b)));
                }
                A[ks][half * 2 + 0] = pack_bf16(h[0][0], h[0][1]);   // row r0
                A[ks][half * 2 + 1] = pack_bf16(h[1][0], h[1][1]);   // row r1
                if (STORE) {
                    H1[r0 * ld + k0] = __bfloat162float(__float2bfloat16_rn(h[0][0]));
                    H1[r0 * ld + k0 + 1] = __bfloat162float(__float2bfloat16_rn(h[0][1]));
                    H1[r1 * ld + k0] = __bfloat162float(__float2bfloat16_rn(h[1][0]));
                    H1[r1 * ld + k0 + 1] = __bfloat162float(__float2bfloat16_rn(h[1][1]));
                }
            }
        }
        zp[tile][0] = 0.f;
        zp[tile][1] = 0.f;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                // B[k][n] = W2[n][k], n = nt*8 + gid, k = ks*16 + tig*2 + {0,1} (+8)
                const int n = nt * 8 + gid;
                const __nv_bfloat16 *w = Wb + MLP_OFF_W2 + n * MLP_H + ks * 16 + tig * 2;
                uint32_t B[2];
                B[0] = *reinterpret_cast<const uint32_t *>(w);
                B[1] = *reinterpret_cast<const uint32_t *>(w + 8);
                // A fragment order: a0a1 (r0, k), a2a3 (r1, k), a4a5 (r0, k+8), a6a7 (r1, k+8)
                const uint32_t Af[4] = {A[ks][0], A[ks][1], A[ks][2], A[ks][3]};
                mma_bf16(acc, Af, B);
            }
            // C layout: acc0,1 -> (r0, n0 + {0,1}); acc2,3 -> (r1, n0 + {0,1})
            const int n0 = nt * 8 + tig * 2;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float b2 = __ldg(F + MLP_OFF_B2 + n0 + q);
                const float w3 = __bfloat162float(Wb[MLP_OFF_W3 + n0 + q]);
                const float h0 = act_tanh<FAST>(acc[q] + b2), h1v = act_tanh<FAST>(acc[2 + q] + b2);
                zp[tile][0] = fmaf(w3, h0, zp[tile][0]);
                zp[tile][1] = fmaf(w3, h1v, zp[tile][1]);
                if (STORE) {
                    H2[r0 * ld + n0 + q] = h0;
                    H2[r1 * ld + n0 + q] = h1v;
                }
            }
        }
        // reduce the 4 threads of a group
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            zp[tile][h] += __shfl_xor_sync(0xffffffffu, zp[tile][h], 1);
            zp[tile][h] += __shfl_xor_sync(0xffffffffu, zp[tile][h], 2);
        }
    }
    // sample l lives in tile l/16, row half (l%16)/8, group l%8 (lane 4*(l%8))
    const int tile = lane >> 4, hh = (lane >> 3) & 1, src = (lane & 7) * 4;
    const float z00 = __shfl_sync(0xffffffffu, zp[0][0], src);
    const float z01 = __shfl_sync(0xffffffffu, zp[0][1], src);
    const float z10 = __shfl_sync(0xffffffffu, zp[1][0], src);
    const float z11 = __shfl_sync(0xffffffffu, zp[1][1], src);
    const float z = (tile == 0 ? (hh == 0 ? z00 : z01) : (hh == 0 ? z10 : z11)) +
                    __ldg(F + MLP_OFF_B3);
    z_out = z;
    const float vc = 3.0f * x / (2.0f + sqrtf(4.0f - 3.0f * x * x));
    return vc + (x - vc) / (1.0f + __expf(-z));
}


// Seed for this lane's state; every lane of the warp must call it together.
__device__ __forceinline__ float mlp_seed_warp(const Scheme &sc, float lnE, float x) {
    const float *F = sc.mlp_f;
    const __nv_bfloat16 *Wb = static_cast<const __nv_bfloat16 *>(sc.mlp_w);
    const float in0 = (lnE - __ldg(F + MLP_OFF_NORM)) / __ldg(F + MLP_OFF_NORM + 1);
    const float in1 = (x - __ldg(F + MLP_OFF_NORM + 2)) / __ldg(F + MLP_OFF_NORM + 3);
    float z;
    __syncwarp();
    return mlp_warp_forward<false, true>(F, Wb, in0, in1, x, nullptr, nullptr, 0, z);
}

}  // namespace hy
