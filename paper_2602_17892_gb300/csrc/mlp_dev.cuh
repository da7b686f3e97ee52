// Device code shared by the learned-lambda network's training kernels and the hybrid step's
// inference: parameter layout, GELU and the 16 x 8 output tile of a matrix product.
//
// Network (not in the paper): 80 features -> 64 -> 64 -> 1, GELU (tanh form) after both hidden
// layers, output log10(lambda / sigma_1).  The features are first standardised in FP32,
// f' = (f - mu) * isd, with mu and isd fixed by training (not trained themselves).  Parameters
// are one FP32 vector in this order: W1[64][80], b1[64], W2[64][64], b2[64], w3[64], b3,
// mu[80], isd[80].  In BF16 mode the weights, the standardised inputs and both hidden
// activations are rounded to BF16 before each product (biases stay FP32) and the products
// accumulate in FP32 on the tensor cores.
#pragma once
#include <cuda_bf16.h>

namespace ct {
namespace mlp {

constexpr int kIn = 80, kHid = 64;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid,
              kOffB2 = kOffW2 + kHid * kHid, kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid,
              kOffMu = kOffB3 + 1, kOffIsd = kOffMu + kIn, kNParams = kOffIsd + kIn;

// standardised feature k (FP32)
__device__ __forceinline__ float standardise(const float *__restrict__ P, float f, int k)
{
    return (f - P[kOffMu + k]) * P[kOffIsd + k];
}

// tanh(u) = 1 - 2 / (exp(2u) + 1): absolute error a few FP32 ulps for every u (exp(2u) = inf
// gives 1, exp(2u) = 0 gives -1), unlike a hardware tanh approximation
__device__ __forceinline__ float tanh_exp(float u) { return 1.f - 2.f / (expf(2.f * u) + 1.f); }

__device__ __forceinline__ float gelu(float z)
{
    const float c = 0.7978845608028654f;   // sqrt(2 / pi)
    return 0.5f * z * (1.f + tanh_exp(c * (z + 0.044715f * z * z * z)));
}

__device__ __forceinline__ float gelu_grad(float z)
{
    const float c = 0.7978845608028654f;
    const float t = tanh_exp(c * (z + 0.044715f * z * z * z));
    return 0.5f * (1.f + t) + 0.5f * z * (1.f - t * t) * c * (1.f + 3.f * 0.044715f * z * z);
}

__device__ __forceinline__ unsigned pack_bf16x2(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

// Storage element of the network's operands: BF16 on the tensor-core path, FP32 on the
// reference CUDA-core path (used to check the index arithmetic of the kernels tightly).
template <bool BF16> struct Elt;
template <> struct Elt<true> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ T from(float v) { return __float2bfloat16(v); }
    static __device__ __forceinline__ float to(T v) { return __bfloat162float(v); }
};
template <> struct Elt<false> {
    using T = float;
    static __device__ __forceinline__ T from(float v) { return v; }
    static __device__ __forceinline__ float to(T v) { return v; }
};

// One warp: C[16 x 8] += A[16 x K] * B[K x 8], K a multiple of 16, with A(m, k) and B(k, n)
// read through accessors.  The accumulator uses the C-fragment layout of
// mma.m16n8k16 (g = lane / 4, t = lane % 4): c0, c1 = C(g, 2t), C(g, 2t + 1);
// c2, c3 = C(g + 8, 2t), C(g + 8, 2t + 1).  A fragment: {A(g, 2t), A(g, 2t+1)},
// {A(g+8, 2t), ..}, {A(g, 2t+8), ..}, {A(g+8, 2t+8), ..}; B fragment: {B(2t, g), B(2t+1, g)},
// {B(2t+8, g), B(2t+9, g)}.
template <bool BF16, class FA, class FB>
__device__ __forceinline__ void tile16x8(FA A, FB B, int K, float c[4])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    if constexpr (BF16) {
        for (int k0 = 0; k0 < K; k0 += 16) {
            const unsigned a0 = pack_bf16x2(A(g, k0 + 2 * t), A(g, k0 + 2 * t + 1));
            const unsigned a1 = pack_bf16x2(A(g + 8, k0 + 2 * t), A(g + 8, k0 + 2 * t + 1));
            const unsigned a2 = pack_bf16x2(A(g, k0 + 2 * t + 8), A(g, k0 + 2 * t + 9));
            const unsigned a3 = pack_bf16x2(A(g + 8, k0 + 2 * t + 8), A(g + 8, k0 + 2 * t + 9));
            const unsigned b0 = pack_bf16x2(B(k0 + 2 * t, g), B(k0 + 2 * t + 1, g));
            const unsigned b1 = pack_bf16x2(B(k0 + 2 * t + 8, g), B(k0 + 2 * t + 9, g));
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
    } else {
        for (int k = 0; k < K; ++k) {
            const float x0 = A(g, k), x1 = A(g + 8, k);
            const float y0 = B(k, 2 * t), y1 = B(k, 2 * t + 1);
            c[0] = fmaf(x0, y0, c[0]);
            c[1] = fmaf(x0, y1, c[1]);
            c[2] = fmaf(x1, y0, c[2]);
            c[3] = fmaf(x1, y1, c[3]);
        }
    }
}

// Output of the BF16 network for ONE feature row f (80 FP32 values in shared memory), computed
// by one full warp on the tensor cores as the first row of a 16-row tile whose other rows are
// zero.  The rounding points and the summation order of the last layer are those of the
// training kernel's forward pass, so both give the same value for the same row.  P: the FP32
// parameter vector in global memory; h: 128 floats of shared scratch.
__device__ __forceinline__ float infer_row_bf16(const float *__restrict__ P, const float *f,
                                                float *h)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    for (int n0 = 0; n0 < kHid; n0 += 8) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        tile16x8<true>([&](int m, int k) {
                           return m == 0 ? __float2bfloat16(standardise(P, f[k], k)) : zero; },
                       [&](int k, int n) { return __float2bfloat16(P[kOffW1 + (n0 + n) * kIn + k]); },
                       kIn, c);
        if (g == 0) {
            h[n0 + 2 * t] = c[0] + P[kOffB1 + n0 + 2 * t];
            h[n0 + 2 * t + 1] = c[1] + P[kOffB1 + n0 + 2 * t + 1];
        }
    }
    __syncwarp();
    for (int j = lane; j < kHid; j += 32) h[kHid + j] = __bfloat162float(__float2bfloat16(gelu(h[j])));
    __syncwarp();
    for (int n0 = 0; n0 < kHid; n0 += 8) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        tile16x8<true>([&](int m, int k) { return m == 0 ? __float2bfloat16(h[kHid + k]) : zero; },
                       [&](int k, int n) { return __float2bfloat16(P[kOffW2 + (n0 + n) * kHid + k]); },
                       kHid, c);
        __syncwarp();
        if (g == 0) {
            h[n0 + 2 * t] = c[0] + P[kOffB2 + n0 + 2 * t];
            h[n0 + 2 * t + 1] = c[1] + P[kOffB2 + n0 + 2 * t + 1];
        }
    }
    __syncwarp();
    const float a0 = __bfloat162float(__float2bfloat16(gelu(h[lane])));
    const float a1 = __bfloat162float(__float2bfloat16(gelu(h[lane + 32])));
    float p = a0 * __bfloat162float(__float2bfloat16(P[kOffW3 + lane])) +
              a1 * __bfloat162float(__float2bfloat16(P[kOffW3 + lane + 32]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    return p + P[kOffB3];
}

}  // namespace mlp
}  // namespace ct
