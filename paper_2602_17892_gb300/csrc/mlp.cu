// Training and batch inference of the learned-lambda network (not in the paper; layout and
// rounding in mlp_dev.cuh).
//
// One CTA of 128 threads owns 64 samples (4 warps x 16 rows).  Every matrix product of the
// forward and backward passes is a sequence of 16 x 8 warp tiles: BF16 operands on the tensor
// cores (mma.sync m16n8k16, FP32 accumulation) or, in the FP32 mode, the same tiles on the
// CUDA cores.  The backward pass writes one partial gradient per CTA and a second kernel adds
// the partials in a fixed order, so a training run is deterministic.  Adam keeps FP32 master
// weights and moments.
#include "ct_internal.h"
#include "mlp_dev.cuh"

namespace ct {

using namespace mlp;
constexpr int kRows = 64, kMlpThreads = 128;

template <bool BF16> struct MlpShared {
    using T = typename Elt<BF16>::T;
    T X[kRows][kIn + 8];      // the CTA's input rows
    T W1[kHid][kIn + 8];
    T W2[kHid][kHid + 8];
    T A1[kRows][kHid + 8];    // GELU(z1), the input of layer 2
    T A2[kRows][kHid + 8];
    T D2[kRows][kHid + 8];    // dL/dz2
    T D1[kRows][kHid + 8];    // dL/dz1
    float Z1[kRows][kHid + 1];
    float Z2[kRows][kHid + 1];
    float b1[kHid], b2[kHid], w3[kHid], b3;
    float dout[kRows];
    float red[kMlpThreads];
};

template <bool BF16>
__device__ void mlp_load(MlpShared<BF16> &S, const float *__restrict__ P,
                         const float *__restrict__ X, int n, int row0)
{
    using E = Elt<BF16>;
    const int tid = threadIdx.x;
    for (int i = tid; i < kHid * kIn; i += kMlpThreads) S.W1[i / kIn][i % kIn] = E::from(P[kOffW1 + i]);
    for (int i = tid; i < kHid * kHid; i += kMlpThreads)
        S.W2[i / kHid][i % kHid] = E::from(P[kOffW2 + i]);
    for (int i = tid; i < kHid; i += kMlpThreads) {
        S.b1[i] = P[kOffB1 + i];
        S.b2[i] = P[kOffB2 + i];
        S.w3[i] = E::to(E::from(P[kOffW3 + i]));
    }
    if (tid == 0) S.b3 = P[kOffB3];
    for (int i = tid; i < kRows * kIn; i += kMlpThreads) {
        const int r = i / kIn, c = i % kIn, row = row0 + r;
        S.X[r][c] = E::from(row < n ? standardise(P, X[(int64_t)row * kIn + c], c) : 0.f);
    }
    __syncthreads();
}

// Forward pass of the CTA's rows: warp w owns rows 16w..16w+15; outputs to S.dout.
template <bool BF16> __device__ void mlp_forward_cta(MlpShared<BF16> &S)
{
    using E = Elt<BF16>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int m0 = warp * 16;
    for (int n0 = 0; n0 < kHid; n0 += 8) {                       // z1 = X W1^T + b1
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        tile16x8<BF16>([&](int m, int k) { return S.X[m0 + m][k]; },
                       [&](int k, int n) { return S.W1[n0 + n][k]; }, kIn, c);
        const int r0 = m0 + g, r1 = r0 + 8, cc = n0 + 2 * t;
        S.Z1[r0][cc] = c[0] + S.b1[cc];
        S.Z1[r0][cc + 1] = c[1] + S.b1[cc + 1];
        S.Z1[r1][cc] = c[2] + S.b1[cc];
        S.Z1[r1][cc + 1] = c[3] + S.b1[cc + 1];
    }
    __syncwarp();
    for (int i = lane; i < 16 * kHid; i += 32) {
        const int r = m0 + i / kHid, cc = i % kHid;
        S.A1[r][cc] = E::from(gelu(S.Z1[r][cc]));
    }
    __syncwarp();
    for (int n0 = 0; n0 < kHid; n0 += 8) {                       // z2 = A1 W2^T + b2
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        tile16x8<BF16>([&](int m, int k) { return S.A1[m0 + m][k]; },
                       [&](int k, int n) { return S.W2[n0 + n][k]; }, kHid, c);
        const int r0 = m0 + g, r1 = r0 + 8, cc = n0 + 2 * t;
        S.Z2[r0][cc] = c[0] + S.b2[cc];
        S.Z2[r0][cc + 1] = c[1] + S.b2[cc + 1];
        S.Z2[r1][cc] = c[2] + S.b2[cc];
        S.Z2[r1][cc + 1] = c[3] + S.b2[cc + 1];
    }
    __syncwarp();
    for (int i = lane; i < 16 * kHid; i += 32) {
        const int r = m0 + i / kHid, cc = i % kHid;
        S.A2[r][cc] = E::from(gelu(S.Z2[r][cc]));
    }
    __syncwarp();
    for (int rr = 0; rr < 16; ++rr) {                             // out = A2 w3 + b3
        const int r = m0 + rr;
        float p = E::to(S.A2[r][lane]) * S.w3[lane] + E::to(S.A2[r][lane + 32]) * S.w3[lane + 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
        if (lane == 0) S.dout[r] = p + S.b3;
    }
    __syncthreads();
}

template <bool BF16>
__global__ void __launch_bounds__(kMlpThreads) mlp_forward_kernel(
    const float *__restrict__ P, const float *__restrict__ X, int n, float *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    MlpShared<BF16> &S = *reinterpret_cast<MlpShared<BF16> *>(smraw);
    const int row0 = blockIdx.x * kRows;
    mlp_load(S, P, X, n, row0);
    mlp_forward_cta(S);
    for (int r = threadIdx.x; r < kRows; r += kMlpThreads)
        if (row0 + r < n) out[row0 + r] = S.dout[r];
}

// Mean-squared error over n samples: forward and backward of the CTA's rows.  The CTA's
// partial gradient goes to part[blockIdx.x][kNParams], its partial sum of squared errors to
// lpart[blockIdx.x].
template <bool BF16>
__global__ void __launch_bounds__(kMlpThreads) mlp_grad_kernel(
    const float *__restrict__ P, const float *__restrict__ X, const float *__restrict__ Y, int n,
    float *__restrict__ part, float *__restrict__ lpart)
{
    using E = Elt<BF16>;
    extern __shared__ __align__(16) unsigned char smraw[];
    MlpShared<BF16> &S = *reinterpret_cast<MlpShared<BF16> *>(smraw);
    const int row0 = blockIdx.x * kRows;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    mlp_load(S, P, X, n, row0);
    mlp_forward_cta(S);
    float *G = part + (int64_t)blockIdx.x * kNParams;
    // dL/dout = 2 (out - y) / n, zero on padding rows
    float lacc = 0.f;
    for (int r = tid; r < kRows; r += kMlpThreads) {
        const int row = row0 + r;
        float d = 0.f;
        if (row < n) {
            const float e = S.dout[r] - Y[row];
            lacc += e * e;
            d = 2.f * e / (float)n;
        }
        S.dout[r] = d;
    }
    S.red[tid] = lacc;
    __syncthreads();
    if (tid == 0) {
        float s = 0.f;
        for (int i = 0; i < kMlpThreads; ++i) s += S.red[i];
        lpart[blockIdx.x] = s;
    }
    // layer 3: dw3 = A2^T dout, db3 = sum dout; dz2 = (dout w3^T) .* gelu'(z2)
    for (int j = tid; j < kHid; j += kMlpThreads) {
        float s = 0.f;
        for (int r = 0; r < kRows; ++r) s += S.dout[r] * E::to(S.A2[r][j]);
        G[kOffW3 + j] = s;
    }
    if (tid == 0) {
        float s = 0.f;
        for (int r = 0; r < kRows; ++r) s += S.dout[r];
        G[kOffB3] = s;
    }
    for (int i = tid; i < kRows * kHid; i += kMlpThreads) {
        const int r = i / kHid, j = i % kHid;
        S.D2[r][j] = E::from(S.dout[r] * S.w3[j] * gelu_grad(S.Z2[r][j]));
    }
    __syncthreads();
    // layer 2: dW2 = D2^T A1 (warp w: rows 16w..16w+15 of dW2), db2 = column sums of D2
    for (int n0 = 0; n0 < kHid; n0 += 8) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        tile16x8<BF16>([&](int m, int k) { return S.D2[k][warp * 16 + m]; },
                       [&](int k, int nn) { return S.A1[k][n0 + nn]; }, kRows, c);
        const int r0 = warp * 16 + g, r1 = r0 + 8, cc = n0 + 2 * t;
        G[kOffW2 + r0 * kHid + cc] = c[0];
        G[kOffW2 + r0 * kHid + cc + 1] = c[1];
        G[kOffW2 + r1 * kHid + cc] = c[2];
        G[kOffW2 + r1 * kHid + cc + 1] = c[3];
    }
    for (int j = tid; j < kHid; j += kMlpThreads) {
        float s = 0.f;
        for (int r = 0; r < kRows; ++r) s += E::to(S.D2[r][j]);
        G[kOffB2 + j] = s;
    }
    // dz1 = (D2 W2) .* gelu'(z1) (warp w: its own 16 sample rows)
    for (int n0 = 0; n0 < kHid; n0 += 8) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        tile16x8<BF16>([&](int m, int k) { return S.D2[warp * 16 + m][k]; },
                       [&](int k, int nn) { return S.W2[k][n0 + nn]; }, kHid, c);
        const int r0 = warp * 16 + g, r1 = r0 + 8, cc = n0 + 2 * t;
        S.D1[r0][cc] = E::from(c[0] * gelu_grad(S.Z1[r0][cc]));
        S.D1[r0][cc + 1] = E::from(c[1] * gelu_grad(S.Z1[r0][cc + 1]));
        S.D1[r1][cc] = E::from(c[2] * gelu_grad(S.Z1[r1][cc]));
        S.D1[r1][cc + 1] = E::from(c[3] * gelu_grad(S.Z1[r1][cc + 1]));
    }
    __syncthreads();
    // layer 1: dW1 = D1^T X, db1 = column sums of D1
    for (int n0 = 0; n0 < kIn; n0 += 8) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        tile16x8<BF16>([&](int m, int k) { return S.D1[k][warp * 16 + m]; },
                       [&](int k, int nn) { return S.X[k][n0 + nn]; }, kRows, c);
        const int r0 = warp * 16 + g, r1 = r0 + 8, cc = n0 + 2 * t;
        G[kOffW1 + r0 * kIn + cc] = c[0];
        G[kOffW1 + r0 * kIn + cc + 1] = c[1];
        G[kOffW1 + r1 * kIn + cc] = c[2];
        G[kOffW1 + r1 * kIn + cc + 1] = c[3];
    }
    for (int j = tid; j < kHid; j += kMlpThreads) {
        float s = 0.f;
        for (int r = 0; r < kRows; ++r) s += E::to(S.D1[r][j]);
        G[kOffB1 + j] = s;
    }
    // the standardisation is fixed: zero gradient (Adam then leaves it unchanged)
    for (int j = tid; j < 2 * kIn; j += kMlpThreads) G[kOffMu + j] = 0.f;
}

// grad[i] = sum over CTAs of part[b][i] in CTA order; loss = (sum of lpart) / n
__global__ void mlp_reduce_kernel(const float *__restrict__ part, int nblk,
                                  const float *__restrict__ lpart, int n, float *__restrict__ grad,
                                  float *__restrict__ loss)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParams; i += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * kNParams + i];
        grad[i] = s;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && loss) {
        float s = 0.f;
        for (int b = 0; b < nblk; ++b) s += lpart[b];
        *loss = s / (float)n;
    }
}

// Adam with bias correction (c1 = 1 - beta1^t, c2 = 1 - beta2^t)
__global__ void mlp_adam_kernel(float *__restrict__ P, const float *__restrict__ G,
                                float *__restrict__ M, float *__restrict__ V, float lr, float b1,
                                float b2, float eps, float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParams; i += gridDim.x * blockDim.x) {
        const float g = G[i];
        const float m = b1 * M[i] + (1.f - b1) * g;
        const float v = b2 * V[i] + (1.f - b2) * g * g;
        M[i] = m;
        V[i] = v;
        P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

int mlp_num_params() { return kNParams; }
int mlp_rows_per_block() { return kRows; }

static cudaError_t mlp_set_attrs()
{
    static bool done[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (done[dev]) return cudaSuccess;
    const int s16 = (int)sizeof(MlpShared<true>), s32 = (int)sizeof(MlpShared<false>);
    if ((e = cudaFuncSetAttribute(mlp_forward_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s16)) ||
        (e = cudaFuncSetAttribute(mlp_grad_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s16)) ||
        (e = cudaFuncSetAttribute(mlp_forward_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32)) ||
        (e = cudaFuncSetAttribute(mlp_grad_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32)))
        return e;
    done[dev] = true;
    return cudaSuccess;
}

cudaError_t mlp_prepare() { return mlp_set_attrs(); }

cudaError_t launch_mlp_forward(const float *P, const float *X, int n, float *out, bool bf16,
                               cudaStream_t s)
{
    cudaError_t e = mlp_set_attrs();
    if (e != cudaSuccess) return e;
    const int nblk = (n + kRows - 1) / kRows;
    if (bf16)
        mlp_forward_kernel<true><<<nblk, kMlpThreads, sizeof(MlpShared<true>), s>>>(P, X, n, out);
    else
        mlp_forward_kernel<false><<<nblk, kMlpThreads, sizeof(MlpShared<false>), s>>>(P, X, n, out);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const float *P, const float *X, const float *Y, int n, float *part,
                            float *lpart, float *grad, float *loss, bool bf16, cudaStream_t s)
{
    cudaError_t e = mlp_set_attrs();
    if (e != cudaSuccess) return e;
    const int nblk = (n + kRows - 1) / kRows;
    if (bf16)
        mlp_grad_kernel<true><<<nblk, kMlpThreads, sizeof(MlpShared<true>), s>>>(P, X, Y, n, part, lpart);
    else
        mlp_grad_kernel<false><<<nblk, kMlpThreads, sizeof(MlpShared<false>), s>>>(P, X, Y, n, part, lpart);
    mlp_reduce_kernel<<<(kNParams + 255) / 256, 256, 0, s>>>(part, nblk, lpart, n, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float *P, const float *G, float *M, float *V, float lr, int t,
                            cudaStream_t s)
{
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - pow(b1, (double)t)), c2 = (float)(1.0 - pow(b2, (double)t));
    mlp_adam_kernel<<<(kNParams + 255) / 256, 256, 0, s>>>(P, G, M, V, lr, (float)b1, (float)b2,
                                                           1e-8f, c1, c2);
    return cudaGetLastError();
}

}  // namespace ct
