// Arnoldi orthogonalisation (Sec. 2.1, Eq. (Hessenberg); Algorithm 1/2 lines 6-11) as
// classical Gram-Schmidt applied twice, plus the basis combination x = x0 + W y of Alg. 1/2
// line 13.
//
// The paper's loop is modified Gram-Schmidt: h_i = <q, w_i>; q -= h_i w_i, one i at a time.
// On a GPU each of those k dot products needs a grid-wide reduction before the next axpy.
// Classical Gram-Schmidt computes all k dots from the same q in one pass over the basis
// (batched dot products, one grid reduction), and the second pass restores orthogonality to
// working precision ("twice is enough"); both give the same H and W in exact arithmetic.
//
// One step is four launches over the basis rows (vectors of L floats, L % 4 == 0, zero tails):
//   K1  h1 = W^T q,          ||q||^2                         (reads W once, last row first)
//   K2  q -= W h1;  h2 = W^T q                              (reads W twice: forwards, backwards)
//   K3  q -= W h2;  ||q||^2 -> h_{k+1,k}, breakdown test      (reads W once, forwards)
//   K4  w_{k+1} = q / h_{k+1,k}
// Each pass starts where the previous one ended, so the rows it needs first are still in L2.
// Block partial sums are FP32 (warp shuffles), the cross-block sum is FP64 in a fixed order
// by the last block to finish, so results are reproducible run to run.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

#include "ct_internal.h"

namespace ct {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr double kBreakdownTol = 1e-6;   // FP32 reading of h_{k+1,k} <= tol ||M w_k||

enum { M_DOTS = 0, M_UPD_DOTS = 1, M_UPD_NORM = 2, M_NORM = 3 };

struct CgsArgs {
    const void *W; int64_t ld; int nvec;        // rows W[0..nvec-1] (storage type T)
    float *q; int64_t L4;                        // vector (float4 count)
    const double *coef;                          // update coefficients (nvec), modes 1, 2
    double *partial; unsigned *counter;
    double *hcol;                                // Hessenberg column (FP64)
    double *aux;                                 // [0] ||q_pre|| [1] 1/h [2] beta, coef buffers
    double *coef_out;                            // where this pass's dots go (modes 0, 1)
    int *stop;                                   // [0] stop step, [1] reason
    int step;                                    // 1-based Arnoldi step (mode 2)
};

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int kGroup = 8;   // basis rows handled together: 8 independent loads in flight

// row index of position p in a pass over n rows, forwards or backwards
__device__ __forceinline__ int row_at(int p, int n, bool backwards) { return backwards ? n - 1 - p : p; }

// Loads and stores of 4 consecutive basis entries in the storage type of the basis; the
// arithmetic is FP32 in every case.
template <typename T> struct BasisIO;
template <> struct BasisIO<float> {
    static __device__ __forceinline__ float4 load(const void *W, int64_t i4)
    {
        return __ldg(reinterpret_cast<const float4 *>(W) + i4);
    }
    static __device__ __forceinline__ float4 store(void *W, int64_t i4, float4 v)
    {
        reinterpret_cast<float4 *>(W)[i4] = v;
        return v;
    }
};
template <> struct BasisIO<__nv_bfloat16> {
    static __device__ __forceinline__ float4 load(const void *W, int64_t i4)
    {
        uint2 r = __ldg(reinterpret_cast<const uint2 *>(W) + i4);
        float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r.x));
        float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ float4 store(void *W, int64_t i4, float4 v)
    {
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
        uint2 r;
        r.x = *reinterpret_cast<unsigned *>(&a);
        r.y = *reinterpret_cast<unsigned *>(&b);
        reinterpret_cast<uint2 *>(W)[i4] = r;
        float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);      // the value actually stored
    }
};
template <> struct BasisIO<__half> {
    static __device__ __forceinline__ float4 load(const void *W, int64_t i4)
    {
        uint2 r = __ldg(reinterpret_cast<const uint2 *>(W) + i4);
        float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&r.x));
        float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&r.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ float4 store(void *W, int64_t i4, float4 v)
    {
        __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
        uint2 r;
        r.x = *reinterpret_cast<unsigned *>(&a);
        r.y = *reinterpret_cast<unsigned *>(&b);
        reinterpret_cast<uint2 *>(W)[i4] = r;
        float2 fa = __half22float2(a), fb = __half22float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
};

template <int MODE, typename T = float>
__global__ void __launch_bounds__(kThreads) cgs_kernel(CgsArgs a)
{
    if (a.stop[0] != 0) return;
    extern __shared__ float sm[];
    const int nvec = (MODE == M_NORM) ? 0 : a.nvec;
    const int ncol = nvec + 1;                       // dots + squared norm
    const int nvec8 = (nvec + kGroup - 1) / kGroup * kGroup;
    float *scoef = sm;                               // nvec8 (zero padded)
    float *acc = sm + nvec8;                         // [kWarps][ncol]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < kWarps * ncol; i += kThreads) acc[i] = 0.f;
    if (MODE == M_UPD_DOTS || MODE == M_UPD_NORM)
        for (int i = tid; i < nvec8; i += kThreads) scoef[i] = (i < nvec) ? (float)a.coef[i] : 0.f;
    __syncthreads();
    // Passes alternate direction so that each one starts on the rows the previous pass read
    // last (still in L2): K1 dots backwards, K2 update forwards then dots backwards, K3 forwards.
    const bool dots_backwards = true;
    float4 *q4 = reinterpret_cast<float4 *>(a.q);
    const int64_t ld4 = a.ld / 4;
    for (int64_t e0 = (int64_t)blockIdx.x * kThreads; e0 < a.L4; e0 += (int64_t)gridDim.x * kThreads) {
        const int64_t e = e0 + tid;
        const bool ok = e < a.L4;
        float4 v = ok ? q4[e] : make_float4(0.f, 0.f, 0.f, 0.f);
        // rows of a group in flight while the previous group is consumed (software pipeline)
        auto load_group = [&](float4 *buf, int p0, bool backwards) {
#pragma unroll
            for (int u = 0; u < kGroup; ++u)
                buf[u] = (ok && p0 + u < nvec)
                             ? BasisIO<T>::load(a.W, (int64_t)row_at(p0 + u, nvec, backwards) * ld4 + e)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        if (MODE == M_UPD_DOTS || MODE == M_UPD_NORM) {
            float4 wb[kGroup], wn[kGroup];
            load_group(wb, 0, false);
            for (int p0 = 0; p0 < nvec; p0 += kGroup) {
                if (p0 + kGroup < nvec) load_group(wn, p0 + kGroup, false);
#pragma unroll
                for (int u = 0; u < kGroup; ++u) {
                    const float c = scoef[p0 + u];          // zero beyond nvec
                    v.x = fmaf(-c, wb[u].x, v.x); v.y = fmaf(-c, wb[u].y, v.y);
                    v.z = fmaf(-c, wb[u].z, v.z); v.w = fmaf(-c, wb[u].w, v.w);
                }
#pragma unroll
                for (int u = 0; u < kGroup; ++u) wb[u] = wn[u];
            }
            if (ok) q4[e] = v;
        }
        if (MODE == M_DOTS || MODE == M_UPD_DOTS) {
            float4 wb[kGroup], wn[kGroup];
            load_group(wb, 0, dots_backwards);
            for (int p0 = 0; p0 < nvec; p0 += kGroup) {
                if (p0 + kGroup < nvec) load_group(wn, p0 + kGroup, dots_backwards);
                float pd[kGroup];
#pragma unroll
                for (int u = 0; u < kGroup; ++u)
                    pd[u] = fmaf(wb[u].x, v.x, fmaf(wb[u].y, v.y, fmaf(wb[u].z, v.z, wb[u].w * v.w)));
                // transpose reduction: after the xor-16/8/4 exchange stages lane l holds a partial
                // sum of group row (l >> 2) over 8 lanes; xor-2/1 complete it (9 shuffles for 8 rows)
                const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
                float q4v[4], q2v[2], q1;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float send = b4 ? pd[j] : pd[j + 4];
                    float keep = b4 ? pd[j + 4] : pd[j];
                    q4v[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    float send = b3 ? q4v[j] : q4v[j + 2];
                    float keep = b3 ? q4v[j + 2] : q4v[j];
                    q2v[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
                }
                {
                    float send = b2 ? q2v[0] : q2v[1];
                    float keep = b2 ? q2v[1] : q2v[0];
                    q1 = keep + __shfl_xor_sync(0xffffffffu, send, 4);
                }
                q1 += __shfl_xor_sync(0xffffffffu, q1, 2);
                q1 += __shfl_xor_sync(0xffffffffu, q1, 1);
                const int pr = p0 + (lane >> 2);
                if ((lane & 3) == 0 && pr < nvec) acc[warp * ncol + row_at(pr, nvec, dots_backwards)] += q1;
#pragma unroll
                for (int u = 0; u < kGroup; ++u) wb[u] = wn[u];
            }
        }
        float nn = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, v.w * v.w)));
        nn = warp_sum(nn);
        if (lane == 0) acc[warp * ncol + nvec] += nn;
    }
    __syncthreads();
    double *prow = a.partial + (int64_t)blockIdx.x * ncol;
    for (int i = tid; i < ncol; i += kThreads) {
        float s = 0.f;
        for (int w = 0; w < kWarps; ++w) s += acc[w * ncol + i];
        prow[i] = (double)s;
    }
    // last block to finish reduces across blocks in a fixed order
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (tid == 0) is_last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    __shared__ double total_nn;
    // column i is summed by warp i % kWarps: lane l adds blocks l, l + 32, ... and the warp's
    // lanes are then added by a fixed xor tree (a fixed order: reproducible run to run)
    for (int i = warp; i < ncol; i += kWarps) {
        double s = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32)
            s += ((volatile double *)a.partial)[(int64_t)b * ncol + i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            if (i < nvec) {
                if (MODE == M_DOTS) { a.hcol[i] = s; a.coef_out[i] = s; }
                if (MODE == M_UPD_DOTS) { a.hcol[i] += s; a.coef_out[i] = s; }
            } else {
                total_nn = s;
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        double nrm = sqrt(total_nn);
        if (MODE == M_DOTS) a.aux[0] = nrm;
        if (MODE == M_UPD_NORM) {
            a.hcol[nvec] = nrm;
            if (!isfinite(nrm)) { a.stop[0] = a.step; a.stop[1] = CT_ENONFINITE; a.aux[1] = 0.0; }
            else if (!(nrm > kBreakdownTol * a.aux[0])) { a.stop[0] = a.step; a.stop[1] = CT_BREAKDOWN; a.aux[1] = 0.0; }
            else a.aux[1] = 1.0 / nrm;
        }
        if (MODE == M_NORM) {
            a.aux[2] = nrm;
            if (!isfinite(nrm)) { a.stop[0] = -1; a.stop[1] = CT_ENONFINITE; a.aux[1] = 0.0; }
            else if (nrm == 0.0) { a.stop[0] = -1; a.stop[1] = CT_BREAKDOWN; a.aux[1] = 0.0; }
            else a.aux[1] = 1.0 / nrm;
        }
        *a.counter = 0u;
    }
}

// dst = src * aux[1] rounded to the basis type (normalisation; skipped once a stop is
// recorded); `cur` (optional) receives the stored values in FP32 for the next operator call.
template <typename T>
__global__ void scale_kernel(const float4 *__restrict__ src, void *__restrict__ dst, int64_t L4,
                             const double *aux, const int *stop, float4 *__restrict__ cur)
{
    if (stop[0] != 0) return;
    const float s = (float)aux[1];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L4;
         e += (int64_t)gridDim.x * blockDim.x) {
        float4 v = src[e];
        v.x *= s; v.y *= s; v.z *= s; v.w *= s;
        float4 st = BasisIO<T>::store(dst, e, v);
        if (cur) cur[e] = st;
    }
}

static int grid_for(int64_t L4, int max_blocks)
{
    int64_t b = (L4 + kThreads - 1) / kThreads;
    if (b > max_blocks) b = max_blocks;
    if (b < 1) b = 1;
    return (int)b;
}

// Blocks of the Gram-Schmidt kernels that are resident at once on the device (one wave): a
// grid larger than that leaves a partial second wave as a tail, so the grid is capped to it and
// the kernels' element loop takes the rest.  Queried once per device for the largest kernel.
static int cgs_wave_blocks()
{
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152 * 2;
    if (!cached[dev]) {
        int per_sm = 0, sms = 0;
        const size_t smem = sizeof(float) * (size_t)(168 + kWarps * 169);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cgs_kernel<M_UPD_DOTS, float>,
                                                          kThreads, smem) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            per_sm < 1 || sms < 1) {
            per_sm = 2;
            sms = 152;
        }
        cached[dev] = per_sm * sms;
    }
    return cached[dev];
}

// Caches the one-wave grid of the Gram-Schmidt kernels for the current device (call before a
// stream capture).
cudaError_t arnoldi_prepare()
{
    return cgs_wave_blocks() > 0 ? cudaSuccess : cudaErrorUnknown;
}

// One CGS2 Arnoldi step on rows W[0..k] (storage type T) with q = M w_k; writes the H column
// (FP64, k+2 entries), W[k+1] and, when `cur` is not null, W[k+1] in FP32.  `aux` / `stop` are
// device scratch words (see CgsArgs).
template <typename T>
static cudaError_t arnoldi_step_t(void *W, int64_t L, int64_t ld, int k, float *q, double *hcol,
                                  const ArnoldiScratch &sc, double *aux, int *stop, int step,
                                  bool reorth, float *cur, cudaStream_t s)
{
    const int64_t L4 = L / 4;
    const int nvec = k + 1;
    const int blocks = grid_for(L4, std::min(sc.max_blocks, cgs_wave_blocks()));
    double *h1 = aux + 8, *h2 = aux + 8 + (sc.kmax + 2);
    CgsArgs a{W, ld, nvec, q, L4, nullptr, sc.partial, sc.counter, hcol, aux, h1, stop, step};
    size_t smem = sizeof(float) * (size_t)((nvec + 7) / 8 * 8 + kWarps * (nvec + 1));
    cgs_kernel<M_DOTS, T><<<blocks, kThreads, smem, s>>>(a);
    if (reorth) {
        a.coef = h1; a.coef_out = h2;
        cgs_kernel<M_UPD_DOTS, T><<<blocks, kThreads, smem, s>>>(a);
        a.coef = h2;
    } else {
        a.coef = h1;
    }
    cgs_kernel<M_UPD_NORM, T><<<blocks, kThreads, smem, s>>>(a);
    const size_t esz = sizeof(T);
    scale_kernel<T><<<grid_for(L4, sc.max_blocks), kThreads, 0, s>>>(
        reinterpret_cast<const float4 *>(q), static_cast<char *>(W) + (size_t)(k + 1) * ld * esz,
        L4, aux, stop, reinterpret_cast<float4 *>(cur));
    return cudaGetLastError();
}

cudaError_t arnoldi_step_dev(float *W, int64_t L, int64_t ld, int k, float *q, double *hcol,
                             const ArnoldiScratch &sc, double *aux, int *stop, int step,
                             bool reorth, cudaStream_t s)
{
    return arnoldi_step_t<float>(W, L, ld, k, q, hcol, sc, aux, stop, step, reorth, nullptr, s);
}

cudaError_t arnoldi_step_basis(int basis, void *W, int64_t L, int64_t ld, int k, float *q,
                               double *hcol, const ArnoldiScratch &sc, double *aux, int *stop,
                               int step, bool reorth, float *cur, cudaStream_t s)
{
    switch (basis) {
    case CT_BASIS_BF16:
        return arnoldi_step_t<__nv_bfloat16>(W, L, ld, k, q, hcol, sc, aux, stop, step, reorth, cur, s);
    case CT_BASIS_F16:
        return arnoldi_step_t<__half>(W, L, ld, k, q, hcol, sc, aux, stop, step, reorth, cur, s);
    default:
        return arnoldi_step_t<float>(W, L, ld, k, q, hcol, sc, aux, stop, step, reorth, cur, s);
    }
}

// beta = ||r||, w0 = r / beta (Alg. 1/2 line 3) in the basis type; beta stored in aux[2].
cudaError_t normalize_first_basis(int basis, const float *r, int64_t L, void *w0,
                                  const ArnoldiScratch &sc, double *aux, int *stop, float *cur,
                                  cudaStream_t s)
{
    const int64_t L4 = L / 4;
    const int blocks = grid_for(L4, sc.max_blocks);
    CgsArgs a{nullptr, L, 0, const_cast<float *>(r), L4, nullptr, sc.partial, sc.counter,
              nullptr, aux, nullptr, stop, 0};
    size_t smem = sizeof(float) * (size_t)(kWarps);
    cgs_kernel<M_NORM><<<blocks, kThreads, smem, s>>>(a);
    const float4 *r4 = reinterpret_cast<const float4 *>(r);
    float4 *c4 = reinterpret_cast<float4 *>(cur);
    if (basis == CT_BASIS_BF16)
        scale_kernel<__nv_bfloat16><<<blocks, kThreads, 0, s>>>(r4, w0, L4, aux, stop, c4);
    else if (basis == CT_BASIS_F16)
        scale_kernel<__half><<<blocks, kThreads, 0, s>>>(r4, w0, L4, aux, stop, c4);
    else
        scale_kernel<float><<<blocks, kThreads, 0, s>>>(r4, w0, L4, aux, stop, c4);
    return cudaGetLastError();
}

cudaError_t normalize_first(const float *r, int64_t L, float *w0, const ArnoldiScratch &sc,
                            double *aux, int *stop, cudaStream_t s)
{
    return normalize_first_basis(CT_BASIS_F32, r, L, w0, sc, aux, stop, nullptr, s);
}

// ----------------------------------------------------------------------------- x = x0 + W y
// y holds K slots of K doubles; the slot of the last valid step kf = stop ? stop : K is used.
template <typename T>
__global__ void __launch_bounds__(kThreads) combine_kernel(
    const void *__restrict__ W, int64_t ld4, int64_t L4, const double *__restrict__ Y, int K,
    int ystride, const int *stop, int kfixed, const float4 *__restrict__ x0, float4 *__restrict__ x)
{
    __shared__ float sy[1024];
    int kf = kfixed;
    if (stop) {
        int st = stop[0];
        kf = (st == 0) ? K : (st < 0 ? 0 : st);
    }
    const double *y = Y + (int64_t)(kf > 0 ? kf - 1 : 0) * ystride;
    for (int i = threadIdx.x; i < kf; i += kThreads) sy[i] = (float)y[i];
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)kThreads + threadIdx.x; e < L4;
         e += (int64_t)gridDim.x * kThreads) {
        float4 v = x0 ? x0[e] : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = 0; i < kf; ++i) {
            float4 w = BasisIO<T>::load(W, i * ld4 + e);
            float c = sy[i];
            v.x = fmaf(c, w.x, v.x); v.y = fmaf(c, w.y, v.y);
            v.z = fmaf(c, w.z, v.z); v.w = fmaf(c, w.w, v.w);
        }
        x[e] = v;
    }
}

cudaError_t launch_combine_basis(int basis, const void *W, int64_t L, int64_t ld, const double *Y,
                                 int K, int ystride, const int *stop, int kfixed, const float *x0,
                                 float *x, int max_blocks, cudaStream_t s)
{
    const int64_t L4 = L / 4;
    const int g = grid_for(L4, max_blocks);
    const float4 *x04 = reinterpret_cast<const float4 *>(x0);
    float4 *x4 = reinterpret_cast<float4 *>(x);
    if (basis == CT_BASIS_BF16)
        combine_kernel<__nv_bfloat16><<<g, kThreads, 0, s>>>(W, ld / 4, L4, Y, K, ystride, stop, kfixed, x04, x4);
    else if (basis == CT_BASIS_F16)
        combine_kernel<__half><<<g, kThreads, 0, s>>>(W, ld / 4, L4, Y, K, ystride, stop, kfixed, x04, x4);
    else
        combine_kernel<float><<<g, kThreads, 0, s>>>(W, ld / 4, L4, Y, K, ystride, stop, kfixed, x04, x4);
    return cudaGetLastError();
}

cudaError_t launch_combine(const float *W, int64_t L, int64_t ld, const double *Y, int K,
                           int ystride, const int *stop, int kfixed, const float *x0, float *x,
                           int max_blocks, cudaStream_t s)
{
    return launch_combine_basis(CT_BASIS_F32, W, L, ld, Y, K, ystride, stop, kfixed, x0, x,
                                max_blocks, s);
}

// r = b - r  (in place on r), float4 vectors
__global__ void rsub_kernel(const float4 *__restrict__ b, float4 *__restrict__ r, int64_t L4)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L4;
         e += (int64_t)gridDim.x * blockDim.x) {
        float4 u = b[e], v = r[e];
        r[e] = make_float4(u.x - v.x, u.y - v.y, u.z - v.z, u.w - v.w);
    }
}

cudaError_t launch_rsub(const float *b, float *r, int64_t L, int max_blocks, cudaStream_t s)
{
    rsub_kernel<<<grid_for(L / 4, max_blocks), kThreads, 0, s>>>(
        reinterpret_cast<const float4 *>(b), reinterpret_cast<float4 *>(r), L / 4);
    return cudaGetLastError();
}

}  // namespace ct

namespace ct {

// ----------------------------------------------------------------------------- no-allocation variant
// Scratch of ct_arnoldi_step_noalloc: a file-scope device array, so the entry point never
// allocates.  Every GPU that loads the library holds it (about 1.3 MB) until the process exits.
constexpr int kNoAllocMaxK = 126;                    // h has at most k + 2 = 128 entries
constexpr int kNoAllocBlocks = 152 * 8;
constexpr size_t kNoAllocPartial = (size_t)kNoAllocBlocks * (kNoAllocMaxK + 3);   // doubles
constexpr size_t kNoAllocAux = 8 + 2 * (kNoAllocMaxK + 3);                          // doubles
constexpr size_t kNoAllocBytes = (kNoAllocPartial + kNoAllocAux) * sizeof(double) + 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[64] = {nullptr};

}  // namespace ct

extern "C" ct_status ct_arnoldi_step_noalloc(float *W_dev, int64_t len, int64_t ld, int k,
                                             float *q_dev, double *h_dev, ct_stream_t stream)
{
    using namespace ct;
    if (!W_dev || !q_dev || !h_dev) {
        set_error("ct_arnoldi_step_noalloc: null argument");
        return CT_EINVAL;
    }
    if (k < 0 || k > kNoAllocMaxK) {
        set_error("ct_arnoldi_step_noalloc: k = " + std::to_string(k) +
                  " exceeds the static scratch (0 <= k <= " + std::to_string(kNoAllocMaxK) + ")");
        return CT_EINVAL;
    }
    if (len < 1 || ld < len || (len % 4) || (ld % 4)) {
        set_error("ct_arnoldi_step_noalloc: need len % 4 == 0, ld % 4 == 0, ld >= len >= 1");
        return CT_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "ct_arnoldi_step_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) {
        set_error("ct_arnoldi_step_noalloc: device ordinal out of range");
        return CT_EINVAL;
    }
    void *base = nullptr;
    {
        // one-time set-up per device, with that device current: the device address of the
        // static array (its name in host code is only a host-side stand-in)
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            e = cudaGetSymbolAddress(&g_noalloc_ptr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_noalloc_ptr[dev] = nullptr;
                return cuda_fail(e, "ct_arnoldi_step_noalloc: cudaGetSymbolAddress");
            }
        }
        base = g_noalloc_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    double *partial = reinterpret_cast<double *>(base);
    double *aux = partial + kNoAllocPartial;
    unsigned *counter = reinterpret_cast<unsigned *>(aux + kNoAllocAux);
    int *stop = reinterpret_cast<int *>(counter + 4);
    // the array keeps the previous call's contents: clear what must start at zero
    e = cudaMemsetAsync(counter, 0, 4 * sizeof(unsigned) + 4 * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(aux, 0, kNoAllocAux * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h_dev, 0, sizeof(double) * (k + 2), s);
    if (e != cudaSuccess) return cuda_fail(e, "ct_arnoldi_step_noalloc: clearing scratch");
    ArnoldiScratch sc{partial, counter, kNoAllocBlocks, kNoAllocMaxK + 1};
    e = arnoldi_step_dev(W_dev, len, ld, k, q_dev, h_dev, sc, aux, stop, 1, true, s);
    if (e != cudaSuccess) return cuda_fail(e, "ct_arnoldi_step_noalloc: launch");
    return CT_OK;
}
