// The normalized cumulative periodogram (NCP) stopping rule (Sec. 3.2) on the device.
//
// The paper names the NCP beside the discrepancy principle and residual norm stagnation: it
// asks whether the residual looks like white noise, through its power spectrum, without
// knowing the noise level.  Hansen's definition, applied here to the data-space residual
// r_k = b - A x_k split into detector rows (each row a 1-D signal of n = n_det_u bins):
//     p_j = |sum_t r_t exp(-2 pi i j t / n)|^2,        j = 1 .. q, q = floor(n / 2)
//     c_i = (p_1 + ... + p_i) / (p_1 + ... + p_q),     i = 1 .. q
// (the zero frequency, the row's mean, is left out).  The rows' NCPs are averaged (rows
// without power are left out) and the distance ||c - (1..q)/q||_2 from the white-noise line
// is recorded for the step.  The solve stops at the first checked step whose distance is
// larger than the previous checked step's and returns the previous checked step's iterate.
//
// Kernels: ncp_rows_kernel, one block per view: the view's rows are loaded (r = b - A x, from
// the caller's dense b and the padded A x), each row's periodogram is formed by a direct DFT
// from a shared-memory twiddle table (one thread per frequency), scanned, normalised and summed
// over the view's rows; ncp_reduce_kernel averages over all views in a fixed order (FP64),
// forms the distance and applies the stopping rule to the solver's stop word.
#include <cuda_runtime.h>

#include "ct_internal.h"

namespace ct {

namespace {
constexpr int kNcpThreads = 256;
}

// dynamic shared memory: r[n], twiddles[n] (float2), p[q], cacc[q], scan[kNcpThreads / 32]
size_t ncp_smem_bytes(int n)
{
    const int q = n / 2;
    return sizeof(float) * (size_t)(n + 1) + sizeof(float2) * (size_t)n +
           2 * sizeof(float) * (size_t)q + sizeof(float) * 64;
}

__global__ void __launch_bounds__(kNcpThreads) ncp_rows_kernel(
    const float *__restrict__ b, int ndu, int ndv, const float *__restrict__ ax,
    int64_t ax_view_ld, int ax_row0, int ax_ld, const float2 *__restrict__ tw,
    float *__restrict__ part, const int *stop)
{
    if (stop && stop[0] != 0) return;
    extern __shared__ float sm[];
    const int n = ndu, q = n / 2;
    float *r = sm;
    float2 *t = reinterpret_cast<float2 *>(r + n + (n & 1));   // 8-byte aligned
    float *p = reinterpret_cast<float *>(t + n);
    float *cacc = p + q;
    float *wsum = cacc + q;
    const int view = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < n; i += kNcpThreads) t[i] = tw[i];
    for (int i = tid; i < q; i += kNcpThreads) cacc[i] = 0.f;
    float count = 0.f;
    // each thread scans a contiguous chunk of the q periodogram values
    const int per = (q + kNcpThreads - 1) / kNcpThreads;
    const int c0 = min(q, tid * per), c1 = min(q, c0 + per);
    for (int v = 0; v < ndv; ++v) {
        __syncthreads();
        const float *brow = b + ((int64_t)view * ndv + v) * ndu;
        const float *arow = ax + (int64_t)view * ax_view_ld + ax_row0 + (int64_t)v * ax_ld + 2;
        for (int i = tid; i < n; i += kNcpThreads) r[i] = brow[i] - arow[i];
        __syncthreads();
        for (int j = tid + 1; j <= q; j += kNcpThreads) {
            float re = 0.f, im = 0.f;
            int idx = 0;                                   // (j * i) mod n
            for (int i = 0; i < n; ++i) {
                const float2 w = t[idx];
                re = fmaf(r[i], w.x, re);
                im = fmaf(r[i], w.y, im);
                idx += j;
                if (idx >= n) idx -= n;
            }
            p[j - 1] = fmaf(re, re, im * im);
        }
        __syncthreads();
        // inclusive scan of p: chunk sums, a scan over the 256 chunk sums, chunk prefixes
        float s = 0.f;
        for (int i = c0; i < c1; ++i) s += p[i];
        float incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            float ws = lane < kNcpThreads / 32 ? wsum[lane] : 0.f;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float u = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += u;
            }
            if (lane < kNcpThreads / 32) wsum[32 + lane] = ws;   // inclusive over warps
        }
        __syncthreads();
        const float total = wsum[32 + kNcpThreads / 32 - 1];
        if (total > 0.f) {
            const float rt = 1.f / total;
            float run = (incl - s) + (warp > 0 ? wsum[32 + warp - 1] : 0.f);
            for (int i = c0; i < c1; ++i) {
                run += p[i];
                cacc[i] += run * rt;
            }
            count += 1.f;
        }
    }
    __syncthreads();
    float *out = part + (int64_t)view * (q + 1);
    for (int i = tid; i < q; i += kNcpThreads) out[i] = cacc[i];
    if (tid == 0) out[q] = count;
}

// dist[step - 1] = || mean NCP - (1..q)/q ||; then the rule: if a previous check `prev` (> 0)
// exists and the distance grew, stop[0] = prev (its iterate is the one returned).
__global__ void __launch_bounds__(1024) ncp_reduce_kernel(
    const float *__restrict__ part, int n_views, int q, double *dist, int step, int prev,
    int *stop)
{
    if (stop[0] != 0) return;
    __shared__ double red[32];
    __shared__ double cnt_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        double c = 0.0;
        for (int v = 0; v < n_views; ++v) c += (double)part[(int64_t)v * (q + 1) + q];
        cnt_s = c;
    }
    __syncthreads();
    const double cnt = cnt_s;
    double d2 = 0.0;
    if (cnt > 0.0) {
        for (int i = tid; i < q; i += blockDim.x) {
            double c = 0.0;
            for (int v = 0; v < n_views; ++v) c += (double)part[(int64_t)v * (q + 1) + i];
            const double e = c / cnt - (double)(i + 1) / (double)q;
            d2 += e * e;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    if (lane == 0) red[warp] = d2;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) s += red[w];
        const double d = sqrt(s);
        dist[step - 1] = d;
        if (prev > 0 && d > dist[prev - 1]) {
            stop[1] = CT_OK;
            stop[0] = prev;
        }
    }
}

// the row kernel's shared-memory limit on the current device, for the longest row allowed
cudaError_t ncp_prepare(int)
{
    return cudaFuncSetAttribute(ncp_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ncp_smem_bytes(kNcpMaxBins));
}

cudaError_t launch_ncp_check(const ct_geom *g, const float *b, const float *ax_pad,
                             const float2 *tw, float *part, double *dist, int step, int prev,
                             int *stop, cudaStream_t s)
{
    const DeviceGeom &d = g->dg;
    const int n = d.ndu, q = n / 2;
    const size_t smem = ncp_smem_bytes(n);     // limit raised by ncp_prepare at set-up
    ncp_rows_kernel<<<d.n_views, kNcpThreads, smem, s>>>(b, n, d.ndv, ax_pad, d.sino_view_ld,
                                                         d.sino_row0, d.sino_ld, tw, part, stop);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ncp_reduce_kernel<<<1, 1024, 0, s>>>(part, d.n_views, q, dist, step, prev, stop);
    return cudaGetLastError();
}

}  // namespace ct
