// Arnoldi orthogonalisation (Sec. 2.1, Eq. (Hessenberg)) as classical Gram-Schmidt applied
// twice, plus the basis combination x = x0 + W y of the hybrid iterate (Sec. 3).
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
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

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

// Sum over blocks b < nblocks of partial[b * ncol + c] by one warp: lane l adds blocks l, l + 32,
// ... in order, the lanes are then added by a fixed xor tree (a fixed order: reproducible run
// to run).  Loads go to L2 (written by other blocks before their fence) in batches of eight.
__device__ __forceinline__ double column_sum(const double *partial, int nblocks, int ncol, int c,
                                             int lane)
{
    double s = 0.0;
    for (int b0 = lane; b0 < nblocks; b0 += 32 * 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int b = b0 + 32 * u;
            v[u] = (b < nblocks) ? __ldcg(partial + (int64_t)b * ncol + c) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) s += v[u];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
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
    // column i is summed by warp i % kWarps (column_sum)
    for (int i = warp; i < ncol; i += kWarps) {
        const double s = column_sum(a.partial, (int)gridDim.x, ncol, i, lane);
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

static cudaError_t tile_prepare();
static int device_sms();

// Caches the one-wave grid of the Gram-Schmidt kernels for the current device and allows the
// tiled kernels their shared memory (call before a stream capture).
cudaError_t arnoldi_prepare()
{
    if (cgs_wave_blocks() <= 0) return cudaErrorUnknown;
    device_sms();
    return tile_prepare();
}

// ============================================================================ tiled CGS2
// The solver's own basis (row stride ld a multiple of 128 elements, q holding ld floats with a
// zero tail) takes a tiled path: a tile is 128 consecutive elements of every basis row (one
// 4-element unit per lane of a warp) plus the same 128 elements of q, copied global -> shared
// memory by the TMA engine (cp.async.bulk, one copy per row segment, completion counted on an
// mbarrier) into a ring of stages, so that several tiles per CTA are in flight while the
// previous one is consumed.  One step is three passes over the basis:
//   T1  h1 = W^T q, ||q||^2                                       (tiles ascending)
//   T2  q' = q - W h1 (written back), h2 = W^T q', ||q'||^2        (tiles descending)
//       -- both from the SAME shared-memory tile, so W is read from memory once --
//   T3  nu = sqrt(||q'||^2 - ||h2||^2) = h_{k+1,k}, breakdown test;
//       w_{k+1} = (q' - W h2) / nu                                 (tiles ascending)
// T1 and T2 leave per-block sums; a small kernel after each adds them across blocks, one warp
// per column with all columns in parallel (a single block doing that serially took longer
// than the pass itself).
// nu uses ||q' - W h2||^2 = ||q'||^2 - 2 h2.W^T q' + h2.W^T W h2 = ||q'||^2 - ||h2||^2 up to
// the basis' loss of orthogonality times ||h2||^2 (h2 is the small second correction).
// Alternating the tile order makes each pass start on the tiles the previous one read last
// (still in L2).  Rows of a tile are split over the 8 warps (row r to warp r % 8) for the
// dots; the updates sum each warp's rows per lane and combine the 8 partial sums in a fixed
// order, so results are reproducible run to run.
constexpr int kTileUnits = 32;                  // 4-element units per tile row (one per lane)
constexpr int kTileElems = 4 * kTileUnits;      // 128 elements
// threads of a tile CTA: the passes stream HBM through TMA copies and their arithmetic is light
// (a few instructions a tile row a warp), so four warps keep up, and a CTA holds half the
// registers that eight would: in a batch the other solve's projector kernels share the SM
constexpr int kTileThreads = 128;
constexpr int kTileWarps = kTileThreads / 32;
constexpr int kTileSmemMax = 220 * 1024;        // dynamic shared memory of one CTA at most
constexpr int kTilePair = 110 * 1024;           // at most this much for two CTAs per SM
constexpr long long kWaitCycles = 1ll << 31;    // bounded mbarrier waits (about a second)
enum { T_DOTS = 0, T_UPD_DOTS = 1, T_UPD_SCALE = 2 };

// Test hook of the bounded waits (off by default, armed only by ct_test_drop_tile_copy): when
// g_drop_tile_copy is set, the next tile pass whose block 0 takes it (atomic exchange) issues
// neither the copies of its first tile nor their expected byte count, so nothing is in flight
// for that stage and its waits run out after g_wait_cycles; the pass then records CT_ETIMEOUT
// in the solver's stop word and returns.
__device__ int g_drop_tile_copy = 0;
__device__ long long g_wait_cycles = kWaitCycles;

struct TileArgs {
    const void *W; int64_t ld; int nvec;         // rows W[0..nvec-1], storage type T
    const float *q; float *qout;                 // q (ld floats); T2 writes q' to qout (= q)
    int ntiles, stages;
    const double *coef;                          // T2: h1, T3: h2
    double *partial; unsigned *counter;
    double *hcol, *aux, *coef_out;               // T1: h1 -> coef_out; T2: h2 -> coef_out;
                                                 // aux[0] ||q||, aux[1] 1 / nu, aux[4] ||q'||^2
    int *stop; int step;
    void *wnext; float *cur;                     // T3: row k+1 of W (type T), FP32 copy
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes) : "memory");
}

// cp.async.bulk global -> shared, completion (bytes) signalled on `bar`; 16-byte aligned
// addresses, size a multiple of 16
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// 2D tiled TMA load of the box at element column x, row 0 of the tensor map into shared
// memory, completion (bytes) signalled on `bar`; x * element size is a multiple of 16 bytes
__device__ __forceinline__ void tensor_g2s(void *dst, const CUtensorMap *map, int x, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(0),
                 "r"(smem_u32(bar)) : "memory");
}

// The same load with an L2 evict-first policy: the basis stream (hundreds of MB per step)
// then gives way in L2 to the projectors' operands (the pair layouts and the ray table, about
// 11 MB at the 512^2 fan workload) that the other solve of a batch reads at the same time
// (measured: 39.8 -> 39.5 ms a step of the AB + BA batch; the passes themselves not slower).
__device__ __forceinline__ void tensor_g2s_ef(void *dst, const CUtensorMap *map, int x, uint64_t *bar)
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
                 " [%0], [%1, {%2, %3}], [%4], %5;"
                 ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(0),
                 "r"(smem_u32(bar)), "l"(pol) : "memory");
}

// waits for phase `parity` of `bar` to complete; false after about `limit` cycles
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, long long limit)
{
    const uint32_t a = smem_u32(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// arms (enable != 0) or disarms the test hook above; while armed the waits give up after
// wait_cycles, disarmed they use the default limit
cudaError_t arnoldi_test_drop_tile_copy(int enable, long long wait_cycles)
{
    const int arm = enable ? 1 : 0;
    const long long lim = enable ? wait_cycles : kWaitCycles;
    cudaError_t e = cudaMemcpyToSymbol(g_wait_cycles, &lim, sizeof(lim));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_drop_tile_copy, &arm, sizeof(arm));
    return e;
}

template <typename T>
__device__ __forceinline__ float4 unit_from_smem(const unsigned char *seg, int lane)
{
    if constexpr (sizeof(T) == 4) {
        return reinterpret_cast<const float4 *>(seg)[lane];
    } else {
        const uint2 r = reinterpret_cast<const uint2 *>(seg)[lane];
        float2 a, b;
        if constexpr (std::is_same<T, __nv_bfloat16>::value) {
            a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r.x));
            b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r.y));
        } else {
            a = __half22float2(*reinterpret_cast<const __half2 *>(&r.x));
            b = __half22float2(*reinterpret_cast<const __half2 *>(&r.y));
        }
        return make_float4(a.x, a.y, b.x, b.y);
    }
}

__device__ __forceinline__ float dot4(float4 a, float4 b)
{
    return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

// shared-memory bytes of one stage: nvec row segments of the basis and one of q
template <typename T>
__host__ __device__ constexpr int tile_stage_bytes(int nvec)
{
    return nvec * kTileElems * (int)sizeof(T) + kTileElems * 4;
}

template <int MODE, typename T>
__global__ void __launch_bounds__(kTileThreads, 2) cgs_tile_kernel(const __grid_constant__ CUtensorMap wmap,
                                                               TileArgs a)
{
    if (a.stop[0] != 0) return;
    extern __shared__ __align__(128) unsigned char tsm[];
    const int nvec = a.nvec, S = a.stages;
    const int seg = kTileElems * (int)sizeof(T);
    const int stage_bytes = tile_stage_bytes<T>(nvec);
    // stages | mbarriers | block sums [nvec + 1] | warp partials [8][32] | q' [32] | coef [nvec]
    // (every region starts on a 16-byte boundary)
    unsigned char *p = tsm + (size_t)S * stage_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(p);
    p += 16 * ((S + 1) / 2);
    float *acc = reinterpret_cast<float *>(p);
    p += 16 * ((nvec + 1 + 3) / 4);
    float4 *red = reinterpret_cast<float4 *>(p);
    float4 *qs = red + kTileWarps * kTileUnits;
    float *scoef = reinterpret_cast<float *>(qs + kTileUnits);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ncol = nvec + 1;
    for (int i = tid; i < ncol; i += kTileThreads) acc[i] = 0.f;
    float inv_nu = 0.f;
    if (MODE == T_UPD_SCALE) {
        // h_{k+1,k} = nu = sqrt(||q'||^2 - ||h2||^2), every block the same value (fixed order);
        // block 0 records it and the breakdown test of the paper's Arnoldi loop
        __shared__ double hsum[kTileWarps];
        double h2 = 0.0;
        for (int i = tid; i < nvec; i += kTileThreads) {
            const double c = a.coef[i];
            h2 = fma(c, c, h2);
            scoef[i] = (float)c;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) h2 += __shfl_xor_sync(0xffffffffu, h2, o);
        if (lane == 0) hsum[warp] = h2;
        __syncthreads();
        double t = 0.0;
        for (int w = 0; w < kTileWarps; ++w) t += hsum[w];
        const double nrm = sqrt(fmax(a.aux[4] - t, 0.0));
        const bool bad = !isfinite(nrm), brk = !(nrm > kBreakdownTol * a.aux[0]);
        if (blockIdx.x == 0 && tid == 0) {
            a.hcol[nvec] = nrm;
            if (bad) { a.stop[0] = a.step; a.stop[1] = CT_ENONFINITE; a.aux[1] = 0.0; }
            else if (brk) { a.stop[0] = a.step; a.stop[1] = CT_BREAKDOWN; a.aux[1] = 0.0; }
            else a.aux[1] = 1.0 / nrm;
        }
        if (bad || brk) return;
        // the solve's last step needs h_{k+1,k} but not w_{k+1}: launched as one block without it
        if (a.wnext == nullptr) return;
        inv_nu = (float)(1.0 / nrm);
    } else if (MODE == T_UPD_DOTS) {
        for (int i = tid; i < nvec; i += kTileThreads) scoef[i] = (float)a.coef[i];
    }
    if (tid == 0) {
        for (int st = 0; st < S; ++st) mbar_init(&bars[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // this CTA's tiles: blockIdx.x + i * gridDim.x, i < nt, in the order of the pass
    const int nt = (a.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    auto tile_of = [&](int i) {
        const int j = (MODE == T_UPD_DOTS) ? nt - 1 - i : i;
        return (int)blockIdx.x + j * (int)gridDim.x;
    };
    // thread 0 issues the copies of tile i into its stage: the nvec x 128 box of the basis (one
    // tensor copy; the map's row extent is nvec) and 128 entries of q (one bulk copy)
    auto issue = [&](int i) {
        const int st = i % S;
        unsigned char *dst = tsm + (size_t)st * stage_bytes;
        const int e0 = tile_of(i) * kTileElems;
        mbar_expect_tx(&bars[st], (unsigned)stage_bytes);
        tensor_g2s_ef(dst, &wmap, e0, &bars[st]);
        bulk_g2s(dst + (size_t)nvec * seg, a.q + e0, kTileElems * 4, &bars[st]);
    };
    const long long wlim = g_wait_cycles;
    if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const bool drop = blockIdx.x == 0 && nt > 0 && atomicExch(&g_drop_tile_copy, 0) != 0;
        for (int i = drop ? 1 : 0; i < S && i < nt; ++i) issue(i);
    }
    bool ok = true;
    float nn = 0.f;                      // lane partial of ||q||^2 (T1) or ||q'||^2 (T2), warp 0
    int i = 0;
    for (; i < nt; ++i) {
        const int st = i % S;
        if (!mbar_wait(&bars[st], (unsigned)((i / S) & 1), wlim)) { ok = false; break; }
        const unsigned char *tileb = tsm + (size_t)st * stage_bytes;
        const float4 qv = reinterpret_cast<const float4 *>(tileb + (size_t)nvec * seg)[lane];
        float4 v = qv;                   // the vector the dots are taken with (q or q')
        if (MODE != T_DOTS) {
            // per-lane sum over this warp's rows of coef_r * W[r], then the 8 warps' sums
            float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int r = warp; r < nvec; r += kTileWarps) {
                const float c = scoef[r];
                const float4 w = unit_from_smem<T>(tileb + (size_t)r * seg, lane);
                u.x = fmaf(c, w.x, u.x); u.y = fmaf(c, w.y, u.y);
                u.z = fmaf(c, w.z, u.z); u.w = fmaf(c, w.w, u.w);
            }
            red[warp * kTileUnits + lane] = u;
            __syncthreads();
            if (warp == 0) {
                float4 t = red[lane];
#pragma unroll
                for (int w = 1; w < kTileWarps; ++w) {
                    const float4 o = red[w * kTileUnits + lane];
                    t.x += o.x; t.y += o.y; t.z += o.z; t.w += o.w;
                }
                float4 r = make_float4(qv.x - t.x, qv.y - t.y, qv.z - t.z, qv.w - t.w);
                const size_t e = (size_t)tile_of(i) * kTileUnits + lane;
                if (MODE == T_UPD_DOTS) {
                    reinterpret_cast<float4 *>(a.qout)[e] = r;
                    qs[lane] = r;
                    nn = fmaf(r.x, r.x, fmaf(r.y, r.y, fmaf(r.z, r.z, fmaf(r.w, r.w, nn))));
                } else {
                    r.x *= inv_nu; r.y *= inv_nu; r.z *= inv_nu; r.w *= inv_nu;
                    const float4 stv = BasisIO<T>::store(a.wnext, (int64_t)e, r);
                    if (a.cur) reinterpret_cast<float4 *>(a.cur)[e] = stv;
                }
            }
            if (MODE == T_UPD_DOTS) {
                __syncthreads();
                v = qs[lane];
            }
        } else if (warp == 0) {
            nn = fmaf(qv.x, qv.x, fmaf(qv.y, qv.y, fmaf(qv.z, qv.z, fmaf(qv.w, qv.w, nn))));
        }
        if (MODE != T_UPD_SCALE) {
            // dots of this warp's rows with v: 8 rows at a time, transposed shuffle reduction
            for (int r0 = warp * 8; r0 < nvec; r0 += kTileWarps * 8) {
                float pd[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    pd[u] = (r0 + u < nvec) ? dot4(unit_from_smem<T>(tileb + (size_t)(r0 + u) * seg, lane), v) : 0.f;
                const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
                float q4v[4], q2v[2], q1;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float send = b4 ? pd[j] : pd[j + 4], keep = b4 ? pd[j + 4] : pd[j];
                    q4v[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const float send = b3 ? q4v[j] : q4v[j + 2], keep = b3 ? q4v[j + 2] : q4v[j];
                    q2v[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
                }
                {
                    const float send = b2 ? q2v[0] : q2v[1], keep = b2 ? q2v[1] : q2v[0];
                    q1 = keep + __shfl_xor_sync(0xffffffffu, send, 4);
                }
                q1 += __shfl_xor_sync(0xffffffffu, q1, 2);
                q1 += __shfl_xor_sync(0xffffffffu, q1, 1);
                const int pr = r0 + (lane >> 2);
                if ((lane & 3) == 0 && pr < nvec) acc[pr] += q1;   // rows of this warp only
            }
        }
        __syncthreads();                 // stage st consumed by every warp
        if (tid == 0 && i + S < nt) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(i + S);
        }
    }
    if (!ok) {
        // a copy never completed: record it, then wait (bounded) for the copies still in flight
        if (lane == 0) atomicCAS(a.stop, 0, a.step > 0 ? a.step : -1);
        if (tid == 0) a.stop[1] = CT_ETIMEOUT;
        for (int j = i; j < nt && j < i + S; ++j)
            mbar_wait(&bars[j % S], (unsigned)((j / S) & 1), wlim);
    }
    if (MODE == T_UPD_SCALE) return;
    if (warp == 0) {
        nn = warp_sum(nn);
        if (lane == 0) acc[nvec] = nn;
    }
    __syncthreads();
    // block sums; cgs_tile_reduce_kernel adds them across blocks
    double *prow = a.partial + (int64_t)blockIdx.x * ncol;
    for (int c = tid; c < ncol; c += kTileThreads) prow[c] = (double)acc[c];
}

// Cross-block sums of a T1 / T2 pass, one warp per column (all columns in parallel, each in a
// fixed order): T1 writes h1 into the H column and the coefficient buffer and ||q|| to aux[0];
// T2 adds h2 to the H column, writes it to the coefficient buffer and ||q'||^2 to aux[4].
template <int MODE>
__global__ void __launch_bounds__(kThreads) cgs_tile_reduce_kernel(TileArgs a, int nblocks)
{
    if (a.stop[0] != 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * kWarps + warp, nvec = a.nvec;
    if (c > nvec) return;
    const double s = column_sum(a.partial, nblocks, nvec + 1, c, lane);
    if (lane != 0) return;
    if (c < nvec) {
        if (MODE == T_DOTS) a.hcol[c] = s;
        else a.hcol[c] += s;
        a.coef_out[c] = s;
    } else if (MODE == T_DOTS) {
        a.aux[0] = sqrt(s);
    } else {
        a.aux[4] = s;
    }
}

// Launch plan of the tiled path: stages per CTA and CTAs per SM from the shared memory a stage
// needs (two CTAs per SM while two stages fit in half the SM's memory); 0 stages = not eligible.
template <typename T>
static void tile_plan(int nvec, int &stages, int &per_sm, size_t &smem)
{
    const int sb = tile_stage_bytes<T>(nvec);
    // mbarriers (<= 6 stages), block sums, warp partials and q', coefficients, spare
    const int extra = 48 + 16 * ((nvec + 4) / 4) + 16 * (kTileWarps + 1) * kTileUnits + 4 * nvec + 64;
    if (2 * sb + extra <= kTilePair) {
        stages = std::min(6, (kTilePair - extra) / sb);
        per_sm = 2;
    } else if (2 * sb + extra <= kTileSmemMax) {
        stages = 2;
        per_sm = 1;
    } else {
        stages = 0;
        per_sm = 0;
    }
    smem = (size_t)stages * sb + extra;
}

static int device_sms()
{
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!cached[dev]) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            sms = 152;
        cached[dev] = sms;
    }
    return cached[dev];
}

// Allows the tile kernels their dynamic shared memory on the current device (before a capture).
static cudaError_t tile_prepare()
{
    static bool done[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (done[dev]) return cudaSuccess;
#define CT_TILE_ATTR(M, T)                                                                        \
    e = cudaFuncSetAttribute(cgs_tile_kernel<M, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             kTileSmemMax);                                                       \
    if (e != cudaSuccess) return e;
    CT_TILE_ATTR(T_DOTS, float) CT_TILE_ATTR(T_UPD_DOTS, float) CT_TILE_ATTR(T_UPD_SCALE, float)
    CT_TILE_ATTR(T_DOTS, __nv_bfloat16) CT_TILE_ATTR(T_UPD_DOTS, __nv_bfloat16)
    CT_TILE_ATTR(T_UPD_SCALE, __nv_bfloat16)
    CT_TILE_ATTR(T_DOTS, __half) CT_TILE_ATTR(T_UPD_DOTS, __half) CT_TILE_ATTR(T_UPD_SCALE, __half)
#undef CT_TILE_ATTR
    done[dev] = true;
    return cudaSuccess;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Tensor map of basis rows 0..nvec-1 (row stride ld entries of T) with nvec x 128 boxes.
template <typename T>
static bool encode_basis_map(CUtensorMap *map, const void *W, int64_t ld, int nvec)
{
    const auto enc = tensor_map_encoder();
    if (!enc || nvec < 1 || nvec > 256) return false;
    const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : std::is_same<T, __nv_bfloat16>::value
                                       ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                       : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)nvec};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(T)};
    const cuuint32_t box[2] = {(cuuint32_t)kTileElems, (cuuint32_t)nvec};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, dt, 2, const_cast<void *>(W), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T>
static bool tile_eligible(int64_t ld, int k, const ArnoldiScratch &sc)
{
    int stages, per_sm;
    size_t smem;
    tile_plan<T>(k + 1, stages, per_sm, smem);
    return stages >= 2 && k + 1 <= 256 && ld % kTileElems == 0 && k + 2 <= sc.kmax + 2 &&
           tensor_map_encoder() != nullptr;
}

// The tiled CGS2 step (three launches); false when the step is not eligible (then nothing ran).
template <typename T>
static bool arnoldi_step_tiled(void *W, int64_t ld, int k, float *q, double *hcol,
                               const ArnoldiScratch &sc, double *aux, int *stop, int step,
                               float *cur, cudaStream_t s, cudaError_t &err, bool next)
{
    const int nvec = k + 1;
    int stages, per_sm;
    size_t smem;
    tile_plan<T>(nvec, stages, per_sm, smem);
    if (!tile_eligible<T>(ld, k, sc) || (reinterpret_cast<uintptr_t>(W) & 255) != 0 ||
        (reinterpret_cast<uintptr_t>(q) & 15) != 0)
        return false;
    if ((err = tile_prepare()) != cudaSuccess) return true;
    CUtensorMap wmap;
    if (!encode_basis_map<T>(&wmap, W, ld, nvec)) return false;
    const int ntiles = (int)(ld / kTileElems);
    const int blocks = std::max(1, std::min({ntiles, per_sm * device_sms(), sc.max_blocks}));
    double *h1 = aux + 8, *h2 = aux + 8 + (sc.kmax + 2);
    TileArgs a{W, ld, nvec, q, q, ntiles, stages, nullptr, sc.partial, sc.counter, hcol, aux,
               h1, stop, step, nullptr, nullptr};
    const int rblocks = (nvec + 1 + kWarps - 1) / kWarps;
    cgs_tile_kernel<T_DOTS, T><<<blocks, kTileThreads, smem, s>>>(wmap, a);
    cgs_tile_reduce_kernel<T_DOTS><<<rblocks, kThreads, 0, s>>>(a, blocks);
    a.coef = h1; a.coef_out = h2;
    cgs_tile_kernel<T_UPD_DOTS, T><<<blocks, kTileThreads, smem, s>>>(wmap, a);
    cgs_tile_reduce_kernel<T_UPD_DOTS><<<rblocks, kThreads, 0, s>>>(a, blocks);
    a.coef = h2; a.coef_out = nullptr;
    a.wnext = next ? static_cast<char *>(W) + (size_t)(k + 1) * ld * sizeof(T) : nullptr;
    a.cur = next ? cur : nullptr;
    cgs_tile_kernel<T_UPD_SCALE, T><<<next ? blocks : 1, kTileThreads, smem, s>>>(wmap, a);
    err = cudaGetLastError();
    return true;
}

// One CGS2 Arnoldi step on rows W[0..k] (storage type T) with q = M w_k; writes the H column
// (FP64, k+2 entries), W[k+1] and, when `cur` is not null, W[k+1] in FP32.  `aux` / `stop` are
// device scratch words (see CgsArgs).
template <typename T>
static cudaError_t arnoldi_step_t(void *W, int64_t L, int64_t ld, int k, float *q, double *hcol,
                                  const ArnoldiScratch &sc, double *aux, int *stop, int step,
                                  bool reorth, float *cur, bool q_padded, cudaStream_t s,
                                  bool next = true)
{
    cudaError_t err = cudaSuccess;
    if (reorth && q_padded &&
        arnoldi_step_tiled<T>(W, ld, k, q, hcol, sc, aux, stop, step, cur, s, err, next))
        return err;
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

// kernel launches of one arnoldi_step_basis call (W and q as the solver allocates them)
int arnoldi_step_launches(int basis, int64_t ld, int k, const ArnoldiScratch &sc, bool reorth,
                          bool q_padded)
{
    if (!reorth) return 3;
    bool tiled = false;
    if (q_padded) {
        if (basis == CT_BASIS_BF16) tiled = tile_eligible<__nv_bfloat16>(ld, k, sc);
        else if (basis == CT_BASIS_F16) tiled = tile_eligible<__half>(ld, k, sc);
        else tiled = tile_eligible<float>(ld, k, sc);
    }
    return tiled ? 5 : 4;
}

cudaError_t arnoldi_step_dev(float *W, int64_t L, int64_t ld, int k, float *q, double *hcol,
                             const ArnoldiScratch &sc, double *aux, int *stop, int step,
                             bool reorth, cudaStream_t s)
{
    return arnoldi_step_t<float>(W, L, ld, k, q, hcol, sc, aux, stop, step, reorth, nullptr,
                                 false, s);
}

cudaError_t arnoldi_step_basis(int basis, void *W, int64_t L, int64_t ld, int k, float *q,
                               double *hcol, const ArnoldiScratch &sc, double *aux, int *stop,
                               int step, bool reorth, float *cur, bool q_padded, cudaStream_t s,
                               bool next)
{
    switch (basis) {
    case CT_BASIS_BF16:
        return arnoldi_step_t<__nv_bfloat16>(W, L, ld, k, q, hcol, sc, aux, stop, step, reorth,
                                             cur, q_padded, s, next);
    case CT_BASIS_F16:
        return arnoldi_step_t<__half>(W, L, ld, k, q, hcol, sc, aux, stop, step, reorth, cur,
                                      q_padded, s, next);
    default:
        return arnoldi_step_t<float>(W, L, ld, k, q, hcol, sc, aux, stop, step, reorth, cur,
                                     q_padded, s, next);
    }
}

// beta = ||r||, w0 = r / beta (the first basis vector of Algorithms 1/2) in the basis type;
// beta stored in aux[2].
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
