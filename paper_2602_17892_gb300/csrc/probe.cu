// Throughput probes: kernels that do only the elementary work of one projector sample, so
// that the rooflines of the gather-bound projectors rest on ceilings measured on the GPU at
// hand rather than on unit counts read from documentation.
//
//   gather8: the floor of one Joseph or pixel-driven sample, one 8-byte tap-pair load from a
//            table resident in L1 (every warp reads 32 consecutive pairs, the best case of the
//            projectors' near-contiguous gathers) and one addition that keeps it live;
//   mufu:    the special-function pair of a fan-beam pixel-driven sample, one reciprocal and
//            one square root (the forms the backprojector uses), chained so nothing is hoisted.
// Both run one wave of resident blocks on every SM, each thread with 8 independent chains so
// that latency is hidden and the pipe under test is the limit.
#include <cuda_runtime.h>

#include "ct_internal.h"

namespace ct {

namespace {
constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;
constexpr int kProbeTablePairs = 4096;     // 32 KB: resident in every SM's L1
}

// the gather probe's table (its contents do not matter: nothing depends on the values)
static __device__ float2 g_probe_table[kProbeTablePairs];

__global__ void __launch_bounds__(kProbeThreads) probe_gather8_kernel(int64_t reps,
                                                                      float *__restrict__ out)
{
    const float2 *table = g_probe_table;
    const int lane = threadIdx.x & 31;
    const unsigned warp_id = blockIdx.x * (kProbeThreads / 32) + (threadIdx.x >> 5);
    float acc[kProbeChains];
    unsigned off[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) {
        acc[c] = 0.f;
        off[c] = ((warp_id * 977u + (unsigned)c * 613u) * 32u) & (kProbeTablePairs - 32);
    }
    for (int64_t r = 0; r < reps; r += kProbeChains) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) {
            // one pair load, one operation that consumes both halves
            const float2 v = __ldg(table + off[c] + (unsigned)lane);
            acc[c] = fmaf(v.x, acc[c], v.y);
            off[c] = (off[c] + 32u * 37u) & (kProbeTablePairs - 32);   // another 256-byte row
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += acc[c];
    out[blockIdx.x * (int64_t)kProbeThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_mufu_kernel(int64_t reps, float seed,
                                                                   float *__restrict__ out)
{
    float x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = seed + 0.001f * (float)(threadIdx.x + c);
    for (int64_t r = 0; r < reps; r += kProbeChains) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) {
            // x -> sqrt(1 + 1/x): one reciprocal, one square root, values stay near 1.6
            const float t = __fdividef(1.f, x[c]);
            x[c] = sqrtf(t + 1.f);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    out[blockIdx.x * (int64_t)kProbeThreads + threadIdx.x] = s;
}

int probe_threads() { return kProbeThreads; }
int probe_chains() { return kProbeChains; }

cudaError_t launch_probe(int kind, int64_t reps, float *out, int blocks, cudaStream_t s)
{
    if (kind == 0)
        probe_gather8_kernel<<<blocks, kProbeThreads, 0, s>>>(reps, out);
    else
        probe_mufu_kernel<<<blocks, kProbeThreads, 0, s>>>(reps, 1.25f, out);
    return cudaGetLastError();
}

int probe_blocks_per_sm(int kind)
{
    int per_sm = 0;
    cudaError_t e = kind == 0
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, probe_gather8_kernel, kProbeThreads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, probe_mufu_kernel, kProbeThreads, 0);
    return (e == cudaSuccess && per_sm > 0) ? per_sm : 1;
}

}  // namespace ct
