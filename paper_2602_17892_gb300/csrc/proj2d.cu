// 2D projector kernels: ray-driven Joseph forward projector A and pixel-driven linear-
// interpolation backprojector B (the unmatched pair of Sec. 2 of arXiv 2602.17892).
//
// Data layout in HBM (all FP32):
//   XR[r][c + 1] = x[r][c], XT[c][r + 1] = x[r][c], with a zero border column/row on each side,
// so the two taps of every Joseph sample are adjacent floats of one line with no bounds test
// (rays driven along x read XT, rays driven along y read XR).  The padded sinogram has 2 zero
// bins on each side of every detector row, so the backprojector's taps need no bounds test
// either.
#include "ct_internal.h"

namespace ct {

// ---------------------------------------------------------------------------- image layouts
// XR[r][c + 1] = x[r][c] and XT[c][r + 1] = x[r][c]; column/row 0 and n + 1 stay zero (the
// buffers are zeroed once when the geometry is created and only interiors are written).
__global__ void __launch_bounds__(256) image_layouts_kernel(
    const float *__restrict__ x, int nx, int ny, float *__restrict__ xr, int ldr,
    float *__restrict__ xt, int ldt, const int *stop)
{
    if (stop && stop[0] != 0) return;
    __shared__ float tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
        int tr = t / 32, tc = t % 32;
        int r = r0 + tr, c = c0 + tc;
        float v = (r < ny && c < nx) ? x[(int64_t)r * nx + c] : 0.f;
        tile[tr][tc] = v;
        if (r < ny && c < nx) xr[(int64_t)r * ldr + c + 1] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
        int tc = t / 32, tr = t % 32;
        int r = r0 + tr, c = c0 + tc;
        if (r < ny && c < nx) xt[(int64_t)c * ldt + r + 1] = tile[tr][tc];
    }
}

cudaError_t launch_image_pairs(const ct_geom *g, const float *x, const int *stop, cudaStream_t s)
{
    const DeviceGeom &d = g->dg;
    dim3 grid((d.nx + 31) / 32, (d.ny + 31) / 32);
    image_layouts_kernel<<<grid, 256, 0, s>>>(x, d.nx, d.ny, g->xr_dev, d.xr_ld, g->xt_dev,
                                              d.xt_ld, stop);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- padded sinogram
__global__ void pad_sino_kernel(const float *__restrict__ y, int rows, int nd, int ld,
                                float *__restrict__ ypad)
{
    int64_t total = (int64_t)rows * ld;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = t / ld;
        int j = (int)(t - r * ld) - 2;
        ypad[t] = (j >= 0 && j < nd) ? y[r * nd + j] : 0.f;
    }
}

cudaError_t launch_pad_sino(const ct_geom *g, const float *y, float *ypad, cudaStream_t s)
{
    const DeviceGeom &d = g->dg;
    int rows = d.n_views * d.ndv;
    int64_t total = (int64_t)rows * d.sino_ld;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    pad_sino_kernel<<<blocks, 256, 0, s>>>(y, rows, d.ndu, d.sino_ld, ypad);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- Joseph A
// One thread per ray.  pos = pmid + slope * (t - t_mid) is the fractional index across the
// driving axis; the two taps floor(pos), floor(pos)+1 are adjacent floats of line t in the
// zero-bordered layout (XT for rays driven along x, XR for rays driven along y), so
// neighbouring rays of a warp share cache sectors.
__global__ void __launch_bounds__(256) joseph2d_kernel(
    const Ray2D *__restrict__ rays, int64_t m, int ndu,
    const float *__restrict__ xr, int ldr, const float *__restrict__ xt, int ldt,
    int nx, int ny, float *__restrict__ y, int y_ld, int y_off, const int *stop)
{
    if (stop && stop[0] != 0) return;
    int64_t ray = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (ray >= m) return;
    const Ray2D R = rays[ray];
    const int t_lo = R.packed & 0x7fff;
    const int t_hi = (R.packed >> 15) & 0x7fff;
    const int axis = (R.packed >> 30) & 1;
    const float *base;
    int64_t stride;
    float tmid, hiclamp;
    if (axis == 0) {        // drive along x: line = column c of XT, taps along rows
        base = xt; stride = ldt; tmid = 0.5f * (float)(nx - 1);
        hiclamp = __int_as_float(__float_as_int((float)ny) - 1);
    } else {                // drive along y: line = row r of XR, taps along columns
        base = xr; stride = ldr; tmid = 0.5f * (float)(ny - 1);
        hiclamp = __int_as_float(__float_as_int((float)nx) - 1);
    }
    float acc = 0.f;
    float tf = (float)t_lo - tmid;
    const float *line = base + (int64_t)t_lo * stride + 1;
#pragma unroll 4
    for (int t = t_lo; t <= t_hi; ++t) {
        float pos = fmaf(R.slope, tf, R.pmid);
        pos = fminf(fmaxf(pos, -1.f), hiclamp);
        float fl = floorf(pos);
        float f = pos - fl;
        const float *tap = line + (int)fl;
        float a = __ldg(tap), b = __ldg(tap + 1);
        acc += fmaf(f, b - a, a);
        tf += 1.f;
        line += stride;
    }
    int64_t view = ray / ndu;
    int bin = (int)(ray - view * ndu);
    y[view * y_ld + y_off + bin] = acc * R.weight;
}

cudaError_t launch_joseph2d(const ct_geom *g, float *y, int y_ld, int y_off, const int *stop,
                            cudaStream_t s)
{
    const DeviceGeom &d = g->dg;
    int64_t m = g->m;
    int blocks = (int)((m + 255) / 256);
    joseph2d_kernel<<<blocks, 256, 0, s>>>(g->rays_dev, m, d.ndu, g->xr_dev, d.xr_ld, g->xt_dev,
                                           d.xt_ld, d.nx, d.ny, y, y_ld, y_off, stop);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- pixel-driven B
// One thread per pixel, blocks of 32 x 8 pixels.  Views are processed in batches of kVB: for
// each view the detector footprint of the block (bins between the projections of its corner
// pixels, plus a margin) is copied from the padded sinogram into shared memory once and read
// by all 256 pixels.
//   parallel: bin position fj = a (c - cm) + b (r - rm) + (nd-1)/2, weight h^2/pitch;
//   fan:      pe = p.e_u, bb = SID - p.(cos, sin) (in units of h), u = SDD pe / bb,
//             weight h SDD / pitch * sqrt(1 + (pe/bb)^2) / bb (= h^2 (SDD^2+u^2)/(L pitch SDD)).
// A view whose footprint is wider than the shared-memory slot reads the sinogram directly.
constexpr int kVB = 32;

template <bool FAN>
__device__ __forceinline__ void bp_pos(const float4 &V, float tc, float tr, float sid_h, float k_u,
                                       float gam, float &fj, float &w)
{
    if (FAN) {
        float pe = fmaf(tr, V.x, -tc * V.y);
        float bb = fmaf(-tc, V.x, fmaf(-tr, V.y, sid_h));
        float rb = __fdividef(1.f, bb);
        float t1 = pe * rb;
        fj = fmaf(t1, k_u, gam);
        float q = fmaf(t1, t1, 1.f);
        w = rb * (q * rsqrtf(q));
    } else {
        fj = fmaf(V.z, tc, fmaf(V.w, tr, gam));
        w = 1.f;
    }
}

template <bool FAN>
__global__ void __launch_bounds__(256) pixbp2d_kernel(
    const ViewBP *__restrict__ views, int n_views, const float *__restrict__ ypad, int ld,
    int nd, int nx, int ny, float sid_h, float k_u, float k_w, float w_par, int slot,
    float *__restrict__ x, const int *stop)
{
    if (stop && stop[0] != 0) return;
    extern __shared__ float smem[];
    float4 *sview = reinterpret_cast<float4 *>(smem);              // kVB
    int *sjlo = reinterpret_cast<int *>(sview + kVB);               // kVB
    int *swid = sjlo + kVB;                                         // kVB
    float *ssino = reinterpret_cast<float *>(swid + kVB);           // kVB * slot
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 8;
    const int c = c0 + threadIdx.x;
    const int r = r0 + threadIdx.y;
    const float cm = 0.5f * (float)(nx - 1), rm = 0.5f * (float)(ny - 1);
    const float tc = (float)c - cm;
    const float tr = (float)r - rm;
    const float gam = 0.5f * (float)(nd - 1) + 2.f;   // +2: padded row offset
    const float hi = (float)(nd + 2);
    // corner pixels of the block (clipped to the image)
    const float cA = (float)c0 - cm, cB = (float)min(c0 + 31, nx - 1) - cm;
    const float rA = (float)r0 - rm, rB = (float)min(r0 + 7, ny - 1) - rm;
    float acc = 0.f;
    for (int v0 = 0; v0 < n_views; v0 += kVB) {
        const int nvb = min(kVB, n_views - v0);
        if (tid < nvb) {
            ViewBP vb = views[v0 + tid];
            float4 V = make_float4(vb.cs, vb.sn, vb.a, vb.b);
            float f0, f1, f2, f3, w;
            bp_pos<FAN>(V, cA, rA, sid_h, k_u, gam, f0, w);
            bp_pos<FAN>(V, cB, rA, sid_h, k_u, gam, f1, w);
            bp_pos<FAN>(V, cA, rB, sid_h, k_u, gam, f2, w);
            bp_pos<FAN>(V, cB, rB, sid_h, k_u, gam, f3, w);
            float fmn = fminf(fminf(f0, f1), fminf(f2, f3));
            float fmx = fmaxf(fmaxf(f0, f1), fmaxf(f2, f3));
            fmn = fminf(fmaxf(fmn, 0.f), hi);
            fmx = fminf(fmaxf(fmx, 0.f), hi);
            int jlo = max((int)floorf(fmn) - 1, 0);
            int jhi = min((int)floorf(fmx) + 2, nd + 3);
            sview[tid] = V;
            sjlo[tid] = jlo;
            swid[tid] = jhi - jlo + 1;            // > slot: this view reads global memory
        }
        __syncthreads();
        for (int idx = tid; idx < nvb * slot; idx += 256) {
            int t = idx / slot, j = idx - t * slot;
            if (j < swid[t]) ssino[idx] = __ldg(ypad + (int64_t)(v0 + t) * ld + sjlo[t] + j);
        }
        __syncthreads();
        if (c < nx && r < ny) {
            const float *row = ypad + (int64_t)v0 * ld;
#pragma unroll 4
            for (int t = 0; t < nvb; ++t, row += ld) {
                float fj, w;
                bp_pos<FAN>(sview[t], tc, tr, sid_h, k_u, gam, fj, w);
                fj = fminf(fmaxf(fj, 0.f), hi);
                float fl = floorf(fj);
                float f = fj - fl;
                int j = (int)fl;
                const int wid = swid[t];
                float a, b;
                if (wid <= slot) {
                    int jj = min(max(j - sjlo[t], 0), wid - 2);
                    a = ssino[t * slot + jj];
                    b = ssino[t * slot + jj + 1];
                } else {
                    a = __ldg(row + j);
                    b = __ldg(row + j + 1);
                }
                acc = fmaf(w, fmaf(f, b - a, a), acc);
            }
        }
        __syncthreads();
    }
    if (c < nx && r < ny) x[(int64_t)r * nx + c] = acc * (FAN ? k_w : w_par);
}

size_t pixbp2d_smem_bytes(int slot)
{
    return sizeof(float4) * kVB + 2 * sizeof(int) * kVB + sizeof(float) * (size_t)kVB * slot;
}

cudaError_t launch_pixbp2d(const ct_geom *g, const float *ypad, float *x, const int *stop,
                           cudaStream_t s)
{
    const DeviceGeom &d = g->dg;
    dim3 block(32, 8), grid((d.nx + 31) / 32, (d.ny + 7) / 8);
    const int slot = d.bp_slot;
    size_t smem = pixbp2d_smem_bytes(slot);
    float sid_h = d.sid / d.h;
    float k_u = d.sdd / d.pitch_u;
    float k_w = d.h * d.sdd / d.pitch_u;
    float w_par = d.h * d.h / d.pitch_u;
    if (d.kind == CT_FANFLAT2D)
        pixbp2d_kernel<true><<<grid, block, smem, s>>>(d.views, d.n_views, ypad, d.sino_ld, d.ndu,
                                                        d.nx, d.ny, sid_h, k_u, k_w, w_par, slot,
                                                        x, stop);
    else
        pixbp2d_kernel<false><<<grid, block, smem, s>>>(d.views, d.n_views, ypad, d.sino_ld, d.ndu,
                                                         d.nx, d.ny, sid_h, k_u, k_w, w_par, slot,
                                                         x, stop);
    return cudaGetLastError();
}

}  // namespace ct
