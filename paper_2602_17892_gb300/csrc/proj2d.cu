// 2D projector kernels: ray-driven Joseph forward projector A and pixel-driven linear-
// interpolation backprojector B (the unmatched pair of Sec. 2 of arXiv 2602.17892).
//
// Data layout in HBM (all FP32), "centred slope pairs": for the segment between samples
// s_{i-1} and s_i of a line, the difference d = s_i - s_{i-1} and the value of the segment's
// line at the line's centre index c, a = s_{i-1} - (i - 1 - c) d, so that at a position p
// (index units) of the segment the linear interpolant is ONE fma, a + (p - c) d, with no
// fraction p - floor(p) to form:
//   P_row[r][j] = (x[r][j-1] - (j-1-cx) d, d), d = x[r][j] - x[r][j-1], j in [0, nx], cx = nx / 2
//   P_col[c][i] = (x[i-1][c] - (i-1-cy) d, d), d = x[i][c] - x[i-1][c], i in [0, ny], cy = ny / 2
// zero outside the image.  Every Joseph sample is one 8-byte load with no bounds test and one
// fma: rays driven along x read P_col (neighbouring rays of a warp read adjacent pairs), rays
// driven along y read P_row.  The rounding: a and p - c carry errors of the order of ulp(c d)
// and ulp(p), the same order as the fraction p - floor(p) that the plain form interpolates
// with (its error is ulp(p)).  The padded sinogram has 2 zero bins on each side of every
// detector row, so the backprojector's two taps also need no bounds test; the 2D
// backprojector reads it as centred slope pairs about the row's centre bin, the cone one as
// plain slope pairs (y_j, y_{j+1} - y_j) (the 3D layouts are plain slope pairs as well).
#include <algorithm>

#include "ct_internal.h"

namespace ct {

// ---------------------------------------------------------------------------- pair layouts
// One 32 x 32 tile of pair indices of one z slice (blockIdx.z) per block; a 33 x 33 halo tile
// of the slice sits in smem.  Pair (r, j) of P_row goes to
// prow[(z + off) * rzs + (r + off) * rs + j] and pair (c, i) of P_col to
// pcol[(z + off) * czs + (c + off) * cs + i] (off = 1: a zero row of padding on each side,
// and in 3D a zero slice on each side; 2D has one slice and rzs = czs = 0).
// centred != 0: the centred form about cx = nx / 2 (P_row) and cy = ny / 2 (P_col) (2D);
// otherwise plain slope pairs (x_{i-1}, x_i - x_{i-1}) (3D).
__global__ void __launch_bounds__(256) image_pairs_kernel(
    const float *__restrict__ x, int nx, int ny, float2 *__restrict__ prow, int64_t rs,
    int64_t rzs, float2 *__restrict__ pcol, int64_t cs, int64_t czs, int off, int centred,
    const int *stop)
{
    if (stop && stop[0] != 0) return;
    __shared__ float tile[33][34];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32, z = blockIdx.z;
    const float *xs = x + (int64_t)z * nx * ny;
    for (int t = threadIdx.x; t < 33 * 33; t += blockDim.x) {
        int tr = t / 33, tc = t % 33;
        int r = r0 - 1 + tr, c = c0 - 1 + tc;
        tile[tr][tc] = (r >= 0 && r < ny && c >= 0 && c < nx) ? xs[(int64_t)r * nx + c] : 0.f;
    }
    __syncthreads();
    // P_row: rows r in [r0, r0+32) (< ny), pair index j in [c0, c0+32) (<= nx)
    float2 *pr = prow + (int64_t)off * rs + (int64_t)(z + off) * rzs;
    for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
        int tr = t / 32, tj = t % 32;
        int r = r0 + tr, j = c0 + tj;
        if (r < ny && j <= nx) {
            const float a = tile[tr + 1][tj], d = tile[tr + 1][tj + 1] - a;
            const float k = centred ? (float)(j - 1 - (nx >> 1)) : 0.f;
            pr[(int64_t)r * rs + j] = make_float2(fmaf(-k, d, a), d);
        }
    }
    // P_col: column c in [c0, c0+32) (< nx), pair index i in [r0, r0+32) (<= ny)
    float2 *pc = pcol + (int64_t)off * cs + (int64_t)(z + off) * czs;
    for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
        int tc = t / 32, ti = t % 32;
        int c = c0 + tc, i = r0 + ti;
        if (c < nx && i <= ny) {
            const float a = tile[ti][tc + 1], d = tile[ti + 1][tc + 1] - a;
            const float k = centred ? (float)(i - 1 - (ny >> 1)) : 0.f;
            pc[(int64_t)c * cs + i] = make_float2(fmaf(-k, d, a), d);
        }
    }
}

cudaError_t launch_image_pairs(const ct_geom *g, const float *x, const int *stop, cudaStream_t s)
{
    const DeviceGeom &d = g->dg;
    dim3 grid((d.nx + 1 + 31) / 32, (d.ny + 1 + 31) / 32, d.nz);
    if (d.kind == CT_CONE3D)
        image_pairs_kernel<<<grid, 256, 0, s>>>(x, d.nx, d.ny, g->prow_dev, d.row_pairs_ld,
                                                d.slice_y, g->pcol_dev, d.col_pairs_ld,
                                                d.slice_x, 1, 0, stop);
    else
        image_pairs_kernel<<<grid, 256, 0, s>>>(x, d.nx, d.ny, g->prow_dev, d.row_pairs_ld, 0,
                                                g->pcol_dev, d.col_pairs_ld, 0, 1, 1, stop);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- padded sinogram
// y[view][v][u] -> ypad[view * view_ld + row0 + v * ld + 2 + u]; the margins are zero
__global__ void pad_sino_kernel(const float *__restrict__ y, int n_views, int nv, int nu, int ld,
                                int64_t view_ld, int row0, float *__restrict__ ypad)
{
    const int64_t total = (int64_t)n_views * nv * ld;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / ld;                   // view * nv + v
        const int j = (int)(t - r * ld) - 2;
        const int64_t view = r / nv;
        const int v = (int)(r - view * nv);
        ypad[view * view_ld + row0 + (int64_t)v * ld + j + 2] =
            (j >= 0 && j < nu) ? y[r * nu + j] : 0.f;
    }
}

cudaError_t launch_pad_sino(const ct_geom *g, const float *y, float *ypad, cudaStream_t s)
{
    const DeviceGeom &d = g->dg;
    const int64_t total = (int64_t)d.n_views * d.ndv * d.sino_ld;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    pad_sino_kernel<<<blocks, 256, 0, s>>>(y, d.n_views, d.ndv, d.ndu, d.sino_ld, d.sino_view_ld,
                                           d.sino_row0, ypad);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- sinogram pairs
// Over the whole padded sinogram (the element after a row's last one is the next row's first
// zero margin, or zero at the end), with d_e = ypad[e + 1] - ypad[e] and j = e mod ld the bin of
// e in its row: centred (2D, rows of ld bins one after the other) pairs[e] =
// (ypad[e] - (j - cb) d_e, d_e), cb the row's centre bin; plain (cone) pairs[e] = (ypad[e], d_e).
// A backprojector tap pair is then one aligned 8-byte load and its interpolation one fma.
__global__ void sino_pairs_kernel(const float *__restrict__ ypad, int64_t total,
                                  float2 *__restrict__ pairs, int ld, int cb, int centred,
                                  const int *stop)
{
    if (stop && stop[0] != 0) return;
    const int64_t n4 = total / 4;               // total and ld are multiples of 4
    const float4 *y4 = reinterpret_cast<const float4 *>(ypad);
    float4 *p4 = reinterpret_cast<float4 *>(pairs);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n4;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = __ldg(y4 + e);
        const float nx = (e + 1 < n4) ? __ldg(ypad + 4 * (e + 1)) : 0.f;
        const float4 d = make_float4(a.y - a.x, a.z - a.y, a.w - a.z, nx - a.w);
        const float k0 = centred ? (float)((int)((4 * e) % ld) - cb) : 0.f;
        const float k1 = centred ? k0 + 1.f : 0.f, k2 = centred ? k0 + 2.f : 0.f;
        const float k3 = centred ? k0 + 3.f : 0.f;
        p4[2 * e] = make_float4(fmaf(-k0, d.x, a.x), d.x, fmaf(-k1, d.y, a.y), d.y);
        p4[2 * e + 1] = make_float4(fmaf(-k2, d.z, a.z), d.z, fmaf(-k3, d.w, a.w), d.w);
    }
}

static cudaError_t launch_sino_pairs(const ct_geom *g, const float *ypad, const int *stop,
                                     cudaStream_t s)
{
    const DeviceGeom &d = g->dg;
    const int64_t total = (int64_t)d.n_views * d.sino_view_ld;
    const int blocks = (int)std::min<int64_t>((total / 4 + 255) / 256, 152 * 8);
    // 2D: one padded row per view (view stride = ld), centred about the backprojector's centre
    // bin (n_det_u + 3) / 2; cone: plain slope pairs
    const bool centred = d.kind != CT_CONE3D;
    sino_pairs_kernel<<<blocks, 256, 0, s>>>(ypad, total, g->sino_pairs_dev, d.sino_ld,
                                             (d.ndu + 3) >> 1, centred ? 1 : 0, stop);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- dispatch
cudaError_t launch_forward_proj(const ct_geom *g, float *y, bool padded, const int *stop,
                                cudaStream_t s)
{
    const DeviceGeom &d = g->dg;
    if (d.kind == CT_CONE3D)
        return padded ? launch_joseph3d(g, y, d.sino_view_ld, d.sino_ld, d.sino_row0 + 2, stop, s)
                      : launch_joseph3d(g, y, (int64_t)d.ndv * d.ndu, d.ndu, 0, stop, s);
    return padded ? launch_joseph2d(g, y, d.sino_ld, 2, stop, s)
                  : launch_joseph2d(g, y, d.ndu, 0, stop, s);
}

cudaError_t launch_back_proj(const ct_geom *g, const float *ypad, float *x, const int *stop,
                             cudaStream_t s)
{
    if (g->dg.back_adjoint) {
        const DeviceGeom &d = g->dg;
        if (d.kind == CT_CONE3D)
            return launch_adjoint3d(g, ypad, d.sino_view_ld, d.sino_ld, d.sino_row0 + 2,
                                    g->adj_acc_dev, x, stop, s);
        return launch_adjoint2d(g, ypad, d.sino_ld, 2, x, stop, s);
    }
    cudaError_t e = launch_sino_pairs(g, ypad, stop, s);
    if (e != cudaSuccess) return e;
    if (g->dg.kind == CT_CONE3D) return launch_voxbp3d(g, g->sino_pairs_dev, x, stop, s);
    return launch_pixbp2d(g, g->sino_pairs_dev, x, stop, s);
}

// ---------------------------------------------------------------------------- Joseph A
// One thread per ray.  pos = pmid + slope * (t - t_mid) is the fractional index across the
// driving axis; the pair at index floor(pos)+1 of line t holds both interpolation taps.
// A block covers blockDim.x / vpb consecutive bins of vpb consecutive views: the views of a
// block cross nearly the same pixels, so their warps share L1 lines.  A warp takes 32 / wv
// consecutive bins of wv consecutive views: at a driving line its lanes' taps then span fewer
// pairs (at the 512^2 fan workload about 1.7 cache lines of 128 B per warp load with 8 bins of
// 4 views, against 3.0 with 32 bins of one view), and the L1 data path, which serves a warp
// load line by line, does fewer passes for the same samples.
//
// The loop works with the centred position pc = pos - co (co = n_other / 2, the layouts'
// centre), pc = fma(slope, t - t_mid, pmid - co), and interpolates with one fma, a + pc d.
// floor(pos) and the pair address come from ONE round-down FP32 addition: for K an integer
// with 2^23 <= K + pos < 2^24 (unit spacing there), s = K + pos rounded towards -infinity is
// exactly K + floor(pos), and the bit pattern of s is the integer 0x4B000000 + (s - 2^23);
// here s = (K + co) + pc with K + co an integer.  K also carries the offset of line t from a
// chunk base (t - t0) * stride, an integer kept exactly in FP32, so the pair address is one
// multiply-add of that bit pattern; chunks of lines keep (t - t0) * stride below 2^22.
//
// No clamp: a sample is taken only where its FP32 position lies in [-1, n_other], so the pair
// index floor(pos) + 1 stays in [0, n_other + 1], which the layouts hold (at least n_other + 2
// pairs per line, zero beyond the image); lines run over [-1, max(nx, ny)] in both layouts, so
// every line of a warp's range exists whatever axis a lane drives along.
// Lines t in [ta, tb] of one ray, two at a time (t and t + 1): both samples' positions and
// floors in paired FP32 arithmetic (one fma.f32x2 / add.rm.f32x2 each, the same operations
// per sample as one line at a time), accumulated in line order.  The lines go in batches of NB
// pairs: first all positions and floors, then all 2 NB gathers, then the sums in line order,
// so that each thread has 2 NB gathers in flight (with one pair per iteration the kernel
// waited on its gathers: 14 long-scoreboard stalls per issue); single pairs finish the range.
// The batch's first line is the base address lb, which moves on by 2 NB lines per batch, so the
// K of line pair q of a batch, 2^23 + 2 + co + (2q, 2q + 1) stride, is the same in every batch
// (held in registers, below 2^22 + 2^23 for strides below 2^22 / (2 NB)).
// A sample is taken where |pc| <= win = co + 1, that is pos in [co - win, co + win]: [-1, n] for
// odd n_other, [-1, n + 1] for even n_other (one compare of |pc|); pair indices run to n + 2
// at most, which every line holds (zero beyond pair n: taps outside the image).
template <int NB>
__device__ __forceinline__ float2 joseph2d_span(int ta, int tb, float win, float pmc, float co,
                                                float slope, float tmid, int stride,
                                                uint64_t abase, float2 acc_even_odd)
{
    // the pairs (t, t + 1) start at ta: their first line is odd when ta is, so the sums of the
    // even and of the odd lines are swapped for the span (the split is by absolute line
    // parity, whatever range a warp walks)
    const bool odd = ta & 1;
    float2 acc = odd ? make_float2(acc_even_odd.y, acc_even_odd.x) : acc_even_odd;
    float2 tf2 = make_float2((float)ta - tmid, (float)ta - tmid + 1.f);
    float2 Kq[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q)
        Kq[q] = make_float2(kFloorK0 + co + (float)(2 * q * stride),
                            kFloorK0 + co + (float)((2 * q + 1) * stride));
    const float2 sl2 = make_float2(slope, slope), pm2 = make_float2(pmc, pmc);
    const float2 d2 = make_float2(2.f, 2.f);
    uint64_t lb = abase + 8ull * (uint64_t)ta * (uint64_t)stride;
    const uint64_t dlb = 16ull * NB * (uint64_t)stride, dlb1 = 16ull * (uint64_t)stride;
    int t = ta;
    // tb - t: a warp whose lanes all have empty ranges has ta = INT_MAX and tb = -1, for which
    // t + 2 NB - 1 would overflow; tb - t >= INT_MIN does not
    for (; tb - t >= 2 * NB - 1; t += 2 * NB, lb += dlb) {
        float2 pc[NB], pa[NB], pb[NB];
        uint32_t ia[NB], ib[NB];
        bool ina[NB], inb[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            pc[q] = __ffma2_rn(sl2, tf2, pm2);                       // pos - co
            const float2 sk2 = __fadd2_rd(pc[q], Kq[q]);
            ia[q] = __float_as_uint(sk2.x);
            ib[q] = __float_as_uint(sk2.y);
            ina[q] = fabsf(pc[q].x) <= win;
            inb[q] = fabsf(pc[q].y) <= win;
            tf2 = __fadd2_rn(tf2, d2);
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            pa[q] = make_float2(0.f, 0.f);
            pb[q] = make_float2(0.f, 0.f);
            if (ina[q]) pa[q] = __ldg(reinterpret_cast<const float2 *>(lb + 8ull * ia[q]));
            if (inb[q]) pb[q] = __ldg(reinterpret_cast<const float2 *>(lb + 8ull * ib[q]));
        }
        // a sample not taken has zero taps, so its term is an exact zero
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const float va = fmaf(pc[q].x, pa[q].y, pa[q].x);
            const float vb = fmaf(pc[q].y, pb[q].y, pb[q].x);
            acc = __fadd2_rn(acc, make_float2(va, vb));
        }
    }
    for (; t <= tb; t += 2, lb += dlb1) {
        const float2 pc2 = __ffma2_rn(sl2, tf2, pm2);
        const float2 sk2 = __fadd2_rd(pc2, Kq[0]);
        float2 pa = make_float2(0.f, 0.f), pb = make_float2(0.f, 0.f);
        if (fabsf(pc2.x) <= win)
            pa = __ldg(reinterpret_cast<const float2 *>(lb + 8ull * __float_as_uint(sk2.x)));
        if (t + 1 <= tb && fabsf(pc2.y) <= win)
            pb = __ldg(reinterpret_cast<const float2 *>(lb + 8ull * __float_as_uint(sk2.y)));
        acc = __fadd2_rn(acc, make_float2(fmaf(pc2.x, pa.y, pa.x), fmaf(pc2.y, pb.y, pb.x)));
        tf2 = __fadd2_rn(tf2, d2);
    }
    return odd ? make_float2(acc.y, acc.x) : acc;
}

// A ray of the table in FP32: slope, weight, driving axis, n_other and a range of lines [lo, hi]
// that contains every line t whose FP32 position fma(slope, t - tmid, pmid) - the sample loop's
// own arithmetic - lies in [-1, n_other] (an FP32 estimate of the crossings widened by two
// lines and clipped to the image; empty when the ray misses it).  The forward loop takes a
// sample only where its position is in [co - win, co + win] ([-1, n_other], or [-1, n_other + 1]
// for even n_other): the tap pair floor(pos) + 1 is then in [0, n_other + 2], inside the line's
// zero-padded pairs, so no position needs a clamp, and the samples beyond pos = n_other have
// both taps outside the image (exact zeros); a line beyond the ray's own image extent (a warp's
// rays may drive along different axes of a non-square image) is one of the zero lines both
// layouts carry up to max(nx, ny).
// co = n_other / 2 (the centre of the layout the ray reads), pmc = pmid - co, win = co + 1 and
// the centred window of the samples with a tap in the image [plo, phi] = [-1 - co, n_other - co].
struct RayJ {
    float pmid, slope, weight, ohi;
    float co, pmc, plo, phi, win;
    int axis, lo, hi;
};

__device__ __forceinline__ RayJ decode_ray2d(const Ray2D R, int nx, int ny, float h)
{
    RayJ r;
    r.pmid = R.pmid;
    r.axis = R.enc & 1;
    r.slope = (float)(R.enc >> 1) * 1.862645149230957e-9f;          // 2^-29
    r.weight = h * sqrtf(fmaf(r.slope, r.slope, 1.f));
    const int n_drive = r.axis ? ny : nx, n_other = r.axis ? nx : ny;
    const float tmid = 0.5f * (float)(n_drive - 1);
    r.ohi = (float)n_other;
    r.co = (float)(n_other >> 1);
    r.pmc = r.pmid - r.co;
    r.plo = -1.f - r.co;
    r.phi = r.ohi - r.co;
    r.win = r.co + 1.f;
    const float tmax = (float)(n_drive - 1);
    if (r.slope != 0.f) {
        const float rs = __frcp_rn(r.slope);
        const float ta = tmid + (-1.f - r.pmid) * rs, tb = tmid + (r.ohi - r.pmid) * rs;
        const float lo = fmaxf(0.f, floorf(fminf(ta, tb)) - 2.f);
        const float hi = fminf(tmax, ceilf(fmaxf(ta, tb)) + 2.f);
        r.lo = lo <= hi ? (int)lo : 1;
        r.hi = lo <= hi ? (int)hi : 0;
    } else {
        const bool in = r.pmid >= -1.f && r.pmid <= r.ohi;
        r.lo = in ? 0 : 1;
        r.hi = in ? n_drive - 1 : 0;
    }
    return r;
}

constexpr int kJBatch = 8;   // line pairs per batch of the Joseph loop

// 16 gathers in flight a thread (8 line pairs per batch) take 96 registers: 5 blocks of 128
// threads (20 warps) per SM, against 27 warps with 8 gathers at 64 registers (4 % slower)
__global__ void __launch_bounds__(512, 1) joseph2d_kernel(
    const Ray2D *__restrict__ rays, int n_views, int ndu, int vpb, int wv,
    const float2 *__restrict__ prow, int prow_ld, const float2 *__restrict__ pcol, int pcol_ld,
    int nx, int ny, float h, float *__restrict__ y, int y_ld, int y_off, const int *stop)
{
    if (stop && stop[0] != 0) return;
    // warp w of the block: bin group w % bgroups (32 / wv bins), view group w / bgroups (wv
    // views); lane: bin lane % (32 / wv) of the group, view lane / (32 / wv)
    const int bins_pb = blockDim.x / vpb, bpw = 32 / wv, bgroups = bins_pb / bpw;
    const int w = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    const int bin = blockIdx.x * bins_pb + (w % bgroups) * bpw + lane % bpw;
    const int view0 = blockIdx.y * vpb + (w / bgroups) * wv + lane / bpw;
    const bool valid = bin < ndu && view0 < n_views;   // all lanes stay for the warp range
    const RayJ R = decode_ray2d(rays[valid ? (int64_t)view0 * ndu + bin : 0], nx, ny, h);
    int t_lo = R.lo, t_hi = R.hi;
    if (!valid) { t_lo = 1; t_hi = 0; }
    const int axis = R.axis;
    const float2 *base;          // line 0 of the layout the ray reads
    int stride, n_drive;
    if (axis == 0) { base = pcol; stride = pcol_ld; n_drive = nx; }   // drive along x
    else { base = prow; stride = prow_ld; n_drive = ny; }             // drive along y
    const float tmid = 0.5f * (float)(n_drive - 1);
    // the warp steps through the union of its lanes' driving ranges together, so that at every
    // step its lanes read neighbouring pairs of one line (a lane outside its own range idles)
    const int wlo = __reduce_min_sync(0xffffffffu, t_hi >= t_lo ? t_lo : 0x7fffffff);
    const int whi = __reduce_max_sync(0xffffffffu, t_hi >= t_lo ? t_hi : -1);
    const uint64_t abase = reinterpret_cast<uint64_t>(base) -
                           8ull * ((uint64_t)__float_as_uint(kFloor2p23) + 1ull);
    // two sums, of the even and of the odd lines (in line order each), added at the end
    const float2 acc = joseph2d_span<kJBatch>(wlo, whi, R.win, R.pmc, R.co, R.slope, tmid, stride,
                                              abase, make_float2(0.f, 0.f));
    if (valid) y[(int64_t)view0 * y_ld + y_off + bin] = (acc.x + acc.y) * R.weight;
}

cudaError_t launch_joseph2d(const ct_geom *g, float *y, int y_ld, int y_off, const int *stop,
                            cudaStream_t s)
{
    const DeviceGeom &d = g->dg;
    const int threads = d.tune_a_threads > 0 ? d.tune_a_threads : 256;
    const int vpb = d.tune_a_views > 0 ? d.tune_a_views : 1;
    const int wv = d.tune_a_wviews > 0 ? d.tune_a_wviews : 1;
    const int bins_pb = threads / vpb;
    // every warp one bin group of wv views: checked when the shapes are set
    if (vpb % wv != 0 || bins_pb * wv < 32 || threads % 32 != 0) return cudaErrorInvalidConfiguration;
    dim3 grid((d.ndu + bins_pb - 1) / bins_pb, (d.n_views + vpb - 1) / vpb);
    // line 0 of each 2D layout follows one zero line
    const float2 *prow = g->prow_dev + d.row_pairs_ld, *pcol = g->pcol_dev + d.col_pairs_ld;
    // the K of a batch's last line pair, 2^23 + 2 + co + (2 kJBatch - 1) stride, must keep
    // unit spacing with the position added (below 2^24): strides below 2^22 / (2 kJBatch)
    const int ldm = std::max(d.row_pairs_ld, d.col_pairs_ld);
    if ((int64_t)ldm * 2 * kJBatch >= kFloorSpan) return cudaErrorInvalidValue;
    joseph2d_kernel<<<grid, threads, 0, s>>>(g->rays_dev, d.n_views, d.ndu, vpb, wv, prow,
                                             d.row_pairs_ld, pcol, d.col_pairs_ld, d.nx, d.ny,
                                             d.h, y, y_ld, y_off, stop);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- matched adjoint
// x = A^T y, the transpose of the Joseph projector above (the matched case B = A^T of Sec. 2,
// where AB-/BA-GMRES reduce to LSQR / LSMR): one thread per ray walks the ray's samples with
// the same FP32 positions as joseph2d_kernel (the centred pc = (pmid - co) + slope (t - t_mid),
// the taps co + floor(pc) and co + floor(pc) + 1 with weights 1 - f and f, f = pc - floor(pc))
// and adds weight (1 - f) y_ray and
// weight f y_ray (FP32 products) to the two taps' pixels by atomic FP64 additions, so the
// order in which the rays arrive changes the sums only far below FP32 resolution; a second
// kernel rounds them to FP32.  Taps outside the image have no pixel.
__global__ void __launch_bounds__(256) joseph2d_adjoint_kernel(
    const Ray2D *__restrict__ rays, int n_views, int ndu, const float *__restrict__ y, int y_ld,
    int y_off, int nx, int ny, float h, double *__restrict__ acc, const int *stop)
{
    if (stop && stop[0] != 0) return;
    const int64_t ray = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (ray >= (int64_t)n_views * ndu) return;
    const int view = (int)(ray / ndu), bin = (int)(ray - (int64_t)view * ndu);
    const RayJ R = decode_ray2d(rays[ray], nx, ny, h);
    const float yw = y[(int64_t)view * y_ld + y_off + bin] * R.weight;
    const int t_lo = R.lo, t_hi = R.hi;
    const int axis = R.axis;
    const int n_drive = axis == 0 ? nx : ny, n_other = axis == 0 ? ny : nx;
    // pixel (line t, tap i): axis 0 drives along x (line = column t, taps along rows i),
    // axis 1 along y (line = row t, taps along columns i)
    const int step_t = axis == 0 ? 1 : nx, step_i = axis == 0 ? nx : 1;
    float tf = (float)t_lo - 0.5f * (float)(n_drive - 1);
    for (int t = t_lo; t <= t_hi; ++t, tf += 1.f) {
        const float pc = fmaf(R.slope, tf, R.pmc);      // the forward kernel's centred position
        if (!(pc >= R.plo && pc <= R.phi)) continue;    // the samples the forward kernel takes
        const float fl = floorf(pc);
        const float f = pc - fl;
        const int i0 = (int)fl + (int)R.co;
        double *p = acc + (int64_t)t * step_t;
        if (i0 >= 0 && i0 < n_other) atomicAdd(p + (int64_t)i0 * step_i, (double)(yw * (1.f - f)));
        if (i0 + 1 >= 0 && i0 + 1 < n_other)
            atomicAdd(p + (int64_t)(i0 + 1) * step_i, (double)(yw * f));
    }
}

__global__ void round_to_float_kernel(const double *__restrict__ a, int64_t n, float *__restrict__ x,
                                      const int *stop)
{
    if (stop && stop[0] != 0) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = (float)a[i];
}

cudaError_t launch_round_to_float(const double *a, int64_t n, float *x, const int *stop,
                                  cudaStream_t s)
{
    round_to_float_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, s>>>(
        a, n, x, stop);
    return cudaGetLastError();
}

cudaError_t launch_adjoint2d(const ct_geom *g, const float *y, int y_ld, int y_off, float *x,
                             const int *stop, cudaStream_t s)
{
    const DeviceGeom &d = g->dg;
    const int64_t n = (int64_t)d.nx * d.ny;
    cudaError_t e = cudaMemsetAsync(g->adj_acc_dev, 0, sizeof(double) * (size_t)n, s);
    if (e != cudaSuccess) return e;
    const int64_t rays = (int64_t)d.n_views * d.ndu;
    joseph2d_adjoint_kernel<<<(unsigned)((rays + 255) / 256), 256, 0, s>>>(
        g->rays_dev, d.n_views, d.ndu, y, y_ld, y_off, d.nx, d.ny, d.h, g->adj_acc_dev, stop);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_round_to_float(g->adj_acc_dev, n, x, stop, s);
}

// ---------------------------------------------------------------------------- pixel-driven B
// One thread per pixel, blocks of 32 x tune_b_rows pixels, per-view constants staged in shared
// memory.  A warp takes a tile of 32 / wr columns by wr rows of its block (wr = 1: one row of 32
// pixels): the bin positions of a view then span fewer pairs of the sinogram row (at the 512^2
// fan workload about 1.4 cache lines of 128 B per warp load with 8 x 4 pixels, against 2.3 with
// 32 x 1), so the L1 data path serves each gather in fewer passes.
// Parallel: bin position fj = a (c - cm) + b (r - rm) + (nd-1)/2, weight h^2/pitch.
// Fan:      pe = p.e_u, bb = SID - p.(cos, sin) (in units of h), u = SDD pe / bb,
//           weight h SDD / pitch * sqrt(1 + (pe/bb)^2) / bb  (= h^2 (SDD^2+u^2)/(L pitch SDD)).
// VP = 2 takes two views at a time with paired FP32 arithmetic (one fma.f32x2 forms both
// views' values), in the same operations and order as VP = 1, so the launch shape never
// changes a result.  It works through batches of kBPBatch view pairs: first the positions and
// weights of the whole batch, then its 2 kBPBatch sinogram gathers, then the sums, so that
// each warp has that many gathers in flight (with one view pair per iteration the kernel
// waited on its gathers: 25 long-scoreboard stalls per issue); the launch bounds trade
// occupancy (24 warps per SM) for the registers this takes.
// floor(fj) and the pair address come from one round-down addition (as in the Joseph kernel):
// K = 2^23 + cb + (v - v0) ld over chunks of views, where the loop works with the centred bin
// position fj - cb (cb = (n_det_u + 3) / 2, the centre of the slope pairs) and interpolates
// with one fma, a + (fj - cb) d; fj >= 0 in the padded row.
// CLAMP = false when every pixel centre of the image projects inside the detector in every
// view (checked on the host at geometry creation): the bin positions then need no clamp.
template <bool FAN, bool CLAMP>
__device__ __forceinline__ void pixbp2d_view(const float4 V, float tc, float tr, float gam,
                                             float clo, float chi, float sid_h, float k_u,
                                             float K, uint64_t rb, float &acc)
{
    float fj, w;
    if (FAN) {
        const float pe = fmaf(tr, V.x, -tc * V.y);
        const float bb = fmaf(-tc, V.x, fmaf(-tr, V.y, sid_h));
        const float rbb = __fdividef(1.f, bb);
        const float t1 = pe * rbb;
        fj = fmaf(t1, k_u, gam);
        w = rbb * sqrtf(fmaf(t1, t1, 1.f));
    } else {
        fj = fmaf(V.z, tc, fmaf(V.w, tr, gam));
        w = 1.f;
    }
    if (CLAMP) fj = fminf(fmaxf(fj, clo), chi);
    const float sk = __fadd_rd(fj, K);
    const float2 ab = __ldg(reinterpret_cast<const float2 *>(rb + 8ull * __float_as_uint(sk)));
    acc = fmaf(w, fmaf(fj, ab.y, ab.x), acc);
}

// centred positions, weights and tap-pair indices of views (2j, 2j + 1) for the paired loop
template <bool FAN, bool CLAMP>
__device__ __forceinline__ void pixbp2d_pair(const float4 V, float2 tr2, float2 tc2, float2 ntc2,
                                             float2 ntr2, float2 sid2, float2 ku2, float2 gam2,
                                             float clo, float chi, float2 K2, float2 &fj2,
                                             float2 &w2, uint32_t &ia, uint32_t &ib)
{
    const float2 one2 = make_float2(1.f, 1.f);
    if (FAN) {
        const float2 cs2 = make_float2(V.x, V.y), sn2 = make_float2(V.z, V.w);
        const float2 pe2 = __ffma2_rn(tr2, cs2, __fmul2_rn(ntc2, sn2));
        const float2 bb2 = __ffma2_rn(ntc2, cs2, __ffma2_rn(ntr2, sn2, sid2));
        const float2 rb2 = make_float2(__fdividef(1.f, bb2.x), __fdividef(1.f, bb2.y));
        const float2 t12 = __fmul2_rn(pe2, rb2);
        fj2 = __ffma2_rn(t12, ku2, gam2);
        const float2 s2 = __ffma2_rn(t12, t12, one2);
        w2 = __fmul2_rn(rb2, make_float2(sqrtf(s2.x), sqrtf(s2.y)));
    } else {
        fj2 = __ffma2_rn(make_float2(V.x, V.y), tc2, __ffma2_rn(make_float2(V.z, V.w), tr2, gam2));
        w2 = one2;
    }
    if (CLAMP) fj2 = make_float2(fminf(fmaxf(fj2.x, clo), chi), fminf(fmaxf(fj2.y, clo), chi));
    const float2 sk2 = __fadd2_rd(fj2, K2);
    ia = __float_as_uint(sk2.x);
    ib = __float_as_uint(sk2.y);
}

constexpr int kBPBatch = 8;   // view pairs per batch of the paired loop

template <bool FAN, bool CLAMP, int VP>
__global__ void __launch_bounds__(VP == 2 ? 256 : 512, VP == 2 ? 3 : 1) pixbp2d_kernel(
    const ViewBP *__restrict__ views, int n_views, const float2 *__restrict__ ypair, int ld,
    int vchunk, int nd, int nx, int ny, float sid_h, float k_u, float k_w, float w_par, int wr,
    float *__restrict__ x, const int *stop)
{
    if (stop && stop[0] != 0) return;
    // VP = 1: sview[v] = (cos, sin, a, b); VP = 2: view pair j as (cos_2j, cos_2j+1,
    // sin_2j, sin_2j+1) (fan) or (a_2j, a_2j+1, b_2j, b_2j+1) (parallel), then view v as above
    extern __shared__ float4 sview[];
    const int nthr = blockDim.x * blockDim.y;
    const int npair = (VP == 2) ? n_views / 2 : 0;
    float4 *sv1 = sview + npair;
    for (int v = threadIdx.y * 32 + threadIdx.x; v < n_views; v += nthr) {
        const ViewBP vb = views[v];
        sv1[v] = make_float4(vb.cs, vb.sn, vb.a, vb.b);
    }
    for (int j = threadIdx.y * 32 + threadIdx.x; j < npair; j += nthr) {
        const ViewBP p = views[2 * j], q = views[2 * j + 1];
        sview[j] = FAN ? make_float4(p.cs, q.cs, p.sn, q.sn) : make_float4(p.a, q.a, p.b, q.b);
    }
    __syncthreads();
    // warp threadIdx.y: column group y % wr, row group y / wr of the block; lane: column
    // lane % (32 / wr), row lane / (32 / wr) of its tile
    const int tw = 32 / wr, wy = threadIdx.y, lane = threadIdx.x;
    const int c = blockIdx.x * 32 + (wy % wr) * tw + lane % tw;
    const int r = blockIdx.y * blockDim.y + (wy / wr) * wr + lane / tw;
    if (c >= nx || r >= ny) return;
    const float tc = (float)c - 0.5f * (float)(nx - 1);
    const float tr = (float)r - 0.5f * (float)(ny - 1);
    // bin position fj (in the padded row: +2) centred on the slope pairs' centre bin cb
    const float cb = (float)((nd + 3) >> 1);
    const float gam = 0.5f * (float)(nd - 1) + 2.f - cb;
    const float clo = -cb, chi = (float)(nd + 2) - cb;
    const uint64_t ybase = reinterpret_cast<uint64_t>(ypair) - 8ull * __float_as_uint(kFloor2p23);
    // two sums, of the even and of the odd views (in view order each), added at the end: the
    // paired loop accumulates both with one fma.f32x2 per view pair, the single-view loop the same
    // way, so every launch shape gives the same result
    float2 acc2 = make_float2(0.f, 0.f);
    int v = 0;
    if (VP == 2) {
        // view pairs (2j, 2j + 1): both views' positions, weights and floors in paired FP32
        const float2 tc2 = make_float2(tc, tc), tr2 = make_float2(tr, tr);
        const float2 ntc2 = make_float2(-tc, -tc), ntr2 = make_float2(-tr, -tr);
        const float2 sid2 = make_float2(sid_h, sid_h), ku2 = make_float2(k_u, k_u);
        const float2 gam2 = make_float2(gam, gam);
        const int vch = vchunk & ~1;
        for (int v0 = 0; v0 < 2 * npair; v0 += vch) {
            const int v1 = min(2 * npair, v0 + vch);
            const uint64_t rb = ybase + 8ull * (uint64_t)v0 * (uint64_t)ld;
            float2 K2 = make_float2(kFloor2p23 + cb, kFloor2p23 + cb + (float)ld);
            const float2 dK2 = make_float2(2.f * (float)ld, 2.f * (float)ld);
            const int j0 = v0 >> 1, j1 = v1 >> 1;
            const int jfull = j1 - (j1 - j0) % kBPBatch;
            for (int jb = j0; jb < jfull; jb += kBPBatch) {
                float2 fc[kBPBatch], w[kBPBatch], a[kBPBatch], b[kBPBatch];
                uint32_t ia[kBPBatch], ib[kBPBatch];
#pragma unroll
                for (int q = 0; q < kBPBatch; ++q) {
                    pixbp2d_pair<FAN, CLAMP>(sview[jb + q], tr2, tc2, ntc2, ntr2, sid2, ku2, gam2,
                                             clo, chi, K2, fc[q], w[q], ia[q], ib[q]);
                    K2 = __fadd2_rn(K2, dK2);
                }
#pragma unroll
                for (int q = 0; q < kBPBatch; ++q) {
                    a[q] = __ldg(reinterpret_cast<const float2 *>(rb + 8ull * ia[q]));
                    b[q] = __ldg(reinterpret_cast<const float2 *>(rb + 8ull * ib[q]));
                }
#pragma unroll
                for (int q = 0; q < kBPBatch; ++q) {
                    const float va = fmaf(fc[q].x, a[q].y, a[q].x);
                    const float vb = fmaf(fc[q].y, b[q].y, b[q].x);
                    acc2 = __ffma2_rn(w[q], make_float2(va, vb), acc2);
                }
            }
            for (int jj = jfull; jj < j1; ++jj) {
                float2 fc, w;
                uint32_t ia, ib;
                pixbp2d_pair<FAN, CLAMP>(sview[jj], tr2, tc2, ntc2, ntr2, sid2, ku2, gam2, clo, chi, K2,
                                         fc, w, ia, ib);
                const float2 a = __ldg(reinterpret_cast<const float2 *>(rb + 8ull * ia));
                const float2 b = __ldg(reinterpret_cast<const float2 *>(rb + 8ull * ib));
                const float va = fmaf(fc.x, a.y, a.x);
                const float vb = fmaf(fc.y, b.y, b.x);
                acc2 = __ffma2_rn(w, make_float2(va, vb), acc2);
                K2 = __fadd2_rn(K2, dK2);
            }
        }
        v = 2 * npair;
    }
    for (int v0 = v; v0 < n_views; v0 += vchunk) {
        const int v1 = min(n_views, v0 + vchunk);
        const uint64_t rb = ybase + 8ull * (uint64_t)v0 * (uint64_t)ld;
        float K = kFloor2p23 + cb;
#pragma unroll 4
        for (int vv = v0; vv < v1; ++vv) {
            if (vv & 1) pixbp2d_view<FAN, CLAMP>(sv1[vv], tc, tr, gam, clo, chi, sid_h, k_u, K, rb, acc2.y);
            else pixbp2d_view<FAN, CLAMP>(sv1[vv], tc, tr, gam, clo, chi, sid_h, k_u, K, rb, acc2.x);
            K += (float)ld;
        }
    }
    x[(int64_t)r * nx + c] = (acc2.x + acc2.y) * (FAN ? k_w : w_par);
}

// ---------------------------------------------------------------------------- four-fold B
// Fan geometries whose views come in quadruples 90 degrees apart (view k + m n/4 at angle
// theta_k + m pi/2, m = 1..3, checked on the host) on a square image of even side N: the pixel
// grid is invariant under a quarter turn, and in centred coordinates view theta + pi/2 sees
// pixel (tc, tr) exactly where view theta sees pixel (tr, -tc): the same bin position fj and
// the same weight.  A thread takes the orbit of four pixels
//   p0 = (tc, tr), p1 = (tr, -tc), p2 = (-tc, -tr), p3 = (-tr, tc)
// (grid (c, r), (r, N-1-c), (N-1-c, N-1-r), (N-1-r, c), with (c, r) in the first quadrant)
// and, for each base view k < n/4, forms the four geometries g_j = (fj, w)(theta_k, p_j) once
// (pe_2 = -pe_0 and pe_3 = -pe_1 exactly); pixel p_i takes view k + m n/4 at g_{(i+m) mod 4}:
// 16 pixel-view pairs from 4 geometry evaluations.  Base views go two at a time: both views'
// geometries, then their 32 gathers together, then the sums (view by view, pixel by pixel, m in
// order); launch bounds for 16 warps per SM at up to 128 registers (24 warps with one view at
// a time: 3 % slower).  The base views are split into
// blockDim.z consecutive parts (2 or 4), one per z layer of the block, whose sums are added in
// shared memory in part order (more parts: more threads in flight and a shorter last wave).
// A warp takes a tile of 32 / wr by wr orbit positions, as in pixbp2d_kernel.  The arithmetic of one
// pixel-view pair is the one of pixbp2d_view; only the views' constants (those of view k, for
// the rotated pixel) and the order of the sums differ from the general kernel.
template <bool CLAMP>
__global__ void __launch_bounds__(256, 2) pixbp2d_rot4_kernel(
    const ViewBP *__restrict__ views, int q4, const float2 *__restrict__ ypair, int ld,
    int vchunk, int nd, int N, float sid_h, float k_u, float k_w, int wr, float *__restrict__ x,
    const int *stop)
{
    if (stop && stop[0] != 0) return;
    extern __shared__ float2 srot[];                 // (cos, sin) of the base views, then sums
    float *red = reinterpret_cast<float *>(srot + q4);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const int tid = ((int)threadIdx.z * blockDim.y + threadIdx.y) * 32 + threadIdx.x;
    for (int k = tid; k < q4; k += nthr) srot[k] = make_float2(views[k].cs, views[k].sn);
    __syncthreads();
    const int half = N >> 1;
    const int tw = 32 / wr, wy = threadIdx.y, lane = threadIdx.x;
    const int c = blockIdx.x * 32 + (wy % wr) * tw + lane % tw;
    const int r = blockIdx.y * blockDim.y + (wy / wr) * wr + lane / tw;
    const bool valid = c < half && r < half;
    const float hN = 0.5f * (float)(N - 1);
    const float tc = (float)c - hN, tr = (float)r - hN;
    // centred bin positions, as in pixbp2d_kernel
    const float cb = (float)((nd + 3) >> 1);
    const float gam = 0.5f * (float)(nd - 1) + 2.f - cb;
    const float clo = -cb, chi = (float)(nd + 2) - cb;
    const int nz = blockDim.z;
    const int kz0 = (int)(((int64_t)q4 * threadIdx.z) / nz), kz1 = (int)(((int64_t)q4 * (threadIdx.z + 1)) / nz);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const uint64_t ybase = reinterpret_cast<uint64_t>(ypair) - 8ull * __float_as_uint(kFloor2p23);
    const uint64_t moff = 8ull * (uint64_t)q4 * (uint64_t)ld;     // bytes from row k to k + n/4
    if (valid) {
        for (int k0 = kz0; k0 < kz1; k0 += vchunk) {
            const int k1 = min(kz1, k0 + vchunk);
            uint64_t rb[4];
            rb[0] = ybase + 8ull * (uint64_t)k0 * (uint64_t)ld;
#pragma unroll
            for (int m = 1; m < 4; ++m) rb[m] = rb[m - 1] + moff;
            float K = kFloor2p23 + cb;                   // + (k - k0) ld
            // two base views per iteration: both views' geometry, then their 32 gathers, then
            // the sums in view order (the same operations and order as one view at a time)
            int k = k0;
            for (; k + 1 < k1; k += 2) {
                float fj[2][4], w[2][4];
                uint32_t ia[2][4];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const float2 V = srot[k + u];
                    const float cs = V.x, sn = V.y;
                    float pe[4], bb[4];
                    pe[0] = fmaf(tr, cs, -tc * sn);
                    pe[1] = fmaf(-tc, cs, -tr * sn);
                    pe[2] = -pe[0];
                    pe[3] = -pe[1];
                    bb[0] = fmaf(-tc, cs, fmaf(-tr, sn, sid_h));
                    bb[1] = fmaf(-tr, cs, fmaf(tc, sn, sid_h));
                    bb[2] = fmaf(tc, cs, fmaf(tr, sn, sid_h));
                    bb[3] = fmaf(tr, cs, fmaf(-tc, sn, sid_h));
                    const float Ku = K + (float)(u * ld);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float rbb = __fdividef(1.f, bb[j]);
                        const float t1 = pe[j] * rbb;
                        float f = fmaf(t1, k_u, gam);
                        if (CLAMP) f = fminf(fmaxf(f, clo), chi);
                        fj[u][j] = f;
                        w[u][j] = rbb * sqrtf(fmaf(t1, t1, 1.f));
                        ia[u][j] = __float_as_uint(__fadd_rd(f, Ku));
                    }
                }
                float2 tap[2][16];
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int m = 0; m < 4; ++m)
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            tap[u][4 * m + i] = __ldg(reinterpret_cast<const float2 *>(rb[m] + 8ull * ia[u][(i + m) & 3]));
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            const int g = (i + m) & 3;
                            acc[i] = fmaf(w[u][g], fmaf(fj[u][g], tap[u][4 * m + i].y, tap[u][4 * m + i].x), acc[i]);
                        }
                K += 2.f * (float)ld;
            }
            for (; k < k1; ++k) {
                const float2 V = srot[k];
                const float cs = V.x, sn = V.y;
                float pe[4], bb[4], fj[4], w[4];
                uint32_t ia[4];
                pe[0] = fmaf(tr, cs, -tc * sn);
                pe[1] = fmaf(-tc, cs, -tr * sn);
                pe[2] = -pe[0];
                pe[3] = -pe[1];
                bb[0] = fmaf(-tc, cs, fmaf(-tr, sn, sid_h));
                bb[1] = fmaf(-tr, cs, fmaf(tc, sn, sid_h));
                bb[2] = fmaf(tc, cs, fmaf(tr, sn, sid_h));
                bb[3] = fmaf(tr, cs, fmaf(-tc, sn, sid_h));
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float rbb = __fdividef(1.f, bb[j]);
                    const float t1 = pe[j] * rbb;
                    float f = fmaf(t1, k_u, gam);
                    if (CLAMP) f = fminf(fmaxf(f, clo), chi);
                    fj[j] = f;
                    w[j] = rbb * sqrtf(fmaf(t1, t1, 1.f));
                    ia[j] = __float_as_uint(__fadd_rd(f, K));
                }
                float2 tap[16];
#pragma unroll
                for (int m = 0; m < 4; ++m)
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        tap[4 * m + i] = __ldg(reinterpret_cast<const float2 *>(rb[m] + 8ull * ia[(i + m) & 3]));
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const int g = (i + m) & 3;
                        acc[i] = fmaf(w[g], fmaf(fj[g], tap[4 * m + i].y, tap[4 * m + i].x), acc[i]);
                    }
                K += (float)ld;
            }
        }
    }
    // the other parts' sums join part 0's, in part order
    const int slots = 4 * 32 * blockDim.y;
    const int slot = 4 * ((int)threadIdx.y * 32 + (int)threadIdx.x);
    if (threadIdx.z > 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) red[(threadIdx.z - 1) * slots + slot + i] = acc[i];
    }
    __syncthreads();
    if (threadIdx.z != 0 || !valid) return;
    for (int z = 1; z < nz; ++z)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] += red[(z - 1) * slots + slot + i];
    const int M = N - 1;
    x[(int64_t)r * N + c] = acc[0] * k_w;
    x[(int64_t)(M - c) * N + r] = acc[1] * k_w;
    x[(int64_t)(M - r) * N + (M - c)] = acc[2] * k_w;
    x[(int64_t)c * N + (M - r)] = acc[3] * k_w;
}

template <bool CLAMP>
static void launch_pixbp2d_rot4_t(const ct_geom *g, const float2 *ypad, float *x, const int *stop,
                                  cudaStream_t s)
{
    const DeviceGeom &d = g->dg;
    // b_rows 4, 8, 16: (orbit rows, view parts) per block (2, 2), (4, 2), (2, 4)
    const int half = d.nx >> 1, ry = d.tune_b_rows == 8 ? 4 : 2, parts = d.tune_b_rows == 16 ? 4 : 2;
    const int wr = d.tune_b_wrows > 0 ? d.tune_b_wrows : 1;
    dim3 block(32, ry, parts), grid((half + 31) / 32, (half + ry - 1) / ry);
    const int q4 = d.n_views / 4;
    const size_t smem = sizeof(float2) * (size_t)q4 + sizeof(float) * 4 * 32 * (size_t)ry * (parts - 1);
    pixbp2d_rot4_kernel<CLAMP><<<grid, block, smem, s>>>(
        d.views, q4, ypad, d.sino_ld, floor_chunk(d.sino_ld), d.ndu, d.nx, d.sid / d.h,
        d.sdd / d.pitch_u, d.h * d.sdd / d.pitch_u, wr, x, stop);
}

template <bool FAN, bool CLAMP, int VP>
static void launch_pixbp2d_t(const ct_geom *g, const float2 *ypad, float *x, const int *stop,
                             cudaStream_t s)
{
    const DeviceGeom &d = g->dg;
    const int rows = d.tune_b_rows > 0 ? d.tune_b_rows : 8;
    dim3 block(32, rows), grid((d.nx + 31) / 32, (d.ny + rows - 1) / rows);
    const size_t smem = sizeof(float4) * (size_t)(d.n_views + (VP == 2 ? d.n_views / 2 : 0));
    const float sid_h = d.sid / d.h, k_u = d.sdd / d.pitch_u, k_w = d.h * d.sdd / d.pitch_u;
    const float w_par = d.h * d.h / d.pitch_u;
    const int wr = d.tune_b_wrows > 0 ? d.tune_b_wrows : 1;
    pixbp2d_kernel<FAN, CLAMP, VP><<<grid, block, smem, s>>>(d.views, d.n_views, ypad, d.sino_ld,
                                                             floor_chunk(d.sino_ld), d.ndu, d.nx,
                                                             d.ny, sid_h, k_u, k_w, w_par, wr, x,
                                                             stop);
}

cudaError_t launch_pixbp2d(const ct_geom *g, const float2 *ypad, float *x, const int *stop,
                           cudaStream_t s)
{
    const DeviceGeom &d = g->dg;
    const bool fan = d.kind == CT_FANFLAT2D, clamp = !d.b_noclamp, two = d.tune_b_views == 2;
    if (two && d.tune_b_rows > 8) return cudaErrorInvalidConfiguration;   // 256-thread bound
    // a warp's tile rows divide the block's (orbit) rows: checked when the shapes are set
    const int brows = d.tune_b_views == 4 ? (d.tune_b_rows == 8 ? 4 : 2) : d.tune_b_rows;
    if (d.tune_b_wrows < 1 || brows % d.tune_b_wrows != 0) return cudaErrorInvalidConfiguration;
    if (d.tune_b_views == 4) {
        if (!fan || !d.b_rot4) return cudaErrorInvalidConfiguration;
        clamp ? launch_pixbp2d_rot4_t<true>(g, ypad, x, stop, s)
              : launch_pixbp2d_rot4_t<false>(g, ypad, x, stop, s);
        return cudaGetLastError();
    }
    if (fan) {
        if (clamp) two ? launch_pixbp2d_t<true, true, 2>(g, ypad, x, stop, s)
                       : launch_pixbp2d_t<true, true, 1>(g, ypad, x, stop, s);
        else two ? launch_pixbp2d_t<true, false, 2>(g, ypad, x, stop, s)
                 : launch_pixbp2d_t<true, false, 1>(g, ypad, x, stop, s);
    } else {
        if (clamp) two ? launch_pixbp2d_t<false, true, 2>(g, ypad, x, stop, s)
                       : launch_pixbp2d_t<false, true, 1>(g, ypad, x, stop, s);
        else two ? launch_pixbp2d_t<false, false, 2>(g, ypad, x, stop, s)
                 : launch_pixbp2d_t<false, false, 1>(g, ypad, x, stop, s);
    }
    return cudaGetLastError();
}

}  // namespace ct
