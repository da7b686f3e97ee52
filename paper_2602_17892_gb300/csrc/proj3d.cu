// 3D cone-beam projector kernels: ray-driven Joseph forward projector A (bilinear taps in the
// planes of the driving axis) and voxel-driven backprojector B (bilinear interpolation on the
// flat detector), the 3D form of the unmatched pair of Sec. 2.
//
// Data layout in HBM (all FP32; the volume is x[z][y][x]), slope pairs as in 2D:
//   P_x[z+1][x+1][y+1] = (x[z][y][x], x[z][y+1][x] - x[z][y][x]) for z in [-1, nz+1], x in [-1, M+1], y in [-1, ny]
//   P_y[z+1][y+1][x+1] = (x[z][y][x], x[z][y][x+1] - x[z][y][x]) for z in [-1, nz+1], y in [-1, M+1], x in [-1, nx]
// with M = max(nx, ny) (zero outside the volume; rows of ld >= n + 2 pairs, one z slice after
// the other).  A Joseph sample is two 8-byte loads (the two z rows of its 2 x 2 taps) with no
// bounds test: rays driven along x read P_x, along y P_y, and the rare rays driven along z read
// P_y (two y rows of one slice).  (Quads holding both z rows in one 16-byte load were measured
// slower: they store every voxel twice, and two rays of neighbouring detector rows then no
// longer share the z row between them in L1 - L1 hit rate 46 % -> 10 %, DRAM reads x4.6.)
// z is the slowest index so that consecutive samples of a ray (one step along x or y) are one
// row apart in memory: a ray stays within a few pages while it crosses the volume, and a z slab
// of rows is one contiguous block.
// The padded sinogram of a cone geometry has, per view, one zero detector row above the
// detector rows and two below, and 2 zero bins on each side of every row, so B's four taps need
// no bounds test either (positions are clamped into the zero margins).
#include <algorithm>
#include <cmath>

#include "ct_internal.h"

namespace ct {

// ---------------------------------------------------------------------------- Joseph A (3D)
// One thread per ray (view, row v, column u); a block covers consecutive u of one (view, v),
// and the grid runs v slowest, so the blocks in flight share a band of z planes in L2.
// In-plane geometry of the ray comes from the (view, u) table (FP64 on the host); the z part
// and the clipped plane range are computed per ray in FP64, the samples in FP32.
// Plane range and sampling parameters of ray (view, iv, column R): mode 0/1 = driven along
// x/y (tap positions b = bmid + bslope t', z = zmid + zslope t', t' = t - (n_drive-1)/2),
// mode 2 = driven along z (x and y positions per sample from the FP64 fields).
struct Ray3D {
    int lo, hi, mode;
    float weight;
    double zmid, zslope;            // modes 0/1
    double xmid, xs, ymid, ys;      // mode 2
};

__device__ __forceinline__ void clip_range(double mid, double sl, double tmid, int n, int &lo,
                                           int &hi)
{
    if (sl == 0.0) {
        if (!(mid >= -1.0 && mid < n)) hi = lo - 1;
        return;
    }
    const double r = 1.0 / sl;
    const double ta = tmid + (-1.0 - mid) * r, tb = tmid + ((double)n - mid) * r;
    const double tl = fmin(ta, tb), th = fmax(ta, tb);
    const double clo = ceil(tl - 1e-6), chi = floor(th + 1e-6);
    if (clo > lo) lo = (clo > hi + 1) ? hi + 1 : (int)clo;
    if (chi < hi) hi = (chi < lo - 1) ? lo - 1 : (int)chi;
}

__device__ __forceinline__ Ray3D setup_ray3d(const RayXY &R, int iv, int ndv, double pitch_v,
                                             double h, int nx, int ny, int nz)
{
    Ray3D q;
    const double v = (iv - 0.5 * (ndv - 1)) * pitch_v;
    if (fabs(v) * fabs(R.rda) <= 1.0) {
        // driven along x or y (ties with z go to x / y): the in-plane part comes from the
        // column table, the second tap axis is z
        q.mode = (R.packed >> 30) & 3;
        q.lo = R.packed & 0x7fff;
        q.hi = (R.packed >> 15) & 0x7fff;
        const int n_drive = q.mode == 0 ? nx : ny;
        q.zslope = v * R.rda;                              // dz per plane (index units)
        q.zmid = 0.5 * (nz - 1) - R.sa_h * q.zslope;       // z at the central driving plane
        clip_range(q.zmid, q.zslope, 0.5 * (n_drive - 1), nz, q.lo, q.hi);
        q.weight = (float)(h * sqrt(R.dxy2 + q.zslope * q.zslope));     // h |D| / |Da|
    } else {
        // driven along z: the ray meets plane z_k = (k - (nz-1)/2) h at
        // x = S_x + z_k D_x / v (S_z = 0), i.e. x(k) = S_x/h + (nx-1)/2 + (k - (nz-1)/2) D_x/v
        q.mode = 2;
        q.lo = 0;
        q.hi = nz - 1;
        q.xs = R.dx / v;
        q.ys = R.dy / v;
        q.xmid = R.sx_h + 0.5 * (nx - 1);
        q.ymid = R.sy_h + 0.5 * (ny - 1);
        clip_range(q.xmid, q.xs, 0.5 * (nz - 1), nx, q.lo, q.hi);
        clip_range(q.ymid, q.ys, 0.5 * (nz - 1), ny, q.lo, q.hi);
        q.weight = (float)(h * sqrt(1.0 + q.xs * q.xs + q.ys * q.ys));
    }
    return q;
}

// z slope and z at the central driving plane of row iv of a column (x- or y-driven rows), in
// FP32 from the table's pairs: with c = iv - (ndv - 1) / 2 (exact), zs = c (pitch_v / Da) and
// zm = (nz - 1) / 2 - c (pitch_v Sa / (h Da)), each product carried to about one FP32 rounding
// (the low halves and the product's exact error folded in).  No FP64 instruction: on GB300 the
// FP64 set-up of a thread's rays took a quarter of the FP64 pipe's cycles of the kernel.
__device__ __forceinline__ void ray_z_f32(const RayXY &R, int iv, int ndv, int nz, float &zs,
                                          float &zm)
{
    const float c = (float)iv - 0.5f * (float)(ndv - 1);
    zs = fmaf(c, R.zp_hi, c * R.zp_lo);
    const float p = c * R.zq_hi;
    const float e = fmaf(c, R.zq_hi, -p);
    zm = (0.5f * (float)(nz - 1) - p) - fmaf(c, R.zq_lo, e);
}

// The volume is processed in z slabs so that the pair rows a launch reads stay in L2: slab s
// owns the samples whose lower tap row r = floor(z) + 1 (padded row index) lies in
// [r_lo, r_hi); membership is decided on the same FP32 position the sample uses, so every
// sample belongs to exactly one slab.  Launches after the first of a call add to y.
constexpr int kJ3Batch = 4;   // planes per batch of the cone Joseph loop

// at most 85 registers a thread (three blocks of 256 threads per SM) for the batched gathers
template <bool SLAB>
__global__ void __launch_bounds__(256, 3) joseph3d_kernel(
    const RayXY *__restrict__ rxy, int ndu, int ndv, double pitch_v, double h,
    const float2 *__restrict__ px, int64_t zsx, int ldx, const float2 *__restrict__ py,
    int64_t zsy, int ldy, int chunk, int nx, int ny, int nz, float *__restrict__ y,
    int64_t y_view_ld, int y_ld, int y_off, int iv0, int iv1, int r_lo, int r_hi, int accumulate,
    const int *stop)
{
    if (stop && stop[0] != 0) return;
    // a block is 32 detector columns x blockDim.y detector rows of one view (a warp is one row):
    // neighbouring rows cross neighbouring z rows of the pair layouts, which they share in L1
    const int iu = blockIdx.x * 32 + threadIdx.x;
    const int view = blockIdx.y;
    const int iv_raw = iv0 + blockIdx.z * blockDim.y + threadIdx.y;
    const bool valid = iu < ndu && iv_raw <= iv1;   // all lanes stay for the warp-wide range
    const int iv = valid ? iv_raw : iv0;
    const RayXY R = rxy[(int64_t)view * ndu + (valid ? iu : 0)];
    const bool zdrive = iv < R.iv_lo || iv > R.iv_hi;    // |v| > |Da|: driven along z
    const int mode = zdrive ? 2 : (int)((R.packed >> 30) & 3);
    const bool ax = mode == 0;
    const int n_drive = ax ? nx : ny;
    const float tmid = 0.5f * (float)(n_drive - 1);
    // z of the samples: z(t) = zmid + zslope (t - tmid), zslope = v / Da
    float zs, zm;
    ray_z_f32(R, iv, ndv, nz, zs, zm);
    float acc = 0.f;
    bool any = false;
    int lo = R.packed & 0x7fff, hi = (R.packed >> 15) & 0x7fff;
    if (!valid || zdrive) {
        lo = 1;
        hi = 0;
    } else if (fabsf(zs) > 1e-20f) {
        // planes whose z can fall in [r_lo - 2, r_hi] (the slab's tap rows, FP32, two planes of
        // margin); samples outside the volume add zero, so a superset is enough
        const float r = __frcp_rn(zs);
        const float ta = tmid + ((float)(r_lo - 2) - zm) * r;
        const float tb = tmid + ((float)r_hi - zm) * r;
        lo = max(lo, (int)floorf(fminf(ta, tb)) - 2);
        hi = min(hi, (int)ceilf(fmaxf(ta, tb)) + 2);
    }
    // the warp steps through the union of its lanes' plane ranges together, so that at every
    // step its lanes read neighbouring pairs of one row (a lane outside its own range idles)
    const int wlo = __reduce_min_sync(0xffffffffu, hi >= lo ? lo : 0x7fffffff);
    const int whi = __reduce_max_sync(0xffffffffu, hi >= lo ? hi : -1);
    if (wlo <= whi) {
        const float2 *L = ax ? px : py;
        const int64_t zsl = ax ? zsx : zsy;       // pairs per z slice
        const int ld = ax ? ldx : ldy;            // pairs per row (one step along the drive)
        const float bhi = (float)(ax ? ny : nx), zhi = (float)nz;
        const float bmid = R.bmid, bsl = R.bslope;
        // taps of the sample on driving row t: pair fb + 1 of row t + 1 in slices fz + 1 and
        // fz + 2.  floor(pb), floor(pz) and the address come from round-down additions (as in
        // the 2D kernel): sb = 2^23 + 2 + (t - t0) ld + floor(pb), sz = 2^23 + 2 + floor(pz)
        // exactly, so the byte address is chunk_base + 8 bits(sb) + 8 zsl bits(sz).
        const uint64_t zsl8 = 8ull * (uint64_t)zsl;
        const uint64_t b23 = __float_as_uint(kFloor2p23);
        const uint64_t lbase = reinterpret_cast<uint64_t>(L) + 8ull * (uint64_t)ld - 8ull * (b23 + 1ull) -
                               zsl8 * (b23 + 1ull);
        const float fz_lo = (float)(r_lo - 1), fz_hi = (float)(r_hi - 1);   // slab: r = fz + 1
        float tf = (float)wlo - tmid;
        // branch-free body (positions are clamped, so every load is in bounds; a sample outside
        // the lane's range or the slab is weighted by zero), in batches of planes so that the
        // loads of several planes are in flight together
        // the z and in-plane coordinates of a sample as one pair (z, b): positions, floors and
        // weights in paired FP32 arithmetic, the same operations per coordinate
        const float2 sl2 = make_float2(zs, bsl), mid2 = make_float2(zm, bmid);
        const float2 m1 = make_float2(-1.f, -1.f), one2 = make_float2(1.f, 1.f);
        float2 tf2 = make_float2(tf, tf);
        for (int t0 = wlo; t0 <= whi; t0 += chunk) {
            const int t1 = min(whi, t0 + chunk - 1);
            const uint64_t cb = lbase + 8ull * (uint64_t)t0 * (uint64_t)ld;
            float2 K2 = make_float2(kFloorK0, kFloorK0);     // (z, b + (t - t0) ld)
            const float2 dK2 = make_float2(0.f, (float)ld);
            // batches of NB planes: the NB samples' positions, weights and addresses first, then
            // their 2 NB gathers, then the sums in plane order (the same operations and order as
            // one plane at a time); single planes finish the range
            constexpr int NB = kJ3Batch;
            int t = t0;
            for (; t1 - t >= NB - 1; t += NB) {
                uint64_t ad[NB];
                float wzq[NB], wbq[NB];
                bool inq[NB];
                float2 p0q[NB], p1q[NB];
#pragma unroll
                for (int q = 0; q < NB; ++q) {
                    const float2 q2 = __ffma2_rn(sl2, tf2, mid2);
                    const float2 p2 = make_float2(fminf(fmaxf(q2.x, -1.f), zhi), fminf(fmaxf(q2.y, -1.f), bhi));
                    const float2 s2 = __fadd2_rd(p2, K2);
                    const float2 fl2 = __ffma2_rn(K2, m1, s2);
                    const float2 w2 = __ffma2_rn(fl2, m1, p2);
                    wzq[q] = w2.x;
                    wbq[q] = w2.y;
                    ad[q] = cb + 8ull * __float_as_uint(s2.y) + zsl8 * __float_as_uint(s2.x);
                    const int tq = t + q;
                    inq[q] = tq >= lo && tq <= hi && (!SLAB || (fl2.x >= fz_lo && fl2.x < fz_hi));
                    tf2 = __fadd2_rn(tf2, one2);
                    K2 = __fadd2_rn(K2, dK2);
                }
#pragma unroll
                for (int q = 0; q < NB; ++q) {
                    p0q[q] = __ldg(reinterpret_cast<const float2 *>(ad[q]));
                    p1q[q] = __ldg(reinterpret_cast<const float2 *>(ad[q] + zsl8));
                }
#pragma unroll
                for (int q = 0; q < NB; ++q) {
                    const float a0v = fmaf(wbq[q], p0q[q].y, p0q[q].x);
                    const float a1v = fmaf(wbq[q], p1q[q].y, p1q[q].x);
                    acc += inq[q] ? fmaf(wzq[q], a1v - a0v, a0v) : 0.f;
                    any |= inq[q];
                }
            }
#pragma unroll 4
            for (; t <= t1; ++t) {
                const float2 q2 = __ffma2_rn(sl2, tf2, mid2);
                const float2 p2 = make_float2(fminf(fmaxf(q2.x, -1.f), zhi), fminf(fmaxf(q2.y, -1.f), bhi));
                const float2 s2 = __fadd2_rd(p2, K2);                  // (sz, sb)
                const float2 fl2 = __ffma2_rn(K2, m1, s2);             // (fz, sb - Kb)
                const float2 w2 = __ffma2_rn(fl2, m1, p2);             // (wz, wb)
                const float fz = fl2.x, wz = w2.x, wb = w2.y;
                const float sb = s2.y, sz = s2.x;
                const uint64_t a0 = cb + 8ull * __float_as_uint(sb) + zsl8 * __float_as_uint(sz);
                const float2 p0 = __ldg(reinterpret_cast<const float2 *>(a0));
                const float2 p1 = __ldg(reinterpret_cast<const float2 *>(a0 + zsl8));
                const float a0v = fmaf(wb, p0.y, p0.x);
                const float a1v = fmaf(wb, p1.y, p1.x);
                const bool in = t >= lo && t <= hi && (!SLAB || (fz >= fz_lo && fz < fz_hi));
                acc += in ? fmaf(wz, a1v - a0v, a0v) : 0.f;
                any |= in;
                tf2 = __fadd2_rn(tf2, one2);
                K2 = __fadd2_rn(K2, dK2);
            }
        }
    }
    float weight = (float)h * sqrtf(R.dxy2 + zs * zs);                  // h |D| / |Da|
    if (valid && zdrive) {
        // driven along z (FP64 per sample; rare): plane t meets the ray at
        // x = S_x/h + (nx-1)/2 + (t - (nz-1)/2) D_x / v, likewise y; taps from P_y (pairs
        // along x; slice t + 1, rows y + 1 and y + 2); plane t is in the slab when t + 1 is
        const Ray3D q = setup_ray3d(R, iv, ndv, pitch_v, h, nx, ny, nz);
        weight = q.weight;
        const double zt = 0.5 * (nz - 1);
        const float xhi = (float)nx, yhi = (float)ny;
        const int zlo = max(q.lo, r_lo - 1), zhi2 = min(q.hi, r_hi - 2);
        for (int t = zlo; t <= zhi2; ++t) {
            const double tf = t - zt;
            const float pxf = fminf(fmaxf((float)(q.xmid + q.xs * tf), -1.f), xhi);
            const float pyf = fminf(fmaxf((float)(q.ymid + q.ys * tf), -1.f), yhi);
            const float fx = floorf(pxf), fy = floorf(pyf);
            const float wx = pxf - fx, wy = pyf - fy;
            const float2 *row = py + (int64_t)(t + 1) * zsy + (int64_t)((int)fy + 1) * ldy + (int)fx + 1;
            const float2 p0 = __ldg(row), p1 = __ldg(row + ldy);
            const float a0 = fmaf(wx, p0.y, p0.x);
            const float a1 = fmaf(wx, p1.y, p1.x);
            acc += fmaf(wy, a1 - a0, a0);
            any = true;
        }
    }
    if (!valid) return;
    float *out = y + (int64_t)view * y_view_ld + (int64_t)iv * y_ld + y_off + iu;
    if (!accumulate) *out = acc * weight;
    else if (any) *out += acc * weight;
}

// The same projector with two rays per thread: detector rows iv and iv + 1 of one column iu.
// Their x-y projections coincide (the fan ray of the column), so at every driving plane they
// share the in-plane tap position, its floor, weight and address part; only z differs (the two
// z coordinates run as one f32x2 pair).  Each ray's plane range is made exact for the
// loop's own FP32 arithmetic: the planes whose z = fma(zslope, t - tmid, zmid) lies in
// [-1, nz] (monotone in t, so an interval, found from an FP32 estimate and checked at its ends).
// Inside that range a sample's taps are slices floor(z) + 1 .. floor(z) + 2 in [0, nz + 2] and
// its in-plane pair index is in [-1, n + 1] (the host range keeps b in [-1, n] up to FP32
// rounding; index -1 is the previous row's zero tail), so no position needs a clamp; lanes
// outside their own range skip the loads.  The samples this leaves out are those whose taps
// all lie in the zero margins, which the one-ray kernel adds as exact zeros: the sums, taken in
// the same order with the same operations, are bitwise those of joseph3d_kernel.  Planes go in
// batches of kJ3PairBatch (four gathers per plane).
constexpr int kJ3PairBatch = 2;

// planes of [lo, hi] whose FP32 z lies in [-1, zhi] (lo > hi when there is none)
__device__ __forceinline__ void exact_z_range(float zs, float zm, float tmid, float zhi, int &lo,
                                              int &hi)
{
    auto zin = [&](int t) {
        const float z = fmaf(zs, (float)t - tmid, zm);
        return z >= -1.f && z <= zhi;
    };
    if (lo > hi) return;
    if (zs == 0.f) {
        if (!zin(lo)) hi = lo - 1;
        return;
    }
    // the crossings of z = -1 and z = zhi in FP32 (within a plane of the exact ones), widened by
    // two planes and clipped to [lo, hi]; then the ends are stepped inwards to the first planes
    // inside (at most eight steps; with none found the range is empty)
    const float r = __frcp_rn(zs);
    const float ta = tmid + (-1.f - zm) * r, tb = tmid + (zhi - zm) * r;
    const float flo = fmaxf((float)lo, fminf((float)hi, floorf(fminf(ta, tb)) - 2.f));
    const float fhi = fmaxf((float)lo, fminf((float)hi, ceilf(fmaxf(ta, tb)) + 2.f));
    int a = (int)flo, b = (int)fhi;
    for (int i = 0; i < 8 && a <= b && !zin(a); ++i) ++a;
    for (int i = 0; i < 8 && b >= a && !zin(b); --b, ++i) {}
    if (a > b || !zin(a) || !zin(b)) {
        hi = lo - 1;
        return;
    }
    lo = a;
    hi = b;
}

// planes whose z can fall in a slab's tap rows [r_lo - 2, r_hi] (FP32, two planes of margin;
// a superset: membership is decided per sample)
__device__ __forceinline__ void ray_z_range(float zs, float tmid, float zm, int r_lo, int r_hi,
                                            int &lo, int &hi)
{
    if (fabsf(zs) > 1e-20f) {
        const float r = __frcp_rn(zs);
        const float ta = tmid + ((float)(r_lo - 2) - zm) * r;
        const float tb = tmid + ((float)r_hi - zm) * r;
        lo = max(lo, (int)floorf(fminf(ta, tb)) - 2);
        hi = min(hi, (int)ceilf(fmaxf(ta, tb)) + 2);
    }
}

template <bool SLAB>
__global__ void __launch_bounds__(256, 3) joseph3d_pair_kernel(
    const RayXY *__restrict__ rxy, int ndu, int ndv, double pitch_v, double h,
    const float2 *__restrict__ px, int64_t zsx, int ldx, const float2 *__restrict__ py,
    int64_t zsy, int ldy, int chunk, int nx, int ny, int nz, float *__restrict__ y,
    int64_t y_view_ld, int y_ld, int y_off, int iv0, int iv1, int r_lo, int r_hi, int accumulate,
    const int *stop)
{
    if (stop && stop[0] != 0) return;
    // a block is 32 detector columns x 2 blockDim.y detector rows of one view; warp w takes rows
    // 2w and 2w + 1 of the block (rays a and b of each lane)
    const int iu = blockIdx.x * 32 + threadIdx.x;
    const int view = blockIdx.y;
    const int iva_raw = iv0 + 2 * (blockIdx.z * blockDim.y + threadIdx.y);
    const bool col_ok = iu < ndu;
    const bool va_ok = col_ok && iva_raw <= iv1, vb_ok = col_ok && iva_raw + 1 <= iv1;
    const int iva = va_ok ? iva_raw : iv0, ivb = vb_ok ? iva_raw + 1 : iv0;
    const RayXY R = rxy[(int64_t)view * ndu + (col_ok ? iu : 0)];
    const bool zda = iva < R.iv_lo || iva > R.iv_hi, zdb = ivb < R.iv_lo || ivb > R.iv_hi;
    const int mode = (int)((R.packed >> 30) & 3);          // in-plane driving axis
    const bool ax = mode == 0;
    const int n_drive = ax ? nx : ny;
    const float tmid = 0.5f * (float)(n_drive - 1);
    float zsa, zma, zsb, zmb;
    ray_z_f32(R, iva, ndv, nz, zsa, zma);
    ray_z_f32(R, ivb, ndv, nz, zsb, zmb);
    const float zhi = (float)nz;
    float acca = 0.f, accb = 0.f;
    bool anya = false, anyb = false;
    const int lo0 = R.packed & 0x7fff, hi0 = (R.packed >> 15) & 0x7fff;
    int loa = lo0, hia = hi0, lob = lo0, hib = hi0;
    if (!va_ok || zda) { loa = 1; hia = 0; }
    else {
        exact_z_range(zsa, zma, tmid, zhi, loa, hia);
        if (SLAB) ray_z_range(zsa, tmid, zma, r_lo, r_hi, loa, hia);
    }
    if (!vb_ok || zdb) { lob = 1; hib = 0; }
    else {
        exact_z_range(zsb, zmb, tmid, zhi, lob, hib);
        if (SLAB) ray_z_range(zsb, tmid, zmb, r_lo, r_hi, lob, hib);
    }
    const int tlo = min(hia >= loa ? loa : 0x7fffffff, hib >= lob ? lob : 0x7fffffff);
    const int thi = max(hia >= loa ? hia : -1, hib >= lob ? hib : -1);
    const int wlo = __reduce_min_sync(0xffffffffu, tlo);
    const int whi = __reduce_max_sync(0xffffffffu, thi);
    if (wlo <= whi) {
        const float2 *L = ax ? px : py;
        const int64_t zsl = ax ? zsx : zsy;
        const int ld = ax ? ldx : ldy;
        const float bmid = R.bmid, bsl = R.bslope;
        const uint32_t zsl8 = 8u * (uint32_t)zsl;           // < 2^32: checked by the launcher
        const uint64_t zsl8w = zsl8;
        const uint64_t b23 = __float_as_uint(kFloor2p23);
        const uint64_t lbase = reinterpret_cast<uint64_t>(L) + 8ull * (uint64_t)ld - 8ull * (b23 + 1ull) -
                               zsl8w * (b23 + 1ull);
        const float fz_lo = (float)(r_lo - 1), fz_hi = (float)(r_hi - 1);
        const float2 zs2 = make_float2(zsa, zsb), zm2 = make_float2(zma, zmb);
        const float2 m1 = make_float2(-1.f, -1.f);
        const float2 Kz2 = make_float2(kFloorK0, kFloorK0);
        // a ray's planes [lo, hi] as an unsigned window: t in range iff (t - lo) <= (hi - lo)
        const uint32_t wa = hia >= loa ? (uint32_t)(hia - loa) : 0u;
        const uint32_t wb_ = hib >= lob ? (uint32_t)(hib - lob) : 0u;
        const int la = hia >= loa ? loa : 0x3fffffff, lb = hib >= lob ? lob : 0x3fffffff;
        float tf = (float)wlo - tmid;
        for (int t0 = wlo; t0 <= whi; t0 += chunk) {
            const int t1 = min(whi, t0 + chunk - 1);
            const uint64_t cb = lbase + 8ull * (uint64_t)t0 * (uint64_t)ld;
            float Kb = kFloorK0;                             // b + (t - t0) ld
            const float dKb = (float)ld;
            constexpr int NB = kJ3PairBatch;
            int t = t0;
            for (; t1 - t >= NB - 1; t += NB) {
                uint64_t ada[NB], adb[NB];
                float wbq[NB];
                float2 wzq[NB];
                bool ina[NB], inb[NB];
                float2 p0a[NB], p1a[NB], p0b[NB], p1b[NB];
#pragma unroll
                for (int q = 0; q < NB; ++q) {
                    // in-plane coordinate (shared): the b half of the one-ray kernel's (z, b)
                    // pair, without its clamp
                    const float pb = fmaf(bsl, tf, bmid);
                    const float sb = __fadd_rd(pb, Kb);
                    const float flb = fmaf(Kb, -1.f, sb);
                    wbq[q] = fmaf(flb, -1.f, pb);
                    const float2 pz = __ffma2_rn(zs2, make_float2(tf, tf), zm2);
                    const float2 sz = __fadd2_rd(pz, Kz2);
                    const float2 flz = __ffma2_rn(Kz2, m1, sz);
                    wzq[q] = __ffma2_rn(flz, m1, pz);
                    const uint64_t base = cb + 8ull * (uint64_t)__float_as_uint(sb);
                    ada[q] = base + (uint64_t)zsl8 * __float_as_uint(sz.x);
                    adb[q] = base + (uint64_t)zsl8 * __float_as_uint(sz.y);
                    const int tq = t + q;
                    ina[q] = (uint32_t)(tq - la) <= wa && (!SLAB || (flz.x >= fz_lo && flz.x < fz_hi));
                    inb[q] = (uint32_t)(tq - lb) <= wb_ && (!SLAB || (flz.y >= fz_lo && flz.y < fz_hi));
                    tf += 1.f;
                    Kb += dKb;
                }
#pragma unroll
                for (int q = 0; q < NB; ++q) {
                    if (ina[q]) {
                        p0a[q] = __ldg(reinterpret_cast<const float2 *>(ada[q]));
                        p1a[q] = __ldg(reinterpret_cast<const float2 *>(ada[q] + zsl8w));
                    }
                    if (inb[q]) {
                        p0b[q] = __ldg(reinterpret_cast<const float2 *>(adb[q]));
                        p1b[q] = __ldg(reinterpret_cast<const float2 *>(adb[q] + zsl8w));
                    }
                }
#pragma unroll
                for (int q = 0; q < NB; ++q) {
                    if (ina[q]) {
                        const float a0 = fmaf(wbq[q], p0a[q].y, p0a[q].x);
                        const float a1 = fmaf(wbq[q], p1a[q].y, p1a[q].x);
                        acca += fmaf(wzq[q].x, a1 - a0, a0);
                        if (SLAB) anya = true;
                    }
                    if (inb[q]) {
                        const float b0 = fmaf(wbq[q], p0b[q].y, p0b[q].x);
                        const float b1 = fmaf(wbq[q], p1b[q].y, p1b[q].x);
                        accb += fmaf(wzq[q].y, b1 - b0, b0);
                        if (SLAB) anyb = true;
                    }
                }
            }
            for (; t <= t1; ++t) {
                const float pb = fmaf(bsl, tf, bmid);
                const float sb = __fadd_rd(pb, Kb);
                const float flb = fmaf(Kb, -1.f, sb);
                const float wb = fmaf(flb, -1.f, pb);
                const float2 pz = __ffma2_rn(zs2, make_float2(tf, tf), zm2);
                const float2 sz = __fadd2_rd(pz, Kz2);
                const float2 flz = __ffma2_rn(Kz2, m1, sz);
                const float2 wz = __ffma2_rn(flz, m1, pz);
                const uint64_t base = cb + 8ull * (uint64_t)__float_as_uint(sb);
                const bool ia = (uint32_t)(t - la) <= wa && (!SLAB || (flz.x >= fz_lo && flz.x < fz_hi));
                const bool ib = (uint32_t)(t - lb) <= wb_ && (!SLAB || (flz.y >= fz_lo && flz.y < fz_hi));
                if (ia) {
                    const uint64_t a_ = base + (uint64_t)zsl8 * __float_as_uint(sz.x);
                    const float2 q0a = __ldg(reinterpret_cast<const float2 *>(a_));
                    const float2 q1a = __ldg(reinterpret_cast<const float2 *>(a_ + zsl8w));
                    const float a0 = fmaf(wb, q0a.y, q0a.x);
                    const float a1 = fmaf(wb, q1a.y, q1a.x);
                    acca += fmaf(wz.x, a1 - a0, a0);
                    if (SLAB) anya = true;
                }
                if (ib) {
                    const uint64_t b_ = base + (uint64_t)zsl8 * __float_as_uint(sz.y);
                    const float2 q0b = __ldg(reinterpret_cast<const float2 *>(b_));
                    const float2 q1b = __ldg(reinterpret_cast<const float2 *>(b_ + zsl8w));
                    const float b0 = fmaf(wb, q0b.y, q0b.x);
                    const float b1 = fmaf(wb, q1b.y, q1b.x);
                    accb += fmaf(wz.y, b1 - b0, b0);
                    if (SLAB) anyb = true;
                }
                tf += 1.f;
                Kb += dKb;
            }
        }
    }
    float wa_ = (float)h * sqrtf(R.dxy2 + zsa * zsa), wbw = (float)h * sqrtf(R.dxy2 + zsb * zsb);
    // rays driven along z (FP64 per sample; rare): as in the single-ray kernel
    for (int r = 0; r < 2; ++r) {
        const bool ok = r == 0 ? (va_ok && zda) : (vb_ok && zdb);
        if (!ok) continue;
        const int iv = r == 0 ? iva : ivb;
        const Ray3D q = setup_ray3d(R, iv, ndv, pitch_v, h, nx, ny, nz);
        const double zt = 0.5 * (nz - 1);
        const float xhi = (float)nx, yhi = (float)ny;
        const int zlo = max(q.lo, r_lo - 1), zhi2 = min(q.hi, r_hi - 2);
        float acc = 0.f;
        bool any = false;
        for (int t = zlo; t <= zhi2; ++t) {
            const double tfd = t - zt;
            const float pxf = fminf(fmaxf((float)(q.xmid + q.xs * tfd), -1.f), xhi);
            const float pyf = fminf(fmaxf((float)(q.ymid + q.ys * tfd), -1.f), yhi);
            const float fx = floorf(pxf), fy = floorf(pyf);
            const float wx = pxf - fx, wy = pyf - fy;
            const float2 *row = py + (int64_t)(t + 1) * zsy + (int64_t)((int)fy + 1) * ldy + (int)fx + 1;
            const float2 p0 = __ldg(row), p1 = __ldg(row + ldy);
            const float a0 = fmaf(wx, p0.y, p0.x);
            const float a1 = fmaf(wx, p1.y, p1.x);
            acc += fmaf(wy, a1 - a0, a0);
            any = true;
        }
        if (r == 0) { acca = acc; anya = any; wa_ = q.weight; }
        else { accb = acc; anyb = any; wbw = q.weight; }
    }
    if (va_ok) {
        float *out = y + (int64_t)view * y_view_ld + (int64_t)iva * y_ld + y_off + iu;
        if (!accumulate) *out = acca * wa_;
        else if (anya) *out += acca * wa_;
    }
    if (vb_ok) {
        float *out = y + (int64_t)view * y_view_ld + (int64_t)ivb * y_ld + y_off + iu;
        if (!accumulate) *out = accb * wbw;
        else if (anyb) *out += accb * wbw;
    }
}

// Total number of Joseph samples of the geometry (sum of the clipped plane ranges), for the
// projector's work count.
__global__ void joseph3d_count_kernel(const RayXY *__restrict__ rxy, int ndu, int ndv,
                                      int n_views, double pitch_v, double h, int nx, int ny,
                                      int nz, unsigned long long *count)
{
    const int64_t total = (int64_t)n_views * ndu * ndv;
    unsigned long long local = 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = t / ndv;
        const int iv = (int)(t - col * ndv);
        const Ray3D q = setup_ray3d(rxy[col], iv, ndv, pitch_v, h, nx, ny, nz);
        if (q.hi >= q.lo) local += (unsigned long long)(q.hi - q.lo + 1);
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(count, local);
}

cudaError_t count_joseph3d_samples(const ct_geom *g, int64_t *out)
{
    const DeviceGeom &d = g->dg;
    unsigned long long *cnt = nullptr, h = 0;
    cudaError_t e = cudaMalloc(&cnt, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(cnt, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) {
        joseph3d_count_kernel<<<152 * 8, 256>>>(d.rays_xy, d.ndu, d.ndv, d.n_views,
                                                (double)g->desc.pitch_v, g->desc.pixel, d.nx,
                                                d.ny, d.nz, cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(cnt);
    *out = (int64_t)h;
    return e;
}

// Detector rows that can see physical heights [z_a, z_b] of a volume whose x-y cross-section
// lies within radius rxy of the axis: v = SDD z / (SID - p . d) with |p . d| <= rxy.
static void rows_for_heights(const ct_geom *g, double z_a, double z_b, int &iv_lo, int &iv_hi)
{
    const ct_geom_desc &d = g->desc;
    // taps may sit one voxel outside the volume: widen the radius by two voxels
    const double rxy = 0.5 * d.pixel * sqrt((double)d.nx * d.nx + (double)d.ny * d.ny) + 2.0 * d.pixel;
    double vmin = 1e300, vmax = -1e300;
    for (double z : {z_a, z_b})
        for (double sd : {-rxy, rxy}) {
            const double v = d.sdd * z / (d.sid - sd);
            vmin = std::min(vmin, v);
            vmax = std::max(vmax, v);
        }
    const double c = 0.5 * (d.n_det_v - 1);
    iv_lo = std::max(0, (int)floor(vmin / d.pitch_v + c) - 2);
    iv_hi = std::min(d.n_det_v - 1, (int)ceil(vmax / d.pitch_v + c) + 2);
}

cudaError_t launch_joseph3d(const ct_geom *g, float *y, int64_t y_view_ld, int y_ld, int y_off,
                            const int *stop, cudaStream_t s)
{
    const DeviceGeom &d = g->dg;
    const int slab = d.tune_a_slab > 0 ? d.tune_a_slab : 16;
    const int n_rows = d.nz + 1;                 // padded tap rows r = floor(z) + 1 in [0, nz]
    const int n_slabs = (n_rows + slab - 1) / slab;
    if (n_slabs > 1) {
        // every launch adds to y: start from zero (margins of a padded layout stay zero)
        const size_t total = (size_t)d.n_views * (size_t)y_view_ld;
        cudaError_t e = cudaMemsetAsync(y, 0, sizeof(float) * total, s);
        if (e != cudaSuccess) return e;
    }
    const double h = g->desc.pixel, zc = 0.5 * (d.nz - 1);
    // rows per chunk whose offsets (t - t0) ld the floor additions carry; one value for both
    // layouts keeps the sample loop's bounds warp-uniform
    const int chunk = floor_chunk(std::max(d.row_pairs_ld, d.col_pairs_ld));
    for (int k = 0; k < n_slabs; ++k) {
        const int r_lo = k * slab, r_hi = std::min(n_rows, (k + 1) * slab);
        int iv_lo = 0, iv_hi = d.ndv - 1;
        if (n_slabs > 1) {
            // heights the slab's samples touch: z index in [r_lo - 2, r_hi], one of margin
            rows_for_heights(g, (r_lo - 2 - zc) * h, (r_hi - zc) * h, iv_lo, iv_hi);
            if (iv_hi < iv_lo) continue;
        }
        const int vb = (d.tune_a_views >= 1 && d.tune_a_views <= 8) ? d.tune_a_views : 8;
        // the two-ray kernel forms slice offsets as 32-bit products: 8 pairs-per-slice < 2^32
        if (d.tune_a_rays == 2 && 8ull * (uint64_t)std::max(d.slice_x, d.slice_y) < (1ull << 32)) {
            // two detector rows per thread: blocks of 32 columns x 2 vb rows
            dim3 block(32, vb), grid((d.ndu + 31) / 32, d.n_views, (iv_hi - iv_lo + 2 * vb) / (2 * vb));
            if (n_slabs > 1)
                joseph3d_pair_kernel<true><<<grid, block, 0, s>>>(
                    d.rays_xy, d.ndu, d.ndv, (double)g->desc.pitch_v, h, g->pcol_dev, d.slice_x,
                    d.col_pairs_ld, g->prow_dev, d.slice_y, d.row_pairs_ld, chunk, d.nx, d.ny, d.nz,
                    y, y_view_ld, y_ld, y_off, iv_lo, iv_hi, r_lo, r_hi, 1, stop);
            else
                joseph3d_pair_kernel<false><<<grid, block, 0, s>>>(
                    d.rays_xy, d.ndu, d.ndv, (double)g->desc.pitch_v, h, g->pcol_dev, d.slice_x,
                    d.col_pairs_ld, g->prow_dev, d.slice_y, d.row_pairs_ld, chunk, d.nx, d.ny, d.nz,
                    y, y_view_ld, y_ld, y_off, iv_lo, iv_hi, r_lo, r_hi, 0, stop);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            continue;
        }
        dim3 block(32, vb), grid((d.ndu + 31) / 32, d.n_views, (iv_hi - iv_lo + vb) / vb);
        if (n_slabs > 1)
            joseph3d_kernel<true><<<grid, block, 0, s>>>(
                d.rays_xy, d.ndu, d.ndv, (double)g->desc.pitch_v, h, g->pcol_dev, d.slice_x,
                d.col_pairs_ld, g->prow_dev, d.slice_y, d.row_pairs_ld, chunk, d.nx, d.ny, d.nz, y,
                y_view_ld, y_ld, y_off, iv_lo, iv_hi, r_lo, r_hi, 1, stop);
        else   // one pass: every tap row is in [0, nz + 1], no slab test
            joseph3d_kernel<false><<<grid, block, 0, s>>>(
                d.rays_xy, d.ndu, d.ndv, (double)g->desc.pitch_v, h, g->pcol_dev, d.slice_x,
                d.col_pairs_ld, g->prow_dev, d.slice_y, d.row_pairs_ld, chunk, d.nx, d.ny, d.nz, y,
                y_view_ld, y_ld, y_off, iv_lo, iv_hi, r_lo, r_hi, 0, stop);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// number of kernel launches one launch_joseph3d makes (for the library's launch count)
int joseph3d_launches(const ct_geom *g)
{
    const DeviceGeom &d = g->dg;
    const int slab = d.tune_a_slab > 0 ? d.tune_a_slab : 16;
    return (d.nz + 1 + slab - 1) / slab;
}

// ---------------------------------------------------------------------------- matched adjoint
// x = A^T y for the cone Joseph projector (the matched case of Sec. 2): one thread per ray
// walks the ray's samples with the forward kernel's FP32 positions (rays driven along x or y:
// b = bmid + bslope t', z = zmid + zslope t' over the ray's in-plane range; rays driven along
// z: x and y from the FP64 fields per plane) and scatters weight * y_ray times the four
// bilinear weights to the taps inside the volume, by atomic FP64 additions (rounded to FP32 by
// a second kernel).  Samples the forward kernel skips (z beyond the volume by more than a
// plane) have all four taps outside and add nothing here either.
__global__ void __launch_bounds__(256) joseph3d_adjoint_kernel(
    const RayXY *__restrict__ rxy, int n_views, int ndu, int ndv, double pitch_v, double h,
    const float *__restrict__ y, int64_t y_view_ld, int y_ld, int y_off, int nx, int ny, int nz,
    double *__restrict__ acc, const int *stop)
{
    if (stop && stop[0] != 0) return;
    const int64_t ray = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (ray >= (int64_t)n_views * ndv * ndu) return;
    const int iu = (int)(ray % ndu);
    const int64_t vr = ray / ndu;
    const int iv = (int)(vr % ndv), view = (int)(vr / ndv);
    const RayXY R = rxy[(int64_t)view * ndu + iu];
    const float yv = y[(int64_t)view * y_view_ld + (int64_t)iv * y_ld + y_off + iu];
    const int64_t sxy = (int64_t)nx * ny;
    const bool zdrive = iv < R.iv_lo || iv > R.iv_hi;
    if (!zdrive) {
        const int mode = (int)((R.packed >> 30) & 3);
        const bool ax = mode == 0;
        const int n_drive = ax ? nx : ny;
        const float tmid = 0.5f * (float)(n_drive - 1);
        float zs, zm;                       // the forward kernels' z set-up
        ray_z_f32(R, iv, ndv, nz, zs, zm);
        const float s = yv * ((float)h * sqrtf(R.dxy2 + zs * zs));
        const int lo = R.packed & 0x7fff, hi = (R.packed >> 15) & 0x7fff;
        float tf = (float)lo - tmid;
        for (int t = lo; t <= hi; ++t, tf += 1.f) {
            const float pz = fmaf(zs, tf, zm), pb = fmaf(R.bslope, tf, R.bmid);
            const float fz = floorf(pz), fb = floorf(pb);
            const float wz = pz - fz, wb = pb - fb;
            const int z0 = (int)fz, b0 = (int)fb;
            if (z0 + 1 < 0 || z0 >= nz) continue;
            // (z, b) taps: b along y when driven along x (line t = x), along x when along y
            for (int dz = 0; dz < 2; ++dz) {
                const int z = z0 + dz;
                if (z < 0 || z >= nz) continue;
                const float wzz = dz ? wz : 1.f - wz;
                for (int db = 0; db < 2; ++db) {
                    const int b = b0 + db;
                    const float w = wzz * (db ? wb : 1.f - wb);
                    if (ax) {
                        if (b >= 0 && b < ny)
                            atomicAdd(acc + (int64_t)z * sxy + (int64_t)b * nx + t, (double)(s * w));
                    } else {
                        if (b >= 0 && b < nx)
                            atomicAdd(acc + (int64_t)z * sxy + (int64_t)t * nx + b, (double)(s * w));
                    }
                }
            }
        }
    } else {
        const Ray3D q = setup_ray3d(R, iv, ndv, pitch_v, h, nx, ny, nz);
        const float s = yv * q.weight;
        const double zt = 0.5 * (nz - 1);
        for (int t = q.lo; t <= q.hi; ++t) {
            const double tfd = t - zt;
            const float pxf = (float)(q.xmid + q.xs * tfd), pyf = (float)(q.ymid + q.ys * tfd);
            const float fx = floorf(pxf), fy = floorf(pyf);
            const float wx = pxf - fx, wy = pyf - fy;
            const int x0 = (int)fx, y0 = (int)fy;
            for (int dy = 0; dy < 2; ++dy) {
                const int yy = y0 + dy;
                if (yy < 0 || yy >= ny) continue;
                const float wyy = dy ? wy : 1.f - wy;
                for (int dx = 0; dx < 2; ++dx) {
                    const int xx = x0 + dx;
                    if (xx < 0 || xx >= nx) continue;
                    atomicAdd(acc + (int64_t)t * sxy + (int64_t)yy * nx + xx,
                              (double)(s * (wyy * (dx ? wx : 1.f - wx))));
                }
            }
        }
    }
}

cudaError_t launch_adjoint3d(const ct_geom *g, const float *y, int64_t y_view_ld, int y_ld,
                             int y_off, double *acc, float *x, const int *stop, cudaStream_t s)
{
    const DeviceGeom &d = g->dg;
    const int64_t n = (int64_t)d.nx * d.ny * d.nz;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)n, s);
    if (e != cudaSuccess) return e;
    const int64_t rays = (int64_t)d.n_views * d.ndv * d.ndu;
    joseph3d_adjoint_kernel<<<(unsigned)((rays + 255) / 256), 256, 0, s>>>(
        d.rays_xy, d.n_views, d.ndu, d.ndv, (double)g->desc.pitch_v, g->desc.pixel, y, y_view_ld,
        y_ld, y_off, d.nx, d.ny, d.nz, acc, stop);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_round_to_float(acc, n, x, stop, s);
}

// ---------------------------------------------------------------------------- voxel-driven B
// One thread per (x, y) column and kZChunk consecutive z; blocks of 32 x 4 columns; all views
// per thread (per-view cos and sin staged in shared memory).  With p the voxel centre in units
// of h, pe = p . e_u, bb = SID/h - p . (cos, sin), rho = 1 / bb:
//   u = SDD pe rho, v = SDD z rho, and the weight h^3 (SDD^2+u^2+v^2)^{3/2} / (L^2 pu pv SDD),
//   L = |p - S| = h bb sqrt(1 + (pe rho)^2 + (z rho)^2), equals
//   (SDD^2 h / (pu pv)) rho^2 sqrt(1 + (pe rho)^2 + (z rho)^2).
constexpr int kZChunk = 8;

__global__ void __launch_bounds__(128) voxbp3d_kernel(
    const ViewBP *__restrict__ views, int n_views, const float2 *__restrict__ ypad,
    int64_t view_ld, int ld, int ndu, int ndv, int nx, int ny, int nz, float sid_h, float ku,
    float kv, float kw, float *__restrict__ x, const int *stop)
{
    if (stop && stop[0] != 0) return;
    extern __shared__ float2 sv3[];
    const int nthr = blockDim.x * blockDim.y;
    for (int v = threadIdx.y * blockDim.x + threadIdx.x; v < n_views; v += nthr)
        sv3[v] = make_float2(views[v].cs, views[v].sn);
    __syncthreads();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    const int z0 = blockIdx.z * kZChunk;
    if (c >= nx || r >= ny) return;
    const float tc = (float)c - 0.5f * (float)(nx - 1);
    const float tr = (float)r - 0.5f * (float)(ny - 1);
    const float tz0 = (float)z0 - 0.5f * (float)(nz - 1);
    const float gu = 0.5f * (float)(ndu - 1) + 2.f;      // +2: padded row offset
    const float gv = 0.5f * (float)(ndv - 1) + 1.f;      // +1: zero row above row 0
    const float uhi = (float)(ndu + 2), vhi = (float)(ndv + 1);
    float acc[kZChunk];
#pragma unroll
    for (int j = 0; j < kZChunk; ++j) acc[j] = 0.f;
    const float2 *vw = ypad;
    for (int v = 0; v < n_views; ++v, vw += view_ld) {
        const float2 V = sv3[v];
        const float pe = fmaf(tr, V.x, -tc * V.y);
        const float bb = fmaf(-tc, V.x, fmaf(-tr, V.y, sid_h));
        const float rho = __fdividef(1.f, bb);
        const float a = pe * rho;
        float fu = fminf(fmaxf(fmaf(a, ku, gu), 0.f), uhi);
        const float ful = floorf(fu);
        const float wu = fu - ful;
        const float2 *col = vw + (int)ful;
        const float s2 = fmaf(a, a, 1.f);
        const float rho2 = rho * rho;
#pragma unroll
        for (int j = 0; j < kZChunk; ++j) {
            const float b = (tz0 + (float)j) * rho;
            float fv = fminf(fmaxf(fmaf(b, kv, gv), 0.f), vhi);
            const float fvl = floorf(fv);
            const float wv = fv - fvl;
            const float2 *p = col + (int64_t)(int)fvl * ld;
            const float2 t0 = __ldg(p), t1 = __ldg(p + ld);     // bin u and its slope, two rows
            const float r0 = fmaf(wu, t0.y, t0.x);
            const float r1 = fmaf(wu, t1.y, t1.x);
            const float q = fmaf(b, b, s2);
            acc[j] = fmaf(rho2 * (q * rsqrtf(q)), fmaf(wv, r1 - r0, r0), acc[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < kZChunk; ++j)
        if (z0 + j < nz) x[((int64_t)(z0 + j) * ny + r) * nx + c] = acc[j] * kw;
}

cudaError_t launch_voxbp3d(const ct_geom *g, const float2 *ypad, float *x, const int *stop,
                           cudaStream_t s)
{
    const DeviceGeom &d = g->dg;
    dim3 block(32, 4), grid((d.nx + 31) / 32, (d.ny + 3) / 4, (d.nz + kZChunk - 1) / kZChunk);
    const double h = g->desc.pixel;
    const float sid_h = (float)(g->desc.sid / h);
    const float ku = (float)(g->desc.sdd / g->desc.pitch_u);
    const float kv = (float)(g->desc.sdd / g->desc.pitch_v);
    const float kw = (float)(g->desc.sdd * g->desc.sdd * h / (g->desc.pitch_u * g->desc.pitch_v));
    voxbp3d_kernel<<<grid, block, sizeof(float2) * (size_t)d.n_views, s>>>(
        d.views, d.n_views, ypad, d.sino_view_ld, d.sino_ld, d.ndu, d.ndv, d.nx, d.ny, d.nz,
        sid_h, ku, kv, kw, x, stop);
    return cudaGetLastError();
}

}  // namespace ct
