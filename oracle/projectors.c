/*
 * FP64 CPU oracle for the CT projector pair of hybrid AB-/BA-GMRES (arXiv 2602.17892).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the GPU path is
 * checked against.  It shares no code, header or table with the CUDA library; only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * What it computes (Sec. 1, Eq. (1): b = A x with A in R^{m x n}; Sec. 2: B in R^{n x m}
 * is a backprojector that is NOT the transpose of A):
 *   og_forward       y = A x : ray-driven Joseph line integrals (every driving line is
 *                     sampled, linear interpolation between the two neighbouring pixel
 *                     centres, zero outside the image, weight h / |d_drive|);
 *   og_back_pixel    x = B y : pixel-driven backprojector, linear interpolation on the
 *                     detector at the point where the ray through the pixel centre lands;
 *   og_back_adjoint  x = A^T y : the exact transpose of og_forward (the matched case).
 *
 * Geometry conventions (pixel centres, angle origin, bin order) are the ones documented in
 * the seeded input module: pixel (r, c) has centre X = (c-(nx-1)/2) h, Y = (r-(ny-1)/2) h.
 *   parallel: ray (theta, s) is the line { p : p . (cos, sin) = s }, s_j = (j-(nd-1)/2) pitch;
 *   fan-flat: source S = SID (cos, sin), detector centre -(SDD-SID)(cos, sin), detector axis
 *             e_u = (-sin, cos), bin j at u_j = (j-(nd-1)/2) pitch;
 *   cone:     as fan-flat in the x-y plane, detector rows along +z at v_i = (i-(nv-1)/2) pv.
 * Joseph drives along x when |d_x| >= |d_y| (ties go to x); in 3D along the largest |d|
 * component (ties x, then y).
 *
 * Backprojector weights (chosen so that B has the scale of A^T):
 *   parallel: h^2 / pitch * tri((s_p - s_j)/pitch),  s_p = p . (cos, sin);
 *   fan:      h^2 (SDD^2 + u^2) / (L pitch SDD) * tri((u_p - u_j)/pitch),
 *             u_p = SDD (p . e_u) / (SID - p . (cos, sin)),  L = |p - S|;
 *   cone:     h^3 (SDD^2+u^2+v^2)^{3/2} / (L^2 pu pv SDD) * bilinear,  with
 *             v_p = SDD z / (SID - p . (cos, sin)).
 */
#include <math.h>
#include <stddef.h>
#include <string.h>

typedef struct {
    int kind;            /* 0 parallel 2D, 1 fan-flat 2D, 2 cone 3D */
    int nx, ny, nz;
    double h;
    int n_views;
    const double *angles;
    int n_det_u, n_det_v;
    double pitch_u, pitch_v;
    double sid, sdd;
} og_geom;

/* value of pixel (r, c) or 0 outside */
static double pix2(const og_geom *g, const double *x, long r, long c)
{
    if (r < 0 || r >= g->ny || c < 0 || c >= g->nx) return 0.0;
    return x[r * (long)g->nx + c];
}

static double vox3(const og_geom *g, const double *x, long k, long r, long c)
{
    if (k < 0 || k >= g->nz || r < 0 || r >= g->ny || c < 0 || c >= g->nx) return 0.0;
    return x[(k * (long)g->ny + r) * (long)g->nx + c];
}

/* The ray of measurement (view, bin u, row v) as a point p0 on it and a unit direction d. */
static void og_ray(const og_geom *g, int view, int iu, int iv, double p0[3], double d[3])
{
    double th = g->angles[view];
    double ct = cos(th), st = sin(th);
    double u = (iu - (g->n_det_u - 1) / 2.0) * g->pitch_u;
    if (g->kind == 0) {
        p0[0] = u * ct; p0[1] = u * st; p0[2] = 0.0;
        d[0] = -st; d[1] = ct; d[2] = 0.0;
        return;
    }
    double v = (g->kind == 2) ? (iv - (g->n_det_v - 1) / 2.0) * g->pitch_v : 0.0;
    double S[3] = { g->sid * ct, g->sid * st, 0.0 };
    double off = g->sdd - g->sid;
    double P[3] = { -off * ct - u * st, -off * st + u * ct, v };
    double D[3] = { P[0] - S[0], P[1] - S[1], P[2] - S[2] };
    double L = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    p0[0] = S[0]; p0[1] = S[1]; p0[2] = S[2];
    d[0] = D[0] / L; d[1] = D[1] / L; d[2] = D[2] / L;
}

/* Joseph line integral of one ray (2D).  When transpose_y is non-NULL the routine instead
 * scatters transpose_y * weight into x (the exact adjoint of the gather). */
static double joseph2d(const og_geom *g, const double *x, const double p0[3], const double d[3],
                       double *xt, double yval)
{
    double h = g->h, sum = 0.0;
    if (fabs(d[0]) >= fabs(d[1])) {
        double w = h / fabs(d[0]);
        for (long c = 0; c < g->nx; ++c) {
            double X = (c - (g->nx - 1) / 2.0) * h;
            double t = (X - p0[0]) / d[0];
            double Y = p0[1] + t * d[1];
            double r = Y / h + (g->ny - 1) / 2.0;
            double r0 = floor(r), f = r - r0;
            long i0 = (long)r0;
            if (xt) {
                if (i0 >= 0 && i0 < g->ny) xt[i0 * g->nx + c] += w * (1.0 - f) * yval;
                if (i0 + 1 >= 0 && i0 + 1 < g->ny) xt[(i0 + 1) * g->nx + c] += w * f * yval;
            } else {
                sum += (1.0 - f) * pix2(g, x, i0, c) + f * pix2(g, x, i0 + 1, c);
            }
        }
        return sum * w;
    } else {
        double w = h / fabs(d[1]);
        for (long r = 0; r < g->ny; ++r) {
            double Y = (r - (g->ny - 1) / 2.0) * h;
            double t = (Y - p0[1]) / d[1];
            double X = p0[0] + t * d[0];
            double c = X / h + (g->nx - 1) / 2.0;
            double c0 = floor(c), f = c - c0;
            long j0 = (long)c0;
            if (xt) {
                if (j0 >= 0 && j0 < g->nx) xt[r * g->nx + j0] += w * (1.0 - f) * yval;
                if (j0 + 1 >= 0 && j0 + 1 < g->nx) xt[r * g->nx + j0 + 1] += w * f * yval;
            } else {
                sum += (1.0 - f) * pix2(g, x, r, j0) + f * pix2(g, x, r, j0 + 1);
            }
        }
        return sum * w;
    }
}

/* Joseph line integral of one ray (3D): sample every plane of the driving axis, bilinear
 * interpolation in the plane, weight h / |d_drive|. */
static double joseph3d(const og_geom *g, const double *x, const double p0[3], const double d[3],
                       double *xt, double yval)
{
    double h = g->h;
    int n[3] = { g->nx, g->ny, g->nz };
    double ad[3] = { fabs(d[0]), fabs(d[1]), fabs(d[2]) };
    int a = 0;                                   /* driving axis */
    if (ad[1] > ad[a]) a = 1;
    if (ad[2] > ad[a]) a = 2;
    int b = (a + 1) % 3, e = (a + 2) % 3;        /* the two in-plane axes */
    double w = h / ad[a], sum = 0.0;
    for (long i = 0; i < n[a]; ++i) {
        double A = (i - (n[a] - 1) / 2.0) * h;
        double t = (A - p0[a]) / d[a];
        double pb = (p0[b] + t * d[b]) / h + (n[b] - 1) / 2.0;
        double pe = (p0[e] + t * d[e]) / h + (n[e] - 1) / 2.0;
        double b0 = floor(pb), e0 = floor(pe);
        double fb = pb - b0, fe = pe - e0;
        for (int db = 0; db < 2; ++db)
            for (int de = 0; de < 2; ++de) {
                double wt = (db ? fb : 1.0 - fb) * (de ? fe : 1.0 - fe);
                long idx[3];
                idx[a] = i; idx[b] = (long)b0 + db; idx[e] = (long)e0 + de;
                if (xt) {
                    if (idx[0] >= 0 && idx[0] < g->nx && idx[1] >= 0 && idx[1] < g->ny &&
                        idx[2] >= 0 && idx[2] < g->nz)
                        xt[(idx[2] * g->ny + idx[1]) * (long)g->nx + idx[0]] += w * wt * yval;
                } else {
                    sum += wt * vox3(g, x, idx[2], idx[1], idx[0]);
                }
            }
    }
    return sum * w;
}

/* One measurement of y = A x. */
double og_forward_ray(const og_geom *g, const double *x, int view, int iu, int iv)
{
    double p0[3], d[3];
    og_ray(g, view, iu, iv, p0, d);
    return g->kind == 2 ? joseph3d(g, x, p0, d, NULL, 0.0) : joseph2d(g, x, p0, d, NULL, 0.0);
}

/* y = A x, y indexed [view][v][u]. */
void og_forward(const og_geom *g, const double *x, double *y)
{
    long nvw = g->n_views, nu = g->n_det_u, nv = (g->kind == 2) ? g->n_det_v : 1;
    long total = nvw * nv * nu;
#pragma omp parallel for schedule(dynamic, 64)
    for (long idx = 0; idx < total; ++idx) {
        int view = (int)(idx / (nv * nu));
        int iv = (int)((idx / nu) % nv);
        int iu = (int)(idx % nu);
        y[idx] = og_forward_ray(g, x, view, iu, iv);
    }
}

/* x = A^T y, the exact transpose of og_forward (serial scatter). */
void og_back_adjoint(const og_geom *g, const double *y, double *x)
{
    long nvw = g->n_views, nu = g->n_det_u, nv = (g->kind == 2) ? g->n_det_v : 1;
    memset(x, 0, sizeof(double) * (size_t)g->nx * g->ny * (g->kind == 2 ? g->nz : 1));
    for (long idx = 0; idx < nvw * nv * nu; ++idx) {
        int view = (int)(idx / (nv * nu));
        int iv = (int)((idx / nu) % nv);
        int iu = (int)(idx % nu);
        double p0[3], d[3];
        og_ray(g, view, iu, iv, p0, d);
        if (g->kind == 2) joseph3d(g, NULL, p0, d, x, y[idx]);
        else joseph2d(g, NULL, p0, d, x, y[idx]);
    }
}

/* linear interpolation of detector row `row` (length n) at fractional bin index f */
static double lerp_row(const double *row, long n, double fj)
{
    double j0 = floor(fj), f = fj - j0;
    long j = (long)j0;
    double v = 0.0;
    if (j >= 0 && j < n) v += (1.0 - f) * row[j];
    if (j + 1 >= 0 && j + 1 < n) v += f * row[j + 1];
    return v;
}

/* One pixel (or voxel) of x = B y. */
double og_back_pixel_one(const og_geom *g, const double *y, long k, long r, long c)
{
    double h = g->h;
    double X = (c - (g->nx - 1) / 2.0) * h;
    double Y = (r - (g->ny - 1) / 2.0) * h;
    double Z = (g->kind == 2) ? (k - (g->nz - 1) / 2.0) * h : 0.0;
    long nu = g->n_det_u, nv = g->n_det_v;
    double acc = 0.0;
    for (int view = 0; view < g->n_views; ++view) {
        double th = g->angles[view];
        double ct = cos(th), st = sin(th);
        if (g->kind == 0) {
            double s = X * ct + Y * st;
            double fj = s / g->pitch_u + (nu - 1) / 2.0;
            acc += h * h / g->pitch_u * lerp_row(y + (long)view * nu, nu, fj);
        } else if (g->kind == 1) {
            double pe = -X * st + Y * ct;                    /* p . e_u */
            double pr = X * ct + Y * st;                     /* p . (cos, sin) */
            double u = g->sdd * pe / (g->sid - pr);
            double Sx = g->sid * ct, Sy = g->sid * st;
            double L = sqrt((X - Sx) * (X - Sx) + (Y - Sy) * (Y - Sy));
            double w = h * h * (g->sdd * g->sdd + u * u) / (L * g->pitch_u * g->sdd);
            double fj = u / g->pitch_u + (nu - 1) / 2.0;
            acc += w * lerp_row(y + (long)view * nu, nu, fj);
        } else {
            double pe = -X * st + Y * ct;
            double pr = X * ct + Y * st;
            double mag = g->sdd / (g->sid - pr);
            double u = pe * mag, v = Z * mag;
            double Sx = g->sid * ct, Sy = g->sid * st;
            double L2 = (X - Sx) * (X - Sx) + (Y - Sy) * (Y - Sy) + Z * Z;
            double q = g->sdd * g->sdd + u * u + v * v;
            double w = h * h * h * q * sqrt(q) / (L2 * g->pitch_u * g->pitch_v * g->sdd);
            double fu = u / g->pitch_u + (nu - 1) / 2.0;
            double fv = v / g->pitch_v + (nv - 1) / 2.0;
            double v0 = floor(fv), f = fv - v0;
            long iv = (long)v0;
            const double *base = y + (long)view * nv * nu;
            double val = 0.0;
            if (iv >= 0 && iv < nv) val += (1.0 - f) * lerp_row(base + iv * nu, nu, fu);
            if (iv + 1 >= 0 && iv + 1 < nv) val += f * lerp_row(base + (iv + 1) * nu, nu, fu);
            acc += w * val;
        }
    }
    return acc;
}

/* x = B y (pixel/voxel-driven, unmatched). */
void og_back_pixel(const og_geom *g, const double *y, double *x)
{
    long nz = (g->kind == 2) ? g->nz : 1;
    long total = nz * (long)g->ny * g->nx;
#pragma omp parallel for schedule(dynamic, 64)
    for (long idx = 0; idx < total; ++idx) {
        long k = idx / ((long)g->ny * g->nx);
        long r = (idx / g->nx) % g->ny;
        long c = idx % g->nx;
        x[idx] = og_back_pixel_one(g, y, k, r, c);
    }
}

int og_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
