// C ABI of libctabba: geometry objects, projector entry points and the hybrid AB-/BA-GMRES
// drivers (Algorithms 1 and 2 of arXiv 2602.17892).  Every numerical step is a kernel of this
// library; the host only validates arguments, builds FP64 geometry tables once per geometry
// and enqueues launches.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "ct_internal.h"

namespace ct {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

ct_status cuda_fail(cudaError_t e, const char *what)
{
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return CT_ECUDA;
}

static ct_status einval(const std::string &msg)
{
    set_error(msg);
    return CT_EINVAL;
}

static int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// declared in arnoldi.cu
cudaError_t arnoldi_step_dev(float *W, int64_t L, int64_t ld, int k, float *q, double *hcol,
                             const ArnoldiScratch &sc, double *aux, int *stop, int step,
                             bool reorth, cudaStream_t s);
cudaError_t normalize_first(const float *r, int64_t L, float *w0, const ArnoldiScratch &sc,
                            double *aux, int *stop, cudaStream_t s);
cudaError_t launch_combine(const float *W, int64_t L, int64_t ld, const double *Y, int K,
                           int ystride, const int *stop, int kfixed, const float *x0, float *x,
                           int max_blocks, cudaStream_t s);
cudaError_t launch_rsub(const float *b, float *r, int64_t L, int max_blocks, cudaStream_t s);
// q_padded: q holds ld floats with a zero tail beyond L (the solver's own vectors), which
// allows the tiled path when ld is a multiple of 128; next = false (a solve's last step): the
// tiled path records h_{k+1,k} without writing w_{k+1}, which no later step reads
cudaError_t arnoldi_step_basis(int basis, void *W, int64_t L, int64_t ld, int k, float *q,
                               double *hcol, const ArnoldiScratch &sc, double *aux, int *stop,
                               int step, bool reorth, float *cur, bool q_padded, cudaStream_t s,
                               bool next);
int arnoldi_step_launches(int basis, int64_t ld, int k, const ArnoldiScratch &sc, bool reorth,
                          bool q_padded);
cudaError_t normalize_first_basis(int basis, const float *r, int64_t L, void *w0,
                                  const ArnoldiScratch &sc, double *aux, int *stop, float *cur,
                                  cudaStream_t s);
cudaError_t launch_combine_basis(int basis, const void *W, int64_t L, int64_t ld, const double *Y,
                                 int K, int ystride, const int *stop, int kfixed, const float *x0,
                                 float *x, int max_blocks, cudaStream_t s);

static size_t basis_bytes(int basis) { return basis == CT_BASIS_F32 ? 4 : 2; }

constexpr int kMaxBlocks = 152 * 8;

// Block cap of the Gram-Schmidt kernels for the solves enqueued on this thread (0: kMaxBlocks).
// A batch of several problems captures its solves with one block per SM: the passes stream HBM
// with one CTA per SM nearly as fast, and the other branches' projectors keep room on every SM
// (measured on the 512^2 fan AB + BA batch: 40.6 -> 39.9 ms a step, the passes alone 13.5 ->
// 15.8 ms).
static thread_local int g_gs_block_cap = 0;
static int gs_blocks() { return g_gs_block_cap > 0 ? g_gs_block_cap : kMaxBlocks; }

// ----------------------------------------------------------------------------- profiling
// Optional CUDA-event timing of launch groups, and a count of every kernel launch.
struct PhaseRec { int phase; int launches; cudaEvent_t a, b; };
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<PhaseRec> g_prof_recs;
static std::vector<cudaEvent_t> g_prof_pool;
static std::atomic<int64_t> g_launches{0};

static cudaEvent_t prof_event()
{
    if (!g_prof_pool.empty()) {
        cudaEvent_t e = g_prof_pool.back();
        g_prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct PhaseScope {
    int phase, launches;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    PhaseScope(int ph, int n, cudaStream_t st) : phase(ph), launches(n), s(st)
    {
        g_launches += n;
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (g_prof_on) {
            a = prof_event();
            if (a) cudaEventRecord(a, s);
        }
    }
    ~PhaseScope()
    {
        if (!a) return;
        std::lock_guard<std::mutex> lk(g_prof_mu);
        cudaEvent_t b = prof_event();
        if (b) {
            cudaEventRecord(b, s);
            g_prof_recs.push_back({phase, launches, a, b});
        }
    }
};
#define CT_CAT2(a, b) a##b
#define CT_CAT(a, b) CT_CAT2(a, b)
#define CT_PHASE(ph, n, s) ::ct::PhaseScope CT_CAT(ct_phase_scope_, __LINE__)((ph), (n), (s))

}  // namespace ct

using namespace ct;

// ============================================================================ workspace
struct Workspace {
    int method = -1, K = 0, basis = 0;
    int *path = nullptr;    // per step: 1 = parallel small-solve path accepted
    int64_t L = 0;          // basis row length in entries (multiple of 4, zero tail)
    int64_t ld = 0;         // basis row stride: L rounded up to 128 entries (zero beyond L)
    void *W = nullptr;      // (K+1) rows of ld entries in the basis storage type
    float *cur = nullptr;   // 16-bit bases: the newest row in FP32 (operator input), ld
    float *q = nullptr;     // ld (zero beyond L)
    float *img = nullptr;   // image scratch, img_ld floats
    float *sino = nullptr;  // padded sinogram scratch
    float *sino2 = nullptr; // second padded sinogram (BA with an initial guess; on first use)
    float *vec = nullptr;   // L (initial residual)
    double *H = nullptr, *Y = nullptr, *lam = nullptr, *res = nullptr, *aux = nullptr;
    double *partial = nullptr;
    unsigned *counter = nullptr;
    int *stop = nullptr;
    // NCP stopping rule (allocated on first use): DFT twiddles of one detector row, per-view
    // partial NCP sums, the distance of every checked step
    float2 *ncp_tw = nullptr;
    float *ncp_part = nullptr;
    double *ncp = nullptr;
};

static void ws_free(Workspace *w)
{
    if (!w) return;
    cudaFree(w->W); cudaFree(w->cur); cudaFree(w->q); cudaFree(w->img); cudaFree(w->sino); cudaFree(w->vec);
    cudaFree(w->sino2);
    cudaFree(w->H); cudaFree(w->Y); cudaFree(w->lam); cudaFree(w->res); cudaFree(w->aux);
    cudaFree(w->partial); cudaFree(w->counter); cudaFree(w->stop); cudaFree(w->path);
    cudaFree(w->ncp_tw); cudaFree(w->ncp_part); cudaFree(w->ncp);
    delete w;
}

struct GeomExtra {
    Workspace *ws[2] = {nullptr, nullptr};
};

template <class T>
static cudaError_t dalloc(T **p, size_t count)
{
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
    if (e == cudaSuccess) e = cudaMemset(*p, 0, sizeof(T) * (count ? count : 1));
    return e;
}

// kernel launches of one forward projection (3D: one per z slab)
static int fwd_launches(const ct_geom *g)
{
    return g->dg.kind == CT_CONE3D ? joseph3d_launches(g) : 1;
}

static ct_status ws_get(ct_geom *g, int method, int K, int basis, Workspace **out)
{
    GeomExtra *ex = reinterpret_cast<GeomExtra *>(g->ws);
    Workspace *w = ex->ws[method];
    const int64_t img_ld = round_up(g->n, 4);
    const int64_t sino_len = (int64_t)g->dg.n_views * g->dg.sino_view_ld;
    const int64_t L = (method == 0) ? sino_len : img_ld;
    if (w && w->K >= K && w->basis == basis && w->L == L) { *out = w; return CT_OK; }
    ws_free(w);
    ex->ws[method] = nullptr;
    w = new Workspace();
    w->method = method; w->K = K; w->basis = basis; w->L = L;
    w->ld = round_up(L, 128);
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dalloc((char **)&w->W, (size_t)(K + 1) * w->ld * basis_bytes(basis));
    if (e == cudaSuccess && basis != CT_BASIS_F32) e = dalloc(&w->cur, (size_t)w->ld);
    if (e == cudaSuccess) e = dalloc(&w->q, (size_t)w->ld);
    if (e == cudaSuccess) e = dalloc(&w->vec, (size_t)L);
    if (e == cudaSuccess) e = dalloc(&w->img, (size_t)img_ld);
    if (e == cudaSuccess) e = dalloc(&w->sino, (size_t)sino_len);
    if (e == cudaSuccess) e = dalloc(&w->H, (size_t)(K + 1) * K);
    if (e == cudaSuccess) e = dalloc(&w->Y, (size_t)K * K);
    if (e == cudaSuccess) e = dalloc(&w->lam, (size_t)K);
    if (e == cudaSuccess) e = dalloc(&w->res, (size_t)K);
    if (e == cudaSuccess) e = dalloc(&w->aux, (size_t)(8 + 2 * (K + 2)));
    if (e == cudaSuccess) e = dalloc(&w->partial, (size_t)kMaxBlocks * (K + 2));
    if (e == cudaSuccess) e = dalloc(&w->counter, 4);
    if (e == cudaSuccess) e = dalloc(&w->stop, 4);
    if (e == cudaSuccess) e = dalloc(&w->path, (size_t)K);
    if (e != cudaSuccess) {
        ws_free(w);
        set_error(std::string("workspace allocation: ") + cudaGetErrorString(e));
        return CT_ENOMEM;
    }
    ex->ws[method] = w;
    *out = w;
    return CT_OK;
}

// The NCP rule's tables (host set-up, before any capture): twiddles cos, sin(2 pi t / n) of
// one detector row in FP64 rounded to FP32, the per-view partial sums, the distances.
static ct_status ncp_ready(ct_geom *g, Workspace *w)
{
    const int n = g->dg.ndu, q = n / 2;
    if (n < 2 || n > kNcpMaxBins)
        return einval("solver: the NCP rule needs 2 <= n_det_u <= " + std::to_string(kNcpMaxBins));
    if (w->ncp_tw) return CT_OK;
    std::vector<float2> tw((size_t)n);
    for (int t = 0; t < n; ++t) {
        const double a = 2.0 * M_PI * (double)t / (double)n;
        tw[(size_t)t] = make_float2((float)cos(a), (float)sin(a));
    }
    cudaError_t e = dalloc(&w->ncp_tw, (size_t)n);
    if (e == cudaSuccess) e = dalloc(&w->ncp_part, (size_t)g->dg.n_views * (q + 1));
    if (e == cudaSuccess) e = dalloc(&w->ncp, (size_t)w->K);
    if (e == cudaSuccess)
        e = cudaMemcpy(w->ncp_tw, tw.data(), sizeof(float2) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = ncp_prepare(n);
    if (e != cudaSuccess) {
        cudaFree(w->ncp_tw); cudaFree(w->ncp_part); cudaFree(w->ncp);
        w->ncp_tw = nullptr; w->ncp_part = nullptr; w->ncp = nullptr;
        set_error(std::string("NCP tables: ") + cudaGetErrorString(e));
        return CT_ENOMEM;
    }
    return CT_OK;
}

// ============================================================================ geometry
static void ray_setup(const ct_geom_desc *d, int view, int bin, double p0[2], double dir[2])
{
    double th = d->angles[view];
    double ct_ = cos(th), st = sin(th);
    double u = (bin - (d->n_det_u - 1) / 2.0) * d->pitch_u;
    if (d->kind == CT_PARALLEL2D) {
        p0[0] = u * ct_; p0[1] = u * st;
        dir[0] = -st; dir[1] = ct_;
    } else {
        double S[2] = {d->sid * ct_, d->sid * st};
        double off = d->sdd - d->sid;
        double P[2] = {-off * ct_ - u * st, -off * st + u * ct_};
        double D[2] = {P[0] - S[0], P[1] - S[1]};
        double L = sqrt(D[0] * D[0] + D[1] * D[1]);
        p0[0] = S[0]; p0[1] = S[1];
        dir[0] = D[0] / L; dir[1] = D[1] / L;
    }
}

// The ray's table entry (FP64 geometry, stored as described at Ray2D) and its number of samples
// (the driving lines whose tap index lies in [-1, n_other), for the projector's work count).
static Ray2D make_ray(const ct_geom_desc *d, int view, int bin, int64_t *samples)
{
    double p0[2], dir[2];
    ray_setup(d, view, bin, p0, dir);
    const double h = d->pixel;
    int axis, n_drive, n_other;
    double a_drive, a_other, p_drive, p_other;
    if (fabs(dir[0]) >= fabs(dir[1])) {        // drive along x
        axis = 0; n_drive = d->nx; n_other = d->ny;
        a_drive = dir[0]; a_other = dir[1]; p_drive = p0[0]; p_other = p0[1];
    } else {
        axis = 1; n_drive = d->ny; n_other = d->nx;
        a_drive = dir[1]; a_other = dir[0]; p_drive = p0[1]; p_other = p0[0];
    }
    // point of the ray on the central driving line (coordinate 0 along the driving axis)
    double t0 = -p_drive / a_drive;
    double other0 = p_other + t0 * a_other;
    double pmid = other0 / h + (n_other - 1) / 2.0;
    double slope = a_other / a_drive;
    double tmid = (n_drive - 1) / 2.0;
    int lo = 0, hi = n_drive - 1;
    if (fabs(slope) < 1e-300) {
        if (!(pmid >= -1.0 && pmid < n_other)) { lo = 1; hi = 0; }
    } else {
        double ta = tmid + (-1.0 - pmid) / slope, tb = tmid + (n_other - pmid) / slope;
        double tl = std::min(ta, tb), th = std::max(ta, tb);
        double clo = ceil(tl - 1e-6), chi = floor(th + 1e-6);
        if (clo > lo) lo = (clo > hi + 1) ? hi + 1 : (int)clo;
        if (chi < hi) hi = (chi < lo - 1) ? lo - 1 : (int)chi;
        if (hi < lo) { lo = 1; hi = 0; }
    }
    *samples = hi >= lo ? hi - lo + 1 : 0;
    Ray2D r;
    r.pmid = (float)pmid;
    const double q = std::max(-1.0, std::min(1.0, slope)) * 536870912.0;   // 2^29
    r.enc = (int32_t)(llround(q) * 2 + axis);
    return r;
}

// Whether every pixel centre projects inside the detector in every view (2D), with half a bin
// of margin in the padded row: the bin position is an affine (parallel) or projective (fan)
// function of the pixel position, so its extremes over the image are at the corner pixels.
static bool pixels_inside_detector(const ct_geom_desc *d)
{
    const double cx = 0.5 * (d->nx - 1), cy = 0.5 * (d->ny - 1);
    const double gam = 0.5 * (d->n_det_u - 1) + 2.0, hi = d->n_det_u + 1.5;
    for (int v = 0; v < d->n_views; ++v) {
        const double c = cos(d->angles[v]), sn = sin(d->angles[v]);
        for (double sx : {-cx, cx})
            for (double sy : {-cy, cy}) {
                double fj;
                if (d->kind == CT_PARALLEL2D) {
                    fj = d->pixel * (c * sx + sn * sy) / d->pitch_u + gam;
                } else {
                    const double pe = sy * c - sx * sn;
                    const double bb = d->sid / d->pixel - sx * c - sy * sn;
                    fj = d->sdd / d->pitch_u * pe / bb + gam;
                }
                if (!(fj >= 0.5 && fj <= hi)) return false;
            }
    }
    return true;
}

// Views in quadruples a quarter turn apart on a square image of even side (fan-flat): view
// k + m n/4 at angle theta_k + m pi/2 for m = 1, 2, 3 (cos and sin within 1e-9), at most 16384
// views.  Then a quarter turn of the image maps pixels onto pixels and each view onto another
// view of the scan, which the four-fold backprojector uses.
static bool rot4_symmetric(const ct_geom_desc *d)
{
    if (d->kind != CT_FANFLAT2D || d->nx != d->ny || (d->nx & 1) || d->n_views % 4 != 0 ||
        d->n_views > 16384)
        return false;
    const int q = d->n_views / 4;
    for (int k = 0; k < q; ++k) {
        const double c0 = cos(d->angles[k]), s0 = sin(d->angles[k]);
        const double ec[3] = {-s0, -c0, s0}, es[3] = {c0, -s0, -c0};   // rotated by m pi/2
        for (int m = 1; m < 4; ++m) {
            const double a = d->angles[k + m * q];
            if (!(fabs(cos(a) - ec[m - 1]) <= 1e-9 && fabs(sin(a) - es[m - 1]) <= 1e-9))
                return false;
        }
    }
    return true;
}

// In-plane (fan) part of the rays of column iu of a cone view: every ray of the column has the
// x-y projection of the fan ray through detector column iu, D = P - S unnormalised.
static RayXY make_ray_xy(const ct_geom_desc *d, int view, int iu)
{
    const double th = d->angles[view];
    const double c = cos(th), sn = sin(th);
    const double u = (iu - (d->n_det_u - 1) / 2.0) * d->pitch_u;
    const double Sx = d->sid * c, Sy = d->sid * sn;
    const double off = d->sdd - d->sid;
    const double Dx = (-off * c - u * sn) - Sx, Dy = (-off * sn + u * c) - Sy;
    const double h = d->pixel;
    const int axis = fabs(Dx) >= fabs(Dy) ? 0 : 1;
    const double Da = axis == 0 ? Dx : Dy, Do = axis == 0 ? Dy : Dx;
    const double Sa = axis == 0 ? Sx : Sy, So = axis == 0 ? Sy : Sx;
    const int n_drive = axis == 0 ? d->nx : d->ny, n_other = axis == 0 ? d->ny : d->nx;
    const double slope = Do / Da;
    const double bmid = (So - Sa * slope) / h + (n_other - 1) / 2.0;
    const double tmid = (n_drive - 1) / 2.0;
    int lo = 0, hi = n_drive - 1;
    if (fabs(slope) < 1e-300) {
        if (!(bmid >= -1.0 && bmid < n_other)) { lo = 1; hi = 0; }
    } else {
        double ta = tmid + (-1.0 - bmid) / slope, tb = tmid + (n_other - bmid) / slope;
        double tl = std::min(ta, tb), tu = std::max(ta, tb);
        double clo = ceil(tl - 1e-6), chi = floor(tu + 1e-6);
        if (clo > lo) lo = (clo > hi + 1) ? hi + 1 : (int)clo;
        if (chi < hi) hi = (chi < lo - 1) ? lo - 1 : (int)chi;
        if (hi < lo) { lo = 1; hi = 0; }
    }
    RayXY r;
    r.bmid = (float)bmid;
    r.bslope = (float)slope;
    r.dxy2 = (float)((Dx * Dx + Dy * Dy) / (Da * Da));
    r.packed = (uint32_t)lo | ((uint32_t)hi << 15) | ((uint32_t)axis << 30);
    r.rda = 1.0 / Da;
    r.sa_h = Sa / h;
    // z part for the kernels' FP32 set-up (pairs hi + lo of the FP64 factors) and the rows the
    // kernels drive along x or y: |v| |rda| <= 1 in the same FP64 expression as before, an
    // interval of rows around the detector's centre row (|v| grows away from it)
    const double P = d->pitch_v * r.rda, Q = r.sa_h * P;
    r.zp_hi = (float)P;
    r.zp_lo = (float)(P - (double)r.zp_hi);
    r.zq_hi = (float)Q;
    r.zq_lo = (float)(Q - (double)r.zq_hi);
    const int ndv = d->n_det_v;
    auto xy_driven = [&](int iv) {
        const double v = (iv - 0.5 * (ndv - 1)) * d->pitch_v;
        return !(fabs(v) * fabs(r.rda) > 1.0);
    };
    const int cen = (ndv - 1) / 2;
    int lo_iv = cen, hi_iv = cen;
    if (!xy_driven(cen)) {
        lo_iv = 1; hi_iv = 0;                      // no row (a pitch this coarse cannot happen)
    } else {
        int a = 0, b = cen;                        // smallest row of the interval
        while (a < b) { const int m = (a + b) / 2; if (xy_driven(m)) b = m; else a = m + 1; }
        lo_iv = a;
        a = cen; b = ndv - 1;                      // largest row of the interval
        while (a < b) { const int m = (a + b + 1) / 2; if (xy_driven(m)) a = m; else b = m - 1; }
        hi_iv = a;
    }
    r.iv_lo = lo_iv;
    r.iv_hi = hi_iv;
    r.pad0 = r.pad1 = 0;
    r.sx_h = Sx / h;
    r.sy_h = Sy / h;
    r.dx = Dx;
    r.dy = Dy;
    return r;
}

extern "C" {

const char *ct_last_error(void) { return g_last_error.c_str(); }

const char *ct_status_string(ct_status s)
{
    switch (s) {
    case CT_OK: return "CT_OK";
    case CT_EINVAL: return "CT_EINVAL";
    case CT_ENOMEM: return "CT_ENOMEM";
    case CT_ECUDA: return "CT_ECUDA";
    case CT_BREAKDOWN: return "CT_BREAKDOWN";
    case CT_ETIMEOUT: return "CT_ETIMEOUT";
    case CT_ENONFINITE: return "CT_ENONFINITE";
    }
    return "CT_UNKNOWN";
}

ct_status ct_geom_create(const ct_geom_desc *d, ct_geom **out)
{
    if (!d || !out) return einval("ct_geom_create: null argument");
    *out = nullptr;
    if (d->kind != CT_PARALLEL2D && d->kind != CT_FANFLAT2D && d->kind != CT_CONE3D)
        return einval("ct_geom_create: unsupported geometry kind");
    const bool cone = d->kind == CT_CONE3D;
    if (d->nx < 1 || d->ny < 1 || d->nx > 16384 || d->ny > 16384)
        return einval("ct_geom_create: image size out of range [1, 16384]");
    if (d->n_views < 1 || d->n_views > 65535 || d->n_det_u < 1 || d->n_det_u > (1 << 20))
        return einval("ct_geom_create: need 1 <= n_views <= 65535 and 1 <= n_det_u <= 2^20");
    if (!d->angles) return einval("ct_geom_create: angles is NULL");
    if (!(d->pixel > 0) || !(d->pitch_u > 0)) return einval("ct_geom_create: pixel and pitch must be > 0");
    for (int v = 0; v < d->n_views; ++v)
        if (!isfinite(d->angles[v])) return einval("ct_geom_create: non-finite angle");
    if (d->kind != CT_PARALLEL2D) {
        double half_diag = 0.5 * d->pixel * sqrt((double)d->nx * d->nx + (double)d->ny * d->ny);
        if (!(d->sid > half_diag) || !(d->sdd > d->sid))
            return einval("ct_geom_create: fan/cone geometry needs SDD > SID > image half-diagonal");
    }
    if (cone) {
        if (d->nz < 1 || d->nz > 16384) return einval("ct_geom_create: nz out of range [1, 16384]");
        if (d->n_det_v < 1 || d->n_det_v > 65535)
            return einval("ct_geom_create: cone needs 1 <= n_det_v <= 65535");
        if (!(d->pitch_v > 0)) return einval("ct_geom_create: pitch_v must be > 0");
    }
    ct_geom *g = new ct_geom();
    memset(g, 0, sizeof(*g));
    g->desc = *d;
    g->angles_host = new double[d->n_views];
    memcpy(g->angles_host, d->angles, sizeof(double) * d->n_views);
    g->desc.angles = g->angles_host;
    if (!cone) {
        g->desc.nz = 1;
        g->desc.n_det_v = 1;
        g->desc.pitch_v = 1.0;
    }
    const int nz = g->desc.nz, ndv = g->desc.n_det_v;
    g->n = (int64_t)d->nx * d->ny * nz;
    g->m = (int64_t)d->n_views * ndv * d->n_det_u;
    DeviceGeom &dg = g->dg;
    dg.kind = d->kind; dg.nx = d->nx; dg.ny = d->ny; dg.nz = nz;
    dg.h = (float)d->pixel; dg.n_views = d->n_views; dg.ndu = d->n_det_u; dg.ndv = ndv;
    dg.pitch_u = (float)d->pitch_u; dg.pitch_v = (float)g->desc.pitch_v;
    dg.sid = (float)d->sid; dg.sdd = (float)d->sdd;
    // at least n + 3 pairs per line: pair 0 holds the taps (-1, 0), pairs n + 1 and n + 2 (taps
    // beyond the edge, which the 2D Joseph loop may read for positions up to n + 1) zeros
    dg.row_pairs_ld = (int)round_up(d->nx + 3, 16);
    dg.col_pairs_ld = (int)round_up(d->ny + 3, 16);
    dg.sino_ld = (int)round_up(d->n_det_u + 4, 4);
    dg.sino_view_ld = cone ? (int64_t)(ndv + 3) * dg.sino_ld : dg.sino_ld;
    dg.sino_row0 = cone ? dg.sino_ld : 0;
    // 3D: both layouts have max(nx, ny) + 3 rows per slice, so that any driving index of any
    // lane of a warp addresses a row inside either layout (lanes outside their own range still
    // load, with zero weight)
    const int nmax = std::max(d->nx, d->ny);
    dg.slice_x = cone ? (int64_t)(nmax + 3) * dg.col_pairs_ld : 0;
    dg.slice_y = cone ? (int64_t)(nmax + 3) * dg.row_pairs_ld : 0;
    dg.tune_a_threads = 256;
    dg.tune_a_views = cone ? 8 : 1;
    dg.tune_b_rows = cone ? 4 : 8;
    dg.tune_b_views = 1;
    dg.back_adjoint = 0;
    dg.b_noclamp = cone ? 0 : (pixels_inside_detector(&g->desc) ? 1 : 0);
    dg.b_rot4 = rot4_symmetric(&g->desc) ? 1 : 0;
    dg.tune_a_slab = 16;
    dg.tune_a_rays = 1;
    dg.tune_a_wviews = 1;
    dg.tune_b_wrows = 1;

    std::vector<Ray2D> rays;
    std::vector<RayXY> rays_xy;
    g->a_samples = 0;
    if (cone) {
        rays_xy.resize((size_t)d->n_views * d->n_det_u);
        for (int v = 0; v < d->n_views; ++v)
            for (int j = 0; j < d->n_det_u; ++j)
                rays_xy[(size_t)v * d->n_det_u + j] = make_ray_xy(&g->desc, v, j);
    } else {
        rays.resize((size_t)g->m);
        for (int v = 0; v < d->n_views; ++v)
            for (int j = 0; j < d->n_det_u; ++j) {
                int64_t ns = 0;
                rays[(size_t)v * d->n_det_u + j] = make_ray(&g->desc, v, j, &ns);
                g->a_samples += ns;
            }
    }
    std::vector<ViewBP> views(d->n_views);
    for (int v = 0; v < d->n_views; ++v) {
        double c = cos(d->angles[v]), s = sin(d->angles[v]);
        views[v].cs = (float)c;
        views[v].sn = (float)s;
        views[v].a = (float)(d->pixel * c / d->pitch_u);
        views[v].b = (float)(d->pixel * s / d->pitch_u);
    }
    // 2D: lines -1 .. max(nx, ny) in both layouts (the Joseph kernel's warps may walk, for a ray
    // driven along the shorter side, lines beyond that side: zero lines)
    const size_t nlines = (size_t)std::max(d->nx, d->ny) + 2;
    const size_t prow_n = cone ? (size_t)(nz + 3) * dg.slice_y : nlines * dg.row_pairs_ld;
    const size_t pcol_n = cone ? (size_t)(nz + 3) * dg.slice_x : nlines * dg.col_pairs_ld;
    cudaError_t e = cudaSuccess;
    if (cone) {
        e = dalloc(&g->rays_xy_dev, rays_xy.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(g->rays_xy_dev, rays_xy.data(), sizeof(RayXY) * rays_xy.size(), cudaMemcpyHostToDevice);
    } else {
        e = dalloc(&g->rays_dev, rays.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(g->rays_dev, rays.data(), sizeof(Ray2D) * rays.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = dalloc(&g->views_dev, views.size());
    if (e == cudaSuccess) e = cudaMemcpy(g->views_dev, views.data(), sizeof(ViewBP) * views.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = dalloc(&g->prow_dev, prow_n);
    if (e == cudaSuccess) e = dalloc(&g->pcol_dev, pcol_n);
    if (e == cudaSuccess) e = dalloc(&g->sino_pad_dev, (size_t)d->n_views * dg.sino_view_ld);
    if (e == cudaSuccess) e = dalloc(&g->sino_pairs_dev, (size_t)d->n_views * dg.sino_view_ld);
    if (e == cudaSuccess && !cone) e = dalloc(&g->adj_acc_dev, (size_t)g->n);
    if (e != cudaSuccess) {
        set_error(std::string("ct_geom_create: ") + cudaGetErrorString(e));
        ct_geom_destroy(g);
        return CT_ENOMEM;
    }
    dg.rays = g->rays_dev;
    dg.rays_xy = g->rays_xy_dev;
    dg.views = g->views_dev;
    if (cone) {
        e = count_joseph3d_samples(g, &g->a_samples);
        if (e != cudaSuccess) {
            set_error(std::string("ct_geom_create: ") + cudaGetErrorString(e));
            ct_geom_destroy(g);
            return CT_ECUDA;
        }
    }
    g->ws = reinterpret_cast<struct Workspace *>(new GeomExtra());
    *out = g;
    return CT_OK;
}

void ct_geom_destroy(ct_geom *g)
{
    if (!g) return;
    if (g->ws) {
        GeomExtra *ex = reinterpret_cast<GeomExtra *>(g->ws);
        ws_free(ex->ws[0]);
        ws_free(ex->ws[1]);
        delete ex;
    }
    cudaFree(g->rays_dev); cudaFree(g->rays_xy_dev); cudaFree(g->views_dev);
    cudaFree(g->prow_dev); cudaFree(g->pcol_dev);
    cudaFree(g->sino_pad_dev);
    cudaFree(g->sino_pairs_dev);
    cudaFree(g->adj_acc_dev);
    delete[] g->angles_host;
    delete g;
}

ct_status ct_geom_dims(const ct_geom *g, int64_t *n, int64_t *m)
{
    if (!g) return einval("ct_geom_dims: null geometry");
    if (n) *n = g->n;
    if (m) *m = g->m;
    return CT_OK;
}

ct_status ct_geom_work(const ct_geom *g, int64_t *a_samples, int64_t *b_samples)
{
    if (!g) return einval("ct_geom_work: null geometry");
    if (a_samples) *a_samples = g->a_samples;
    if (b_samples) *b_samples = g->n * (int64_t)g->desc.n_views;
    return CT_OK;
}

ct_status ct_forward_A(ct_geom *g, const float *x_dev, float *y_dev, ct_stream_t stream)
{
    if (!g || !x_dev || !y_dev) return einval("ct_forward_A: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    {
        CT_PHASE(CT_PH_LAYOUT, 1, s);
        CT_CUDA(launch_image_pairs(g, x_dev, nullptr, s));
    }
    CT_PHASE(CT_PH_FORWARD, fwd_launches(g), s);
    CT_CUDA(launch_forward_proj(g, y_dev, false, nullptr, s));
    return CT_OK;
}

// the FP64 accumulators of A^T (cone geometries allocate them on first use: n doubles)
static ct_status adjoint_scratch(ct_geom *g)
{
    if (g->adj_acc_dev) return CT_OK;
    if (dalloc(&g->adj_acc_dev, (size_t)g->n) != cudaSuccess) {
        set_error("ct_back_AT: allocating the adjoint's FP64 accumulators failed");
        return CT_ENOMEM;
    }
    return CT_OK;
}

ct_status ct_back_AT(ct_geom *g, const float *y_dev, float *x_dev, ct_stream_t stream)
{
    if (!g || !y_dev || !x_dev) return einval("ct_back_AT: null argument");
    ct_status st = adjoint_scratch(g);
    if (st != CT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const DeviceGeom &d = g->dg;
    CT_PHASE(CT_PH_BACK, 2, s);
    if (d.kind == CT_CONE3D)
        CT_CUDA(launch_adjoint3d(g, y_dev, (int64_t)d.ndv * d.ndu, d.ndu, 0, g->adj_acc_dev,
                                 x_dev, nullptr, s));
    else
        CT_CUDA(launch_adjoint2d(g, y_dev, d.ndu, 0, x_dev, nullptr, s));
    return CT_OK;
}

ct_status ct_geom_set_backprojector(ct_geom *g, ct_backprojector kind)
{
    if (!g) return einval("ct_geom_set_backprojector: null geometry");
    if (kind != CT_BACK_PIXEL && kind != CT_BACK_ADJOINT)
        return einval("ct_geom_set_backprojector: unknown backprojector");
    if (kind == CT_BACK_ADJOINT) {
        ct_status st = adjoint_scratch(g);
        if (st != CT_OK) return st;
    }
    g->dg.back_adjoint = kind == CT_BACK_ADJOINT ? 1 : 0;
    return CT_OK;
}

ct_status ct_back_B(ct_geom *g, const float *y_dev, float *x_dev, ct_stream_t stream)
{
    if (!g || !y_dev || !x_dev) return einval("ct_back_B: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    {
        CT_PHASE(CT_PH_LAYOUT, 1, s);
        CT_CUDA(launch_pad_sino(g, y_dev, g->sino_pad_dev, s));
    }
    CT_PHASE(CT_PH_BACK, 2, s);   // pair copy + B, or A^T scatter + rounding
    CT_CUDA(launch_back_proj(g, g->sino_pad_dev, x_dev, nullptr, s));
    return CT_OK;
}

void ct_hybrid_opts_default(ct_hybrid_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->max_iters = 30;
    o->rule = CT_LAMBDA_GCV;
    o->tau = 1.01;
    o->reorth = 1;
    o->basis = CT_BASIS_F32;
    o->stop_rule = CT_STOP_NONE;
    o->stop_tol = 1e-3;
    o->stop_every = 5;
}

}  // extern "C"

// ============================================================================ solvers
static ct_status check_opts(const ct_hybrid_opts *o)
{
    if (!o) return einval("solver: opts is NULL");
    if (o->max_iters < 1 || o->max_iters > kMaxSmallK)
        return einval("solver: max_iters must be in [1, " + std::to_string(kMaxSmallK) + "]");
    if (o->rule < CT_LAMBDA_NONE || o->rule > CT_LAMBDA_LCURVE) return einval("solver: bad lambda rule");
    if (o->rule == CT_LAMBDA_LEARNED && !o->lambda_net_dev)
        return einval("solver: CT_LAMBDA_LEARNED needs lambda_net_dev");
    if (o->rule == CT_LAMBDA_FIXED && !(o->lambda_fixed >= 0)) return einval("solver: lambda_fixed must be >= 0");
    if (o->rule == CT_LAMBDA_DP && (!(o->noise_norm >= 0) || !(o->tau > 0)))
        return einval("solver: DP needs noise_norm >= 0 and tau > 0");
    if (o->basis < CT_BASIS_F32 || o->basis > CT_BASIS_F16) return einval("solver: bad basis type");
    if (o->stop_rule < CT_STOP_NONE || o->stop_rule > CT_STOP_NCP) return einval("solver: bad stop rule");
    if (o->stop_rule != CT_STOP_NONE && o->stop_every < 1) return einval("solver: stop_every must be >= 1");
    if (o->stop_rule == CT_STOP_DP && (!(o->noise_norm >= 0) || !(o->tau > 0)))
        return einval("solver: the DP stop needs noise_norm >= 0 and tau > 0");
    if (o->stop_rule == CT_STOP_RNS && !(o->stop_tol > 0)) return einval("solver: stop_tol must be > 0");
    return CT_OK;
}

static ct_status read_info(Workspace *w, const ct_hybrid_opts *o, ct_hybrid_info *info);

static ct_status finish(Workspace *w, const ct_hybrid_opts *o, ct_hybrid_info *info, cudaStream_t s)
{
    CT_CUDA(cudaStreamSynchronize(s));
    return read_info(w, o, info);
}

// host copies of the solve's status, lambda and residual histories (after a synchronisation)
static ct_status read_info(Workspace *w, const ct_hybrid_opts *o, ct_hybrid_info *info)
{
    int stop[2];
    double beta;
    CT_CUDA(cudaMemcpy(stop, w->stop, sizeof(stop), cudaMemcpyDeviceToHost));
    CT_CUDA(cudaMemcpy(&beta, w->aux + 2, sizeof(double), cudaMemcpyDeviceToHost));
    const int K = o->max_iters;
    int kf = (stop[0] == 0) ? K : std::max(stop[0], 0);
    std::vector<double> lam(K), res(K);
    std::vector<int> path(K);
    CT_CUDA(cudaMemcpy(path.data(), w->path, sizeof(int) * K, cudaMemcpyDeviceToHost));
    CT_CUDA(cudaMemcpy(lam.data(), w->lam, sizeof(double) * K, cudaMemcpyDeviceToHost));
    CT_CUDA(cudaMemcpy(res.data(), w->res, sizeof(double) * K, cudaMemcpyDeviceToHost));
    for (int i = kf; i < K; ++i) lam[i] = res[i] = NAN;
    if (o->lambda_hist) memcpy(o->lambda_hist, lam.data(), sizeof(double) * K);
    if (o->resid_hist) memcpy(o->resid_hist, res.data(), sizeof(double) * K);
    if (o->ncp_hist) {
        if (o->stop_rule == CT_STOP_NCP && w->ncp)
            CT_CUDA(cudaMemcpy(o->ncp_hist, w->ncp, sizeof(double) * K, cudaMemcpyDeviceToHost));
        else
            for (int i = 0; i < K; ++i) o->ncp_hist[i] = NAN;
    }
    ct_status st = (stop[0] == 0) ? CT_OK : (ct_status)stop[1];
    if (info) {
        info->iters_done = kf;
        info->beta = beta;
        info->final_lambda = kf > 0 ? lam[kf - 1] : 0.0;
        info->final_resid = kf > 0 ? res[kf - 1] : beta;
        info->status = st;
        info->fast_path_steps = 0;
        info->lambda_fallback_steps = 0;
        if (o->rule != CT_LAMBDA_NONE)
            for (int i = 0; i < kf; ++i) {
                info->fast_path_steps += path[i] & 1;
                info->lambda_fallback_steps += (path[i] >> 1) & 1;
            }
    }
    if (st == CT_ENONFINITE) { set_error("solver: non-finite value met"); return st; }
    if (st == CT_ETIMEOUT) {
        set_error("solver: a bounded device wait of the Gram-Schmidt pass expired (the returned "
                  "iterate is not valid)");
        return st;
    }
    return CT_OK;
}

// The hybrid step (Eq. (hybrid_proj)) of step k depends only on H's first k columns, and with
// a fixed iteration count nothing in the Arnoldi chain depends on it.  All K projected problems
// are therefore solved after the loop in one launch, one CTA per k (the lambda_k history is
// the same as if each had been solved inside its iteration); y is formed for the final k.
static SmallSolveParams small_params(Workspace *w, const ct_hybrid_opts *o, double dp_target)
{
    SmallSolveParams p;
    p.H = w->H; p.ldh = w->K + 1; p.k = o->max_iters; p.beta = 0.0; p.betap = w->aux + 2;
    p.rule = o->rule; p.lambda_fixed = o->lambda_fixed; p.dp_target = dp_target;
    p.y = w->Y; p.ystride = w->K;
    p.lambda_out = w->lam;
    p.resid_out = w->res;
    p.stop = w->stop;
    p.kmax = o->max_iters;
    p.always_y = 0;
    p.path = w->path;
    p.net = (o->rule == CT_LAMBDA_LEARNED) ? o->lambda_net_dev : nullptr;
    p.features = o->features_dev;
    return p;
}

// With a stopping rule the hybrid steps run inside the loop, every stop_every steps, for the
// steps since the last check, followed by the device-side check of the rule; after the loop
// one launch forms y at the stopping (or last) step.
// The NCP rule (Sec. 3.2) needs the residual vector itself: at a checked step the iterate
// x_k = x0 + B W_k y_k (AB) or x0 + W_k y_k (BA) is formed, projected, and the periodograms of
// the rows of b - A x_k are taken (one extra B and A for AB, one extra A for BA per check).
struct NcpCtx {
    ct_geom *g = nullptr;
    int method = 0;
    const float *b = nullptr;       // the caller's dense data
    const float *x0 = nullptr;      // AB: padded u0 (or null); BA: x0 image (or null)
};

static ct_status stop_checkpoint(Workspace *w, const ct_hybrid_opts *o, cudaStream_t s,
                                 double dp_target, int step, int &checked, const NcpCtx &nc)
{
    if (o->stop_rule == CT_STOP_NONE) return CT_OK;
    if (step % o->stop_every != 0 && step != o->max_iters) return CT_OK;
    SmallSolveParams p = small_params(w, o, dp_target);
    p.kfirst = checked;
    p.k = step - checked;
    if (o->stop_rule != CT_STOP_NCP) {
        CT_PHASE(CT_PH_SMALL, 2, s);
        CT_CUDA(launch_small_solve_batched(p, s));
        CT_CUDA(launch_stop_check(w->res, checked, step, o->stop_rule, o->tau * o->noise_norm,
                                  o->stop_tol, w->stop, s));
        checked = step;
        return CT_OK;
    }
    p.y_at = step;
    {
        CT_PHASE(CT_PH_SMALL, 1, s);
        CT_CUDA(launch_small_solve_batched(p, s));
    }
    ct_geom *g = nc.g;
    const int64_t L = w->L, ld = w->ld;
    const float *ax;                         // A x_k in the padded sinogram layout
    if (nc.method == 0) {
        {
            CT_PHASE(CT_PH_OTHER, 1, s);     // u = u0 + W_k y_k
            CT_CUDA(launch_combine_basis(o->basis, w->W, L, ld, w->Y, w->K, w->K, nullptr, step,
                                         nc.x0, w->q, kMaxBlocks, s));
        }
        {
            CT_PHASE(CT_PH_BACK, 2, s);      // x_k = B u
            CT_CUDA(launch_back_proj(g, w->q, w->img, w->stop, s));
        }
        {
            CT_PHASE(CT_PH_LAYOUT, 1, s);
            CT_CUDA(launch_image_pairs(g, w->img, w->stop, s));
        }
        {
            CT_PHASE(CT_PH_FORWARD, fwd_launches(g), s);
            CT_CUDA(launch_forward_proj(g, w->q, true, w->stop, s));
        }
        ax = w->q;
    } else {
        {
            CT_PHASE(CT_PH_OTHER, 1, s);     // x_k = x0 + W_k y_k
            if (nc.x0) {
                CT_CUDA(cudaMemsetAsync(w->img, 0, sizeof(float) * L, s));
                CT_CUDA(cudaMemcpyAsync(w->img, nc.x0, sizeof(float) * g->n,
                                        cudaMemcpyDeviceToDevice, s));
            }
            CT_CUDA(launch_combine_basis(o->basis, w->W, L, ld, w->Y, w->K, w->K, nullptr, step,
                                         nc.x0 ? w->img : nullptr, w->q, kMaxBlocks, s));
        }
        {
            CT_PHASE(CT_PH_LAYOUT, 1, s);
            CT_CUDA(launch_image_pairs(g, w->q, w->stop, s));
        }
        {
            CT_PHASE(CT_PH_FORWARD, fwd_launches(g), s);
            CT_CUDA(launch_forward_proj(g, w->sino, true, w->stop, s));
        }
        ax = w->sino;
    }
    {
        CT_PHASE(CT_PH_OTHER, 2, s);
        CT_CUDA(launch_ncp_check(g, nc.b, ax, w->ncp_tw, w->ncp_part, w->ncp, step, checked,
                                 w->stop, s));
    }
    checked = step;
    return CT_OK;
}

static ct_status run_small_solves(Workspace *w, const ct_hybrid_opts *o, cudaStream_t s,
                                  double dp_target)
{
    if (o->stop_rule != CT_STOP_NONE) {            // y of the final step only
        SmallSolveParams p = small_params(w, o, dp_target);
        p.only_y = 1;
        CT_PHASE(CT_PH_SMALL, 1, s);
        CT_CUDA(launch_small_solve_batched(p, s));
        return CT_OK;
    }
    SmallSolveParams p;
    p.H = w->H; p.ldh = w->K + 1; p.k = o->max_iters; p.beta = 0.0; p.betap = w->aux + 2;
    p.rule = o->rule; p.lambda_fixed = o->lambda_fixed; p.dp_target = dp_target;
    p.y = w->Y; p.ystride = w->K;
    p.lambda_out = w->lam;
    p.resid_out = w->res;
    p.stop = w->stop;
    p.kmax = o->max_iters;
    p.always_y = 0;
    p.path = w->path;
    p.net = (o->rule == CT_LAMBDA_LEARNED) ? o->lambda_net_dev : nullptr;
    p.features = o->features_dev;
    CT_PHASE(CT_PH_SMALL, 1, s);
    CT_CUDA(launch_small_solve_batched(p, s));
    return CT_OK;
}

// One hybrid solve (Algorithm 1 or 2) enqueued in pieces: set-up, then per step the operator
// phase (the projectors and their layouts, w_k -> q) and the Arnoldi phase (Eq. (Hessenberg) and
// the stopping checkpoint), then the small solves and the iterate.  enqueue_ab / enqueue_ba run
// the pieces in order on one stream; a batch of two solves interleaves them across its streams.
struct SolveRun {
    ct_geom *g = nullptr;
    const float *b = nullptr;
    const float *init = nullptr;    // AB: u0 (padded when u0_padded), BA: x0; may be null
    float *x = nullptr;
    const ct_hybrid_opts *o = nullptr;
    cudaStream_t s = nullptr;
    int method = 0;
    bool u0_padded = false;
    Workspace *w = nullptr;
    int K = 0, ldh = 0, checked = 0;
    int64_t L = 0, ld = 0;
    ArnoldiScratch sc{nullptr, nullptr, 0, 0};
    double dp_target = 0.0;
    NcpCtx nc;
};

// Algorithm 1 (AB) / 2 (BA) set-up, enqueued on r.s without any host synchronisation
// (graph-capturable once the workspace exists); the caller reads the results with read_info
// after synchronising.
static ct_status run_begin(SolveRun &r)
{
    ct_status st;
    const ct_hybrid_opts *o = r.o;
    ct_geom *g = r.g;
    cudaStream_t s = r.s;
    if ((st = ws_get(g, r.method, o->max_iters, o->basis, &r.w)) != CT_OK) return st;
    Workspace *w = r.w;
    r.K = o->max_iters;
    r.L = w->L;
    r.ld = w->ld;
    r.ldh = w->K + 1;
    r.sc = ArnoldiScratch{w->partial, w->counter, gs_blocks(), w->K};
    r.dp_target = o->tau * o->noise_norm;
    const int64_t L = r.L;
    const ArnoldiScratch &sc = r.sc;
    if (o->stop_rule == CT_STOP_NCP && (st = ncp_ready(g, w)) != CT_OK) return st;
    CT_CUDA(cudaMemsetAsync(w->stop, 0, 2 * sizeof(int), s));
    CT_CUDA(cudaMemsetAsync(w->counter, 0, 4 * sizeof(unsigned), s));
    CT_CUDA(cudaMemsetAsync(w->path, 0, sizeof(int) * r.K, s));
    if (w->ncp) CT_CUDA(cudaMemsetAsync(w->ncp, 0xff, sizeof(double) * w->K, s));   // NaN
    r.nc.g = g; r.nc.method = r.method; r.nc.b = r.b;
    if (r.method == 0) {
        const float *u0_dev = r.init;
        const bool u0_padded = r.u0_padded;
        r.nc.x0 = u0_dev ? (u0_padded ? u0_dev : w->sino) : nullptr;   // padded u0 (kept in sino)
        // Algorithm 1 set-up: x0 = B u0, r0 = b - A x0, w1 = r0 / ||r0||
        CT_PHASE(CT_PH_OTHER, u0_dev ? 8 : 3, s);
        CT_CUDA(launch_pad_sino(g, r.b, w->vec, s));
        if (u0_dev) {
            if (!u0_padded) CT_CUDA(launch_pad_sino(g, u0_dev, w->sino, s));
            CT_CUDA(launch_back_proj(g, u0_padded ? u0_dev : w->sino, w->img, nullptr, s));
            CT_CUDA(launch_image_pairs(g, w->img, nullptr, s));
            CT_CUDA(launch_forward_proj(g, w->q, true, nullptr, s));
            CT_CUDA(launch_rsub(w->vec, w->q, L, kMaxBlocks, s));
            CT_CUDA(normalize_first_basis(o->basis, w->q, L, w->W, sc, w->aux, w->stop, w->cur, s));
        } else {
            CT_CUDA(normalize_first_basis(o->basis, w->vec, L, w->W, sc, w->aux, w->stop, w->cur, s));
        }
    } else {
        const float *x0_dev = r.init;
        const int64_t msino = (int64_t)g->dg.n_views * g->dg.sino_view_ld;
        r.nc.x0 = x0_dev;
        // Algorithm 2 set-up: r0 = B (b - A x0), w1 = r0 / ||r0||
        CT_PHASE(CT_PH_OTHER, x0_dev ? 7 : 4, s);
        CT_CUDA(launch_pad_sino(g, r.b, w->sino, s));
        if (x0_dev) {
            if (!w->sino2) {            // b - A x0 needs a second sinogram (q is image-sized)
                cudaError_t e = dalloc(&w->sino2, (size_t)msino);
                if (e != cudaSuccess) {
                    set_error(std::string("workspace allocation: ") + cudaGetErrorString(e));
                    return CT_ENOMEM;
                }
            }
            CT_CUDA(cudaMemsetAsync(w->img, 0, sizeof(float) * L, s));
            CT_CUDA(cudaMemcpyAsync(w->img, x0_dev, sizeof(float) * g->n, cudaMemcpyDeviceToDevice, s));
            CT_CUDA(launch_image_pairs(g, w->img, nullptr, s));
            CT_CUDA(launch_forward_proj(g, w->sino2, true, nullptr, s));      // A x0
            CT_CUDA(launch_rsub(w->sino, w->sino2, msino, kMaxBlocks, s));    // b - A x0
            CT_CUDA(launch_back_proj(g, w->sino2, w->vec, nullptr, s));
        } else {
            CT_CUDA(launch_back_proj(g, w->sino, w->vec, nullptr, s));
        }
        CT_CUDA(normalize_first_basis(o->basis, w->vec, L, w->W, sc, w->aux, w->stop, w->cur, s));
    }
    return CT_OK;
}

// the operator phase of step `step`: q = A B w_k (AB) or q = B A w_k (BA)
static ct_status run_operator(SolveRun &r, int step)
{
    Workspace *w = r.w;
    ct_geom *g = r.g;
    cudaStream_t s = r.s;
    const int k = step - 1;
    const float *wk = w->cur ? w->cur : static_cast<float *>(w->W) + (int64_t)k * r.ld;
    if (r.method == 0) {
        {
            CT_PHASE(CT_PH_BACK, 2, s);   // pair copy + B, or A^T scatter + rounding
            CT_CUDA(launch_back_proj(g, wk, w->img, w->stop, s));       // q = A B w_k: B w_k
        }
        {
            CT_PHASE(CT_PH_LAYOUT, 1, s);
            CT_CUDA(launch_image_pairs(g, w->img, w->stop, s));
        }
        {
            CT_PHASE(CT_PH_FORWARD, fwd_launches(g), s);
            CT_CUDA(launch_forward_proj(g, w->q, true, w->stop, s));   //          A (B w_k)
        }
    } else {
        {
            CT_PHASE(CT_PH_LAYOUT, 1, s);
            CT_CUDA(launch_image_pairs(g, wk, w->stop, s));           // q = B A w_k: A w_k
        }
        {
            CT_PHASE(CT_PH_FORWARD, fwd_launches(g), s);
            CT_CUDA(launch_forward_proj(g, w->sino, true, w->stop, s));
        }
        {
            CT_PHASE(CT_PH_BACK, 2, s);   // pair copy + B, or A^T scatter + rounding
            CT_CUDA(launch_back_proj(g, w->sino, w->q, w->stop, s));     //          B (A w_k)
        }
    }
    return CT_OK;
}

// the Arnoldi phase of step `step`: column k of H_k and w_{k+1} (Eq. (Hessenberg)), then the
// stopping checkpoint
static ct_status run_arnoldi(SolveRun &r, int step)
{
    Workspace *w = r.w;
    const ct_hybrid_opts *o = r.o;
    cudaStream_t s = r.s;
    const int k = step - 1;
    {
        CT_PHASE(CT_PH_ARNOLDI, arnoldi_step_launches(o->basis, r.ld, k, r.sc, o->reorth != 0, true),
                 s);
        CT_CUDA(arnoldi_step_basis(o->basis, w->W, r.L, r.ld, k, w->q, w->H + (int64_t)k * r.ldh,
                                   r.sc, w->aux, w->stop, step, o->reorth != 0, w->cur, true, s,
                                   step < r.K));
    }
    return stop_checkpoint(w, o, s, r.dp_target, step, r.checked, r.nc);
}

// the hybrid step (Eq. (hybrid_proj)) and the iterate at the last (or stopping) step:
// AB x = x0 + B W y = B (u0 + W y), BA x = x0 + W y
static ct_status run_end(SolveRun &r)
{
    ct_status st;
    Workspace *w = r.w;
    ct_geom *g = r.g;
    const ct_hybrid_opts *o = r.o;
    cudaStream_t s = r.s;
    const int64_t L = r.L, ld = r.ld;
    if ((st = run_small_solves(w, o, s, r.dp_target)) != CT_OK) return st;
    if (r.method == 0) {
        const float *u0_dev = r.init;
        const bool u0_padded = r.u0_padded;
        {
            CT_PHASE(CT_PH_OTHER, u0_dev ? 2 : 1, s);
            if (u0_dev && !u0_padded) CT_CUDA(launch_pad_sino(g, u0_dev, w->sino, s));
            CT_CUDA(launch_combine_basis(o->basis, w->W, L, ld, w->Y, r.K, w->K, w->stop, 0,
                                         u0_dev ? (u0_padded ? u0_dev : w->sino) : nullptr, w->q,
                                         kMaxBlocks, s));
        }
        {
            CT_PHASE(CT_PH_BACK, 2, s);   // pair copy + B, or A^T scatter + rounding
            CT_CUDA(launch_back_proj(g, w->q, r.x, nullptr, s));
        }
    } else {
        const float *x0_dev = r.init;
        CT_PHASE(CT_PH_OTHER, 1, s);
        if (x0_dev) {
            CT_CUDA(cudaMemsetAsync(w->img, 0, sizeof(float) * L, s));
            CT_CUDA(cudaMemcpyAsync(w->img, x0_dev, sizeof(float) * g->n, cudaMemcpyDeviceToDevice, s));
        }
        CT_CUDA(launch_combine_basis(o->basis, w->W, L, ld, w->Y, r.K, w->K, w->stop, 0,
                                     x0_dev ? w->img : nullptr, w->q, kMaxBlocks, s));
        CT_CUDA(cudaMemcpyAsync(r.x, w->q, sizeof(float) * g->n, cudaMemcpyDeviceToDevice, s));
    }
    return CT_OK;
}

static ct_status run_all(SolveRun &r, Workspace **wout)
{
    ct_status st = run_begin(r);
    *wout = r.w;
    if (st != CT_OK) return st;
    for (int step = 1; step <= r.K; ++step) {
        if ((st = run_operator(r, step)) != CT_OK) return st;
        if ((st = run_arnoldi(r, step)) != CT_OK) return st;
    }
    return run_end(r);
}

// Algorithm 1, enqueued on s without any host synchronisation (graph-capturable once the
// workspace exists); the caller reads the results with read_info after synchronising.
static ct_status enqueue_ab(ct_geom *g, const float *b_dev, const float *u0_dev, float *x_dev,
                            const ct_hybrid_opts *o, cudaStream_t s, Workspace **wout,
                            bool u0_padded = false)
{
    SolveRun r;
    r.g = g; r.b = b_dev; r.init = u0_dev; r.x = x_dev; r.o = o; r.s = s; r.method = 0;
    r.u0_padded = u0_padded;
    return run_all(r, wout);
}

extern "C" ct_status ab_gmres_hybrid(ct_geom *g, const float *b_dev, const float *u0_dev,
                                     float *x_dev, const ct_hybrid_opts *o, ct_hybrid_info *info,
                                     ct_stream_t stream)
{
    if (!g || !b_dev || !x_dev) return einval("ab_gmres_hybrid: null argument");
    ct_status st = check_opts(o);
    if (st != CT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Workspace *w = nullptr;
    if ((st = enqueue_ab(g, b_dev, u0_dev, x_dev, o, s, &w)) != CT_OK) return st;
    return finish(w, o, info, s);
}

// Algorithm 2, enqueued on s without host synchronisation (see enqueue_ab).
static ct_status enqueue_ba(ct_geom *g, const float *b_dev, const float *x0_dev, float *x_dev,
                            const ct_hybrid_opts *o, cudaStream_t s, Workspace **wout)
{
    SolveRun r;
    r.g = g; r.b = b_dev; r.init = x0_dev; r.x = x_dev; r.o = o; r.s = s; r.method = 1;
    return run_all(r, wout);
}

extern "C" ct_status ba_gmres_hybrid(ct_geom *g, const float *b_dev, const float *x0_dev,
                                     float *x_dev, const ct_hybrid_opts *o, ct_hybrid_info *info,
                                     ct_stream_t stream)
{
    if (!g || !b_dev || !x_dev) return einval("ba_gmres_hybrid: null argument");
    ct_status st = check_opts(o);
    if (st != CT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Workspace *w = nullptr;
    if ((st = enqueue_ba(g, b_dev, x0_dev, x_dev, o, s, &w)) != CT_OK) return st;
    return finish(w, o, info, s);
}

// ============================================================================ restarts
// Sec. 3.3 (Restarting): cycles of o->max_iters steps, each restarted from the previous
// iterate.  AB keeps the iterate in its own variable u (x = B u), in the padded sinogram layout,
// so a restart is r0 = b - A B u, exactly the restart from x = B u; BA restarts from x.
static ct_status restarted(ct_geom *g, const float *b_dev, float *x_dev, int cycles,
                           const ct_hybrid_opts *o, ct_hybrid_info *info, cudaStream_t s,
                           bool ab)
{
    ct_status st = check_opts(o);
    if (st != CT_OK) return st;
    if (cycles < 1) return einval("restarted solver: cycles must be >= 1");
    const int K = o->max_iters;
    ct_hybrid_opts oc = *o;
    std::vector<double> lam((size_t)K), res((size_t)K);
    oc.lambda_hist = o->lambda_hist ? lam.data() : nullptr;
    oc.resid_hist = o->resid_hist ? res.data() : nullptr;
    oc.features_dev = nullptr;
    oc.ncp_hist = nullptr;
    float *u = nullptr;
    ct_hybrid_info total{};
    for (int c = 0; c < cycles; ++c) {
        Workspace *w = nullptr;
        if (ab) st = enqueue_ab(g, b_dev, c == 0 ? nullptr : u, x_dev, &oc, s, &w, true);
        else st = enqueue_ba(g, b_dev, c == 0 ? nullptr : x_dev, x_dev, &oc, s, &w);
        if (st != CT_OK) break;
        if (ab) {
            if (!u) {
                cudaError_t e = cudaMallocAsync((void **)&u, sizeof(float) * (size_t)w->L, s);
                if (e != cudaSuccess) { st = cuda_fail(e, "restarted solver"); break; }
            }
            cudaError_t e = cudaMemcpyAsync(u, w->q, sizeof(float) * (size_t)w->L,
                                            cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) { st = cuda_fail(e, "restarted solver"); break; }
        }
        ct_hybrid_info ic{};
        st = finish(w, &oc, &ic, s);
        if (st != CT_OK) break;
        if (o->lambda_hist) memcpy(o->lambda_hist + (size_t)c * K, lam.data(), sizeof(double) * K);
        if (o->resid_hist) memcpy(o->resid_hist + (size_t)c * K, res.data(), sizeof(double) * K);
        if (c == 0) total.beta = ic.beta;
        total.iters_done += ic.iters_done;
        total.final_lambda = ic.final_lambda;
        total.final_resid = ic.final_resid;
        total.fast_path_steps += ic.fast_path_steps;
        total.lambda_fallback_steps += ic.lambda_fallback_steps;
        total.status = ic.status;
        if (ic.iters_done == 0) break;           // r0 = 0: the iterate is exact
    }
    if (u) cudaFreeAsync(u, s);
    if (info) *info = total;
    return st;
}

extern "C" ct_status ab_gmres_hybrid_restarted(ct_geom *g, const float *b_dev, float *x_dev,
                                               int cycles, const ct_hybrid_opts *o,
                                               ct_hybrid_info *info, ct_stream_t stream)
{
    if (!g || !b_dev || !x_dev) return einval("ab_gmres_hybrid_restarted: null argument");
    return restarted(g, b_dev, x_dev, cycles, o, info, (cudaStream_t)stream, true);
}

extern "C" ct_status ba_gmres_hybrid_restarted(ct_geom *g, const float *b_dev, float *x_dev,
                                               int cycles, const ct_hybrid_opts *o,
                                               ct_hybrid_info *info, ct_stream_t stream)
{
    if (!g || !b_dev || !x_dev) return einval("ba_gmres_hybrid_restarted: null argument");
    return restarted(g, b_dev, x_dev, cycles, o, info, (cudaStream_t)stream, false);
}

// ============================================================================ building blocks
extern "C" ct_status ct_arnoldi_step(float *W_dev, int64_t len, int64_t ld, int k, float *q_dev,
                                     double *h_dev, ct_stream_t stream)
{
    if (!W_dev || !q_dev || !h_dev) return einval("ct_arnoldi_step: null argument");
    if (k < 0 || k > 1022 || len < 1 || ld < len || (len % 4) || (ld % 4))
        return einval("ct_arnoldi_step: need 0 <= k <= 1022, len % 4 == 0, ld % 4 == 0, ld >= len");
    cudaStream_t s = (cudaStream_t)stream;
    // scratch for this call (the building-block entry point allocates; solvers do not)
    double *partial = nullptr, *aux = nullptr;
    unsigned *counter = nullptr;
    int *stop = nullptr;
    CT_CUDA(cudaMallocAsync((void **)&partial, sizeof(double) * kMaxBlocks * (k + 3), s));
    CT_CUDA(cudaMallocAsync((void **)&aux, sizeof(double) * (8 + 2 * (k + 3)), s));
    CT_CUDA(cudaMallocAsync((void **)&counter, sizeof(unsigned) * 4, s));
    CT_CUDA(cudaMallocAsync((void **)&stop, sizeof(int) * 4, s));
    CT_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned) * 4, s));
    CT_CUDA(cudaMemsetAsync(stop, 0, sizeof(int) * 4, s));
    CT_CUDA(cudaMemsetAsync(h_dev, 0, sizeof(double) * (k + 2), s));
    ArnoldiScratch sc{partial, counter, kMaxBlocks, k + 1};
    CT_CUDA(arnoldi_step_dev(W_dev, len, ld, k, q_dev, h_dev, sc, aux, stop, 1, true, s));
    CT_CUDA(cudaFreeAsync(partial, s));
    CT_CUDA(cudaFreeAsync(aux, s));
    CT_CUDA(cudaFreeAsync(counter, s));
    CT_CUDA(cudaFreeAsync(stop, s));
    return CT_OK;
}

extern "C" ct_status ct_projected_solve(const double *H_dev, int ldh, int k, double beta,
                                        ct_lambda_rule rule, double lambda_fixed, double dp_target,
                                        double *y_dev, double *lambda_dev, double *resid_dev,
                                        ct_stream_t stream)
{
    if (!H_dev || !y_dev || !lambda_dev || !resid_dev) return einval("ct_projected_solve: null argument");
    if (k < 1 || k > kMaxSmallK || ldh < k + 1)
        return einval("ct_projected_solve: need 1 <= k <= " + std::to_string(kMaxSmallK) + " and ldh >= k+1");
    if (rule < CT_LAMBDA_NONE || rule > CT_LAMBDA_LCURVE || rule == CT_LAMBDA_LEARNED)
        return einval("ct_projected_solve: bad rule");
    SmallSolveParams p;
    p.H = H_dev; p.ldh = ldh; p.k = k; p.beta = beta; p.betap = nullptr;
    p.rule = rule; p.lambda_fixed = lambda_fixed; p.dp_target = dp_target;
    p.y = y_dev; p.lambda_out = lambda_dev; p.resid_out = resid_dev; p.stop = nullptr;
    p.kmax = k; p.always_y = 1; p.path = nullptr; p.ystride = 0;
    CT_CUDA(launch_small_solve(p, (cudaStream_t)stream));
    return CT_OK;
}

// ============================================================================ learned lambda
extern "C" ct_status ct_mlp_forward(const float *params_dev, const float *X_dev, int n,
                                    float *out_dev, int bf16, ct_stream_t stream)
{
    if (!params_dev || !X_dev || !out_dev) return einval("ct_mlp_forward: null argument");
    if (n < 0) return einval("ct_mlp_forward: n < 0");
    if (n == 0) return CT_OK;
    CT_CUDA(launch_mlp_forward(params_dev, X_dev, n, out_dev, bf16 != 0, (cudaStream_t)stream));
    g_launches += 1;
    return CT_OK;
}

static ct_status mlp_grad_into(const float *P, const float *X, const float *Y, int n, float *grad,
                               float *loss, bool bf16, float *part, float *lpart, cudaStream_t s)
{
    CT_CUDA(launch_mlp_grad(P, X, Y, n, part, lpart, grad, loss, bf16, s));
    g_launches += 2;
    return CT_OK;
}

extern "C" ct_status ct_mlp_grad(const float *params_dev, const float *X_dev, const float *Y_dev,
                                 int n, float *grad_dev, float *loss_dev, int bf16,
                                 ct_stream_t stream)
{
    if (!params_dev || !X_dev || !Y_dev || !grad_dev) return einval("ct_mlp_grad: null argument");
    if (n < 1) return einval("ct_mlp_grad: n must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    const int nblk = (n + mlp_rows_per_block() - 1) / mlp_rows_per_block();
    float *part = nullptr, *lpart = nullptr;
    CT_CUDA(cudaMallocAsync((void **)&part, sizeof(float) * (size_t)nblk * mlp_num_params(), s));
    CT_CUDA(cudaMallocAsync((void **)&lpart, sizeof(float) * (size_t)nblk, s));
    ct_status st = mlp_grad_into(params_dev, X_dev, Y_dev, n, grad_dev, loss_dev, bf16 != 0, part,
                                 lpart, s);
    CT_CUDA(cudaFreeAsync(part, s));
    CT_CUDA(cudaFreeAsync(lpart, s));
    return st;
}

extern "C" ct_status ct_mlp_adam(float *params_dev, const float *grad_dev, float *m_dev,
                                 float *v_dev, float lr, int t, ct_stream_t stream)
{
    if (!params_dev || !grad_dev || !m_dev || !v_dev) return einval("ct_mlp_adam: null argument");
    if (t < 1 || !(lr > 0.f)) return einval("ct_mlp_adam: need t >= 1 and lr > 0");
    CT_CUDA(launch_mlp_adam(params_dev, grad_dev, m_dev, v_dev, lr, t, (cudaStream_t)stream));
    g_launches += 1;
    return CT_OK;
}

extern "C" ct_status ct_mlp_train(float *params_dev, float *m_dev, float *v_dev, const float *X_dev,
                                  const float *Y_dev, int n, int batch, int epochs, float lr,
                                  int *t, float *loss_hist_dev, int bf16, ct_stream_t stream)
{
    if (!params_dev || !m_dev || !v_dev || !X_dev || !Y_dev || !t)
        return einval("ct_mlp_train: null argument");
    if (n < 1 || batch < 1 || epochs < 0 || *t < 0 || !(lr > 0.f))
        return einval("ct_mlp_train: need n >= 1, batch >= 1, epochs >= 0, *t >= 0, lr > 0");
    cudaStream_t s = (cudaStream_t)stream;
    const int bmax = std::min(batch, n);
    const int nblk = (bmax + mlp_rows_per_block() - 1) / mlp_rows_per_block();
    float *part = nullptr, *lpart = nullptr, *grad = nullptr;
    CT_CUDA(cudaMallocAsync((void **)&part, sizeof(float) * (size_t)nblk * mlp_num_params(), s));
    CT_CUDA(cudaMallocAsync((void **)&lpart, sizeof(float) * (size_t)nblk, s));
    CT_CUDA(cudaMallocAsync((void **)&grad, sizeof(float) * (size_t)mlp_num_params(), s));
    ct_status st = CT_OK;
    int64_t step = 0;
    for (int ep = 0; ep < epochs && st == CT_OK; ++ep) {
        for (int off = 0; off < n && st == CT_OK; off += batch, ++step) {
            const int nb = std::min(batch, n - off);
            st = mlp_grad_into(params_dev, X_dev + (int64_t)off * CT_MLP_NIN, Y_dev + off, nb, grad,
                               loss_hist_dev ? loss_hist_dev + step : nullptr, bf16 != 0, part,
                               lpart, s);
            if (st != CT_OK) break;
            cudaError_t e = launch_mlp_adam(params_dev, grad, m_dev, v_dev, lr, *t + 1, s);
            if (e != cudaSuccess) { st = cuda_fail(e, "ct_mlp_train"); break; }
            g_launches += 1;
            *t += 1;
        }
    }
    cudaFreeAsync(part, s);
    cudaFreeAsync(lpart, s);
    cudaFreeAsync(grad, s);
    return st;
}

extern "C" ct_status ct_lambda_samples(ct_geom *g, const float *b_dev, const float *x_true_dev,
                                       const ct_hybrid_opts *o, float *x_dev, float *feats_dev,
                                       float *labels_dev, ct_hybrid_info *info, ct_stream_t stream)
{
    if (!g || !b_dev || !x_true_dev || !x_dev || !feats_dev || !labels_dev)
        return einval("ct_lambda_samples: null argument");
    ct_status st = check_opts(o);
    if (st != CT_OK) return st;
    if (o->max_iters > 64) return einval("ct_lambda_samples: max_iters must be <= 64");
    if (o->basis != CT_BASIS_F32) return einval("ct_lambda_samples: needs the FP32 basis");
    if (o->rule == CT_LAMBDA_NONE) return einval("ct_lambda_samples: rule must not be CT_LAMBDA_NONE");
    cudaStream_t s = (cudaStream_t)stream;
    ct_hybrid_opts oo = *o;
    oo.features_dev = feats_dev;
    Workspace *w = nullptr;
    if ((st = enqueue_ab(g, b_dev, nullptr, x_dev, &oo, s, &w)) != CT_OK) return st;
    const int K = o->max_iters;
    const int64_t img_ld = round_up(g->n, 4);
    float *Z = nullptr;
    double *G = nullptr;
    CT_CUDA(cudaMallocAsync((void **)&Z, sizeof(float) * (size_t)K * img_ld, s));
    CT_CUDA(cudaMallocAsync((void **)&G, sizeof(double) * (size_t)K * (K + 1), s));
    for (int j = 0; j < K; ++j)         // Z = B W_K (the AB basis is in padded-sinogram layout)
        CT_CUDA(launch_back_proj(g, static_cast<const float *>(w->W) + (int64_t)j * w->ld,
                               Z + (int64_t)j * img_ld, nullptr, s));
    CT_CUDA(launch_gram(Z, img_ld, g->n, K, x_true_dev, G, G + (size_t)K * K, s));
    CT_CUDA(launch_lambda_labels(w->H, w->K + 1, w->aux + 2, G, K, G + (size_t)K * K, labels_dev, s));
    g_launches += 2 * K + 2;
    CT_CUDA(cudaFreeAsync(Z, s));
    CT_CUDA(cudaFreeAsync(G, s));
    return finish(w, &oo, info, s);
}

// ============================================================================ instrumentation
extern "C" ct_status ct_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &r : g_prof_recs) { g_prof_pool.push_back(r.a); g_prof_pool.push_back(r.b); }
    g_prof_recs.clear();
    g_prof_on = (on != 0);
    return CT_OK;
}

extern "C" ct_status ct_profile_collect(ct_phase_time *out)
{
    if (!out) return einval("ct_profile_collect: out is NULL");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (int i = 0; i < CT_PH_COUNT; ++i) out[i] = ct_phase_time{0.0, 0, 0};
    ct_status st = CT_OK;
    for (auto &r : g_prof_recs) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) st = cuda_fail(e, "ct_profile_collect");
        out[r.phase].ms += ms;
        out[r.phase].launches += r.launches;
        out[r.phase].groups += 1;
        g_prof_pool.push_back(r.a);
        g_prof_pool.push_back(r.b);
    }
    g_prof_recs.clear();
    return st;
}

extern "C" int64_t ct_launch_count(void) { return g_launches.load(); }

extern "C" ct_status ct_probe(int kind, int64_t reps, float *out_dev, int64_t out_floats,
                              int64_t *ops, ct_stream_t stream)
{
    if (kind != CT_PROBE_GATHER8 && kind != CT_PROBE_MUFU) return einval("ct_probe: bad kind");
    if (!out_dev || !ops || reps < 1) return einval("ct_probe: need out_dev, ops and reps >= 1");
    int dev = 0, sms = 0;
    CT_CUDA(cudaGetDevice(&dev));
    CT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = probe_blocks_per_sm(kind) * sms;
    const int64_t threads = (int64_t)blocks * probe_threads();
    if (out_floats < threads)
        return einval("ct_probe: out_dev needs " + std::to_string(threads) + " floats");
    const int64_t r = (reps + probe_chains() - 1) / probe_chains() * probe_chains();
    CT_CUDA(launch_probe(kind, r, out_dev, blocks, (cudaStream_t)stream));
    g_launches += 1;
    *ops = threads * r;
    return CT_OK;
}

extern "C" ct_status ct_test_drop_tile_copy(int enable, int64_t wait_cycles)
{
    if (enable && (wait_cycles < (1 << 16) || wait_cycles > (1ll << 31)))
        return einval("ct_test_drop_tile_copy: wait_cycles must be in [2^16, 2^31]");
    CT_CUDA(arnoldi_test_drop_tile_copy(enable, (long long)wait_cycles));
    return CT_OK;
}

// ============================================================================ autotuning
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int, int, int, int, int, int>, ct_launch_shapes> g_tune_cache;

// pixel rows of a B block: b_rows, or the orbit rows of the four-fold kernel's blocks
static int b_block_rows(int b_rows, int b_views)
{
    return b_views == 4 ? (b_rows == 8 ? 4 : 2) : b_rows;
}

static ct_launch_shapes shapes_of(const DeviceGeom &d)
{
    ct_launch_shapes r;
    r.a_threads = d.tune_a_threads;
    r.a_views = d.tune_a_views;
    r.a_slab = d.tune_a_slab;
    r.b_rows = d.tune_b_rows;
    r.b_views = d.tune_b_views;
    r.a_rays = d.tune_a_rays;
    r.a_warp_views = d.tune_a_wviews;
    r.b_warp_rows = d.tune_b_wrows;
    return r;
}

extern "C" ct_status ct_geom_set_launch_shapes(ct_geom *g, const ct_launch_shapes *sh)
{
    if (!g || !sh) return einval("ct_geom_set_launch_shapes: null argument");
    const bool cone = g->desc.kind == CT_CONE3D;
    const auto in = [](int v, std::initializer_list<int> set) {
        for (int u : set) if (v == u) return true;
        return false;
    };
    // the paired-view B kernel is compiled for blocks of at most 256 threads (8 rows); the
    // four-fold kernel (b_views 4) needs a b_rot4 geometry
    bool ok = in(sh->b_rows, {4, 8, 16}) && in(sh->b_views, {1, 2, 4}) &&
              !(sh->b_views == 2 && sh->b_rows > 8) && !(sh->b_views == 4 && !g->dg.b_rot4);
    if (cone)
        ok = ok && sh->a_slab >= 1 && sh->a_views >= 1 && sh->a_views <= 8 && in(sh->a_rays, {1, 2});
    else
        ok = ok && in(sh->a_threads, {128, 256, 512}) && in(sh->a_views, {1, 2, 4, 8}) &&
             in(sh->a_warp_views, {1, 2, 4, 8}) && sh->a_views % sh->a_warp_views == 0 &&
             sh->a_threads / sh->a_views >= 32 / sh->a_warp_views &&
             in(sh->b_warp_rows, {1, 2, 4}) && sh->b_warp_rows <= b_block_rows(sh->b_rows, sh->b_views);
    if (!ok) return einval("ct_geom_set_launch_shapes: launch shape out of range");
    DeviceGeom &dg = g->dg;
    dg.tune_a_threads = sh->a_threads;
    dg.tune_a_views = sh->a_views;
    dg.tune_a_slab = sh->a_slab;
    dg.tune_b_rows = sh->b_rows;
    dg.tune_b_views = sh->b_views;
    dg.tune_a_rays = cone ? sh->a_rays : 1;
    dg.tune_a_wviews = cone ? 1 : sh->a_warp_views;
    dg.tune_b_wrows = cone ? 1 : sh->b_warp_rows;
    return CT_OK;
}

extern "C" ct_status ct_geom_get_launch_shapes(const ct_geom *g, ct_launch_shapes *out)
{
    if (!g || !out) return einval("ct_geom_get_launch_shapes: null argument");
    *out = shapes_of(g->dg);
    return CT_OK;
}

extern "C" ct_status ct_geom_autotune(ct_geom *g, ct_stream_t stream, ct_launch_shapes *out)
{
    if (!g) return einval("ct_geom_autotune: null geometry");
    const bool cone = g->desc.kind == CT_CONE3D;
    DeviceGeom &dg = g->dg;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    CT_CUDA(cudaGetDevice(&dev));
    const auto key = std::make_tuple(dev, (int)g->desc.kind, g->desc.nx, g->desc.ny, g->desc.nz,
                                     g->desc.n_views, g->desc.n_det_u, g->desc.n_det_v,
                                     dg.b_rot4);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            dg.tune_a_threads = it->second.a_threads;
            dg.tune_a_views = it->second.a_views;
            dg.tune_a_slab = it->second.a_slab;
            dg.tune_b_rows = it->second.b_rows;
            dg.tune_b_views = it->second.b_views;
            dg.tune_a_rays = it->second.a_rays;
            dg.tune_a_wviews = it->second.a_warp_views;
            dg.tune_b_wrows = it->second.b_warp_rows;
            if (out) *out = it->second;
            return CT_OK;
        }
    }
    float *x = nullptr, *y = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const size_t ylen = (size_t)dg.n_views * (size_t)dg.sino_view_ld;
    CT_CUDA(cudaMalloc(&x, sizeof(float) * (size_t)g->n));
    CT_CUDA(cudaMalloc(&y, sizeof(float) * ylen));
    CT_CUDA(cudaMemsetAsync(x, 0, sizeof(float) * (size_t)g->n, s));
    CT_CUDA(cudaMemsetAsync(y, 0, sizeof(float) * ylen, s));
    CT_CUDA(cudaEventCreate(&e0));
    CT_CUDA(cudaEventCreate(&e1));
    CT_CUDA(launch_image_pairs(g, x, nullptr, s));
    // time each candidate (one warm-up, best of three) and keep the fastest
    auto time_best = [&](auto launch, int ncand, auto set) -> ct_status {
        float best = 1e30f;
        int best_c = 0;
        for (int c = 0; c < ncand; ++c) {
            set(c);
            CT_CUDA(launch());
            float t = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                CT_CUDA(cudaEventRecord(e0, s));
                CT_CUDA(launch());
                CT_CUDA(cudaEventRecord(e1, s));
                CT_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                CT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                t = std::min(t, ms);
            }
            if (t < best) { best = t; best_c = c; }
        }
        set(best_c);
        return CT_OK;
    };
    // 2D Joseph A: (rays per block, views per block); 3D: z-slab thickness of the Joseph passes;
    // 2D B: (pixel rows per 32-wide block, views per loop iteration); the 3D backprojector has
    // one shape
    // 2D Joseph: (threads, views per block, views per warp)
    static const int a2[15][3] = {{128, 1, 1}, {128, 2, 1}, {128, 4, 1}, {256, 1, 1},
                                  {256, 2, 1}, {256, 4, 1}, {512, 4, 1}, {512, 8, 1},
                                  {128, 2, 2}, {128, 4, 2}, {128, 4, 4}, {256, 4, 4},
                                  {256, 8, 4}, {256, 8, 8}, {512, 8, 4}};
    // 3D: (z-slab thickness, warp rows per block, detector rows per thread); 1 << 20 = one
    // pass over the volume
    static const int a3[12][3] = {{16, 1, 1}, {16, 4, 1}, {16, 8, 1}, {64, 4, 1}, {64, 8, 1},
                                  {1 << 20, 1, 1}, {1 << 20, 4, 1}, {1 << 20, 8, 1},
                                  {16, 4, 2}, {64, 4, 2}, {1 << 20, 2, 2}, {1 << 20, 4, 2}};
    // B: (pixel rows per block, views per iteration, pixel rows per warp); b_views 4 = the
    // four-fold kernel (its blocks have 2, 4, 2 orbit rows for b_rows 4, 8, 16)
    static const int b2[22][3] = {{4, 1, 1}, {8, 1, 1}, {16, 1, 1}, {4, 2, 1}, {8, 2, 1},
                                  {4, 1, 2}, {8, 1, 2}, {16, 1, 2}, {4, 2, 2}, {8, 2, 2},
                                  {4, 1, 4}, {8, 1, 4}, {16, 1, 4}, {4, 2, 4}, {8, 2, 4},
                                  {4, 4, 1}, {8, 4, 1}, {16, 4, 1}, {4, 4, 2}, {8, 4, 2},
                                  {16, 4, 2}, {8, 4, 4}};
    auto fwd = [&]() { return launch_forward_proj(g, y, true, nullptr, s); };
    ct_status st;
    if (cone)
        st = time_best(fwd, 12, [&](int c) {
            dg.tune_a_slab = a3[c][0];
            dg.tune_a_views = a3[c][1];
            dg.tune_a_rays = a3[c][2];
        });
    else
        st = time_best(fwd, 15, [&](int c) {
            dg.tune_a_threads = a2[c][0];
            dg.tune_a_views = a2[c][1];
            dg.tune_a_wviews = a2[c][2];
        });
    if (st == CT_OK && !cone)
        st = time_best([&]() { return launch_back_proj(g, y, x, nullptr, s); }, dg.b_rot4 ? 22 : 15,
                       [&](int c) {
            dg.tune_b_rows = b2[c][0];
            dg.tune_b_views = b2[c][1];
            dg.tune_b_wrows = b2[c][2];
        });
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(y);
    if (st != CT_OK) return st;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = shapes_of(dg);
    }
    if (out) *out = shapes_of(dg);
    return CT_OK;
}

// ============================================================================ batched solves
struct ct_batch {
    int n = 0;
    std::vector<ct_geom *> g;
    std::vector<int> method;
    ct_hybrid_opts o{};
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaEvent_t opdone[2] = {nullptr, nullptr};   // two-solve batches: the operator phases
    cudaStream_t cap = nullptr;         // capture stream (the legacy default stream cannot capture)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const float *> b_ptrs;
    std::vector<float *> x_ptrs;
    std::vector<double> noise;
    std::vector<Workspace *> ws;
    int64_t launches = 0;
};

extern "C" void ct_batch_destroy(ct_batch *bt)
{
    if (!bt) return;
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    for (auto s : bt->streams) if (s) cudaStreamDestroy(s);
    for (auto e : bt->join) if (e) cudaEventDestroy(e);
    if (bt->fork) cudaEventDestroy(bt->fork);
    for (auto e : bt->opdone) if (e) cudaEventDestroy(e);
    if (bt->cap) cudaStreamDestroy(bt->cap);
    delete bt;
}

extern "C" int64_t ct_batch_launches(const ct_batch *bt) { return bt ? bt->launches : 0; }

extern "C" ct_status ct_batch_create(int n_prob, ct_geom *const *geoms, const int *methods,
                                     const ct_hybrid_opts *o, int autotune, ct_batch **out)
{
    if (!out || !geoms || n_prob < 1) return einval("ct_batch_create: need n_prob >= 1, geoms, out");
    *out = nullptr;
    ct_status st = check_opts(o);
    if (st != CT_OK) return st;
    if (o->lambda_hist || o->resid_hist || o->features_dev || o->ncp_hist)
        return einval("ct_batch_create: history and feature pointers must be NULL");
    for (int i = 0; i < n_prob; ++i) {
        if (!geoms[i]) return einval("ct_batch_create: null geometry");
        for (int j = 0; j < i; ++j)
            if (geoms[j] == geoms[i]) return einval("ct_batch_create: each problem needs its own ct_geom");
        int mth = methods ? methods[i] : 2;
        if (mth < 0 || mth > 2) return einval("ct_batch_create: method must be 0, 1 or 2");
    }
    ct_batch *bt = new ct_batch();
    bt->n = n_prob;
    bt->o = *o;
    bt->g.assign(geoms, geoms + n_prob);
    bt->method.resize(n_prob);
    bt->ws.assign(n_prob, nullptr);
    cudaError_t e = small_solve_prepare();
    if (e == cudaSuccess) e = arnoldi_prepare();
    if (e == cudaSuccess) e = mlp_prepare();
    if (e != cudaSuccess) { ct_batch_destroy(bt); return cuda_fail(e, "ct_batch_create"); }
    for (int i = 0; i < n_prob; ++i) {
        int mth = methods ? methods[i] : 2;
        if (mth == 2) mth = (geoms[i]->m < geoms[i]->n) ? 0 : 1;
        bt->method[i] = mth;
        if (autotune && (st = ct_geom_autotune(geoms[i], nullptr, nullptr)) != CT_OK) {
            ct_batch_destroy(bt);
            return st;
        }
        if ((st = ws_get(geoms[i], mth, o->max_iters, o->basis, &bt->ws[i])) != CT_OK ||
            (o->stop_rule == CT_STOP_NCP && (st = ncp_ready(geoms[i], bt->ws[i])) != CT_OK)) {
            ct_batch_destroy(bt);
            return st;
        }
    }
    bt->streams.assign(n_prob, nullptr);
    bt->join.assign(n_prob, nullptr);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->fork, cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&bt->opdone[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking);
    for (int i = 0; i < n_prob && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&bt->streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->join[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) { ct_batch_destroy(bt); return cuda_fail(e, "ct_batch_create"); }
    *out = bt;
    return CT_OK;
}

// Capture every problem's solve as one independent branch of a CUDA graph.
static ct_status batch_capture(ct_batch *bt)
{
    cudaStream_t s = bt->cap;
    if (bt->exec) { cudaGraphExecDestroy(bt->exec); bt->exec = nullptr; }
    if (bt->graph) { cudaGraphDestroy(bt->graph); bt->graph = nullptr; }
    bool prof;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        prof = g_prof_on;
        g_prof_on = false;                  // no per-phase events inside the graph
    }
    const int64_t l0 = g_launches.load();
    ct_status st = CT_OK;
    int dev = 0, sms = 0;
    if (bt->n >= 2 && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
        g_gs_block_cap = std::min(sms, kMaxBlocks);
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(bt->fork, s);
    if (bt->n == 2) {
        // two solves: their steps alternate operator phases (each waits for the other solve's
        // last one), so one solve's projectors run beside the other's HBM-bound Gram-Schmidt
        // passes instead of beside its projectors
        ct_hybrid_opts oi[2];
        SolveRun r[2];
        for (int i = 0; i < 2; ++i) {
            oi[i] = bt->o;
            oi[i].noise_norm = bt->noise[i];
            r[i].g = bt->g[i]; r[i].b = bt->b_ptrs[i]; r[i].x = bt->x_ptrs[i]; r[i].o = &oi[i];
            r[i].s = bt->streams[i]; r[i].method = bt->method[i];
        }
        for (int i = 0; i < 2 && e == cudaSuccess && st == CT_OK; ++i) {
            e = cudaStreamWaitEvent(r[i].s, bt->fork, 0);
            if (e == cudaSuccess) st = run_begin(r[i]);
            bt->ws[i] = r[i].w;
        }
        for (int step = 1; step <= bt->o.max_iters && e == cudaSuccess && st == CT_OK; ++step)
            for (int i = 0; i < 2 && e == cudaSuccess && st == CT_OK; ++i) {
                if (step > 1 || i == 1) e = cudaStreamWaitEvent(r[i].s, bt->opdone[1 - i], 0);
                if (e == cudaSuccess) st = run_operator(r[i], step);
                if (st == CT_OK && e == cudaSuccess) e = cudaEventRecord(bt->opdone[i], r[i].s);
                if (st == CT_OK && e == cudaSuccess) st = run_arnoldi(r[i], step);
            }
        for (int i = 0; i < 2 && e == cudaSuccess && st == CT_OK; ++i) {
            st = run_end(r[i]);
            if (st == CT_OK) e = cudaEventRecord(bt->join[i], r[i].s);
            if (st == CT_OK && e == cudaSuccess) e = cudaStreamWaitEvent(s, bt->join[i], 0);
        }
    }
    for (int i = 0; bt->n != 2 && i < bt->n && e == cudaSuccess && st == CT_OK; ++i) {
        cudaStream_t si = bt->streams[i];
        e = cudaStreamWaitEvent(si, bt->fork, 0);
        if (e != cudaSuccess) break;
        ct_hybrid_opts oi = bt->o;
        oi.noise_norm = bt->noise[i];
        Workspace *w = nullptr;
        st = (bt->method[i] == 0)
                 ? enqueue_ab(bt->g[i], bt->b_ptrs[i], nullptr, bt->x_ptrs[i], &oi, si, &w)
                 : enqueue_ba(bt->g[i], bt->b_ptrs[i], nullptr, bt->x_ptrs[i], &oi, si, &w);
        if (st != CT_OK) break;
        bt->ws[i] = w;
        e = cudaEventRecord(bt->join[i], si);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, bt->join[i], 0);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &graph);
    g_gs_block_cap = 0;
    bt->launches = g_launches.load() - l0;
    g_launches -= bt->launches;             // counted again at every replay
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof_on = prof;
    }
    if (st != CT_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(e, "batch capture"); }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    bt->graph = graph;
    CT_CUDA(cudaGraphInstantiate(&bt->exec, graph, 0));
    return CT_OK;
}

extern "C" ct_status ct_batch_solve(ct_batch *bt, const float *const *b_dev, float *const *x_dev,
                                    const double *noise_norms, ct_hybrid_info *info,
                                    ct_stream_t stream)
{
    if (!bt || !b_dev || !x_dev) return einval("ct_batch_solve: null argument");
    for (int i = 0; i < bt->n; ++i)
        if (!b_dev[i] || !x_dev[i]) return einval("ct_batch_solve: null buffer");
    if (bt->o.rule == CT_LAMBDA_DP && !noise_norms) return einval("ct_batch_solve: DP needs noise_norms");
    cudaStream_t s = (cudaStream_t)stream;
    bool same = bt->exec && bt->b_ptrs.size() == (size_t)bt->n;
    for (int i = 0; same && i < bt->n; ++i) {
        double nz = noise_norms ? noise_norms[i] : 0.0;
        same = bt->b_ptrs[i] == b_dev[i] && bt->x_ptrs[i] == x_dev[i] && bt->noise[i] == nz;
    }
    if (!same) {
        bt->b_ptrs.assign(b_dev, b_dev + bt->n);
        bt->x_ptrs.assign(x_dev, x_dev + bt->n);
        bt->noise.resize(bt->n);
        for (int i = 0; i < bt->n; ++i) {
            bt->noise[i] = noise_norms ? noise_norms[i] : 0.0;
            if (!(bt->noise[i] >= 0)) return einval("ct_batch_solve: noise norms must be >= 0");
        }
        ct_status st = batch_capture(bt);
        if (st != CT_OK) return st;
    }
    CT_CUDA(cudaGraphLaunch(bt->exec, s));
    g_launches += bt->launches;
    CT_CUDA(cudaStreamSynchronize(s));
    ct_status first_err = CT_OK;
    for (int i = 0; i < bt->n; ++i) {
        ct_hybrid_opts oi = bt->o;
        oi.noise_norm = bt->noise[i];
        ct_status st = read_info(bt->ws[i], &oi, info ? &info[i] : nullptr);
        if (st != CT_OK && first_err == CT_OK) first_err = st;
    }
    return first_err;
}

extern "C" ct_status abba_solve(int n_prob, ct_geom *const *geoms, const float *const *b_dev,
                                float *const *x_dev, const int *methods, const ct_hybrid_opts *o,
                                const double *noise_norms, ct_hybrid_info *info, ct_stream_t stream)
{
    ct_batch *bt = nullptr;
    ct_status st = ct_batch_create(n_prob, geoms, methods, o, 1, &bt);
    if (st != CT_OK) return st;
    st = ct_batch_solve(bt, b_dev, x_dev, noise_norms, info, stream);
    ct_batch_destroy(bt);
    return st;
}
