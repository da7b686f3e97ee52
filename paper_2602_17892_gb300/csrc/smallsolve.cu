// The hybrid step of Algorithms 1 and 2 (the lambda choice and Eq. (hybrid_proj)) on the
// device, in FP64 (the fast path's bidiagonalisation in double-float, about 48 bits):
// choose lambda for the (k+1) x k Hessenberg matrix H_k and solve Eq. (hybrid_proj)
//     y = argmin || [H_k; lambda I] y - beta [e1; 0] ||.
//
// lambda = 0 (plain AB/BA-GMRES, Eq. (proj_pbm)): Givens QR of H_k and back substitution.
//
// lambda > 0.  GCV (Sec. 3.1) and the discrepancy principle (Sec. 3.2) need the singular values
// sigma_i of H_k and c_i^2, c = U^T beta e1:
//     rho^2(lambda) = sum_i (lambda^2 c_i / (sigma_i^2 + lambda^2))^2 + c_{k+1}^2,
//     trace(I - H H_lambda) = (k+1) - sum_i sigma_i^2 / (sigma_i^2 + lambda^2).
// GB300 executes FP64 at 1/64 of the FP32 rate, so a sequential FP64 bidiagonal QR (one thread,
// O(k^2) dependent rotations) costs milliseconds.  The fast path keeps the work parallel:
//  1. Householder reduction of H_k to (k+1) x k LOWER bidiagonal Bd = P^T H_k Q with P e1 = e1
//     (the left reflectors act on rows >= 2), so c_i = beta u_i(1) with u_i the left singular
//     vectors of Bd: only first components are needed.  Reflectors are applied one row or one
//     column per thread, in double-float arithmetic (pairs of FP32 numbers) on the FP32 pipe.
//  2. sigma_i: eigenvalues of the Golub-Kahan tridiagonal T of Bd (order 2k+1, zero diagonal,
//     off-diagonals alpha_1, beta_2, alpha_2, ..., beta_{k+1}; eigenvalues +-sigma_i and 0):
//     FP32 bisection (one thread per sigma_i, Sturm counts) gives a bracket, FP64 safeguarded
//     Newton on det(theta I - T) refines it; brackets that touch a neighbour's are first
//     isolated by FP64 Sturm-count multisection, one warp per value (32 counts a round).
//  3. c_i^2 = 2 beta^2 z_i(1)^2 with z_i(1)^2 = det(sigma_i I - T_{2:n}) / p'(sigma_i), the
//     first-component formula of a symmetric tridiagonal's eigenvectors.  For clusters
//     (relative gap < 1e-6) the formula is ill-conditioned; their total weight is a contour
//     integral of e1^T (zI - T)^{-1} e1 around the cluster, shared by its members (GCV and DP
//     depend on a cluster only through that total, to O(gap)).
//  4. c_{k+1}^2 = beta^2 / ||u||^2 with u the left null vector of Bd (an O(k) recurrence).
//  5. Self-check: sum_i c_i^2 + c_{k+1}^2 must equal beta^2.  If it does not, the kernel
//     recomputes sigma and c with the exact sequential path: Householder upper
//     bidiagonalisation of H_k and implicit-shift Golub-Kahan QR.
// The lambda functions are evaluated by the whole block (two lambdas at a time).  y is formed
// only where it is needed (the last step, or a breakdown step): the damped bidiagonal problem
// min ||Bd z - beta e1||^2 + lambda^2 ||z||^2 is eliminated with 2k Givens rotations, and
// y = Q z applies the stored right reflectors.
//
// Parameter readings shared with the FP64 CPU oracle: GCV is evaluated on 256 log-spaced
// lambda in [sigma_1 1e-8, sigma_1], the first grid minimum is refined by 40 golden-section
// steps in log lambda on the neighbouring bracket (kept only if not worse); DP takes the root
// of rho(lambda) = tau ||e|| in that range (the oracle by 60 bisection steps in log lambda,
// this kernel by safeguarded Newton steps in log lambda: the same root up to rounding).
#include <algorithm>

#include "ct_internal.h"
#include "mlp_dev.cuh"

namespace ct {

constexpr int kSSThreads = 256;
constexpr int kGcvGrid = 256;

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// rho^2 and the GCV denominator's trace at lambda, reduced over one warp
__device__ void eval_lambda_warp(double lam, const double *sig, const double *cv, int k,
                                 double &rho2, double &trace)
{
    const int lane = threadIdx.x & 31;
    const double l2 = lam * lam;
    double r = 0.0, t = 0.0;
    for (int i = lane; i < k; i += 32) {
        double s2 = sig[i] * sig[i];
        double den = s2 + l2;
        double f = l2 / den;
        double fc = f * cv[i];
        r += fc * fc;
        t += s2 / den;
    }
    r = warp_sum_d(r);
    t = warp_sum_d(t);
    rho2 = r + cv[k] * cv[k];
    trace = (double)(k + 1) - t;
}

__device__ __forceinline__ void givens(double a, double b, double &c, double &s, double &r)
{
    if (b == 0.0) { c = 1.0; s = 0.0; r = a; return; }
    const double r2 = fma(a, a, b * b);
    if (r2 > 1e-280 && r2 < 1e280) {         // one rsqrt instead of hypot and two divisions
        const double ri = rsqrt(r2);
        c = a * ri;
        s = b * ri;
        r = r2 * ri;
        return;
    }
    r = hypot(a, b);
    c = a / r;
    s = b / r;
}

// The rescaling tests and the Sturm signs read only the high 32 bits of an FP64 value (sign,
// exponent, top of the mantissa): 32-bit integer operations on the value's upper register.
// With 64-bit patterns the same tests cost a Sturm step about 300 cycles instead of 185 on
// GB300, where each FP64 instruction takes about 67 cycles of its sub-partition's pipe.
// |v|'s high word ordered as an integer
__device__ __forceinline__ int abs_hi(double v) { return __double2hiint(v) & 0x7fffffff; }

// 1/x in FP64 from the FP32 reciprocal and two Newton steps (relative error ~1e-16); the range
// test (|x| in (2^-100, 2^100), else a division) on the high word, in integer operations
__device__ __forceinline__ double rcp64(double x)
{
    const int ax = abs_hi(x);
    if (!(ax > 0x39b00000 && ax < 0x46300000)) return 1.0 / x;
    double r = (double)__frcp_rn((float)x);
    r = r * fma(-x, r, 2.0);
    r = r * fma(-x, r, 2.0);
    return r;
}

// Householder vector (LAPACK dlarfg convention): H = I - tau [1; v][1; v]^T maps [alpha; x]
// to [beta; 0] with v = x * scale.  The two reciprocals come from rcp64 (a division costs
// about twice its FP64 instructions, and a reflector's set-up is serial work of the block).
__device__ void make_reflector(double alpha, double xnorm2, double &beta, double &tau, double &scale)
{
    if (xnorm2 == 0.0) { beta = alpha; tau = 0.0; scale = 0.0; return; }
    double nrm = sqrt(alpha * alpha + xnorm2);
    beta = (alpha >= 0.0) ? -nrm : nrm;
    tau = (beta - alpha) * rcp64(beta);
    scale = rcp64(alpha - beta);
}

// Double-FP32 ("double-float") arithmetic for the fast path's bidiagonalisation: a value is an
// unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2 (about 48 significant
// bits).  The error-free transformations are the published ones: Knuth's TwoSum for a sum,
// the fused multiply-add form of Dekker's TwoProduct for a product, and Dekker's FastTwoSum to
// renormalise; the operations carry explicit rounding (no contraction into other operations).
// On GB300 an FP64 instruction holds its sub-partition's FP64 unit for about 67 cycles, while
// these FP32 operations pipeline at full rate, so a double-float multiply-add of about fifteen
// FP32 operations is several times faster than one FP64 multiply-add in a serial chain.
__device__ __forceinline__ float2 df_fast_two_sum(float s, float e)
{
    const float h = __fadd_rn(s, e);
    return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ float2 df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
// c + a b
__device__ __forceinline__ float2 df_fma(float2 c, float2 a, float2 b)
{
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    const float2 st = df_two_sum(c.x, p);
    return df_fast_two_sum(st.x, __fadd_rn(st.y, __fadd_rn(c.y, e)));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b)
{
    const float2 st = df_two_sum(a.x, b.x);
    return df_fast_two_sum(st.x, __fadd_rn(st.y, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 df_mul(float2 a, float2 b)
{
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_from(double v)
{
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}
__device__ __forceinline__ double df_to(float2 a) { return (double)a.x + (double)a.y; }
// x[m * sx] += w * v[m * sv] for m in [0, n), four elements at a time: their loads first, then
// the four independent double-float multiply-adds, then the stores (a shared-memory load cannot
// pass a store to a possibly equal address, so one element at a time would serialise them)
__device__ __forceinline__ void df_axpy(float2 *x, int sx, const float2 *v, int sv, int n, float2 w)
{
    int m = 0;
    for (; m + 3 < n; m += 4) {
        const float2 x0 = x[m * sx], x1 = x[(m + 1) * sx], x2 = x[(m + 2) * sx], x3 = x[(m + 3) * sx];
        const float2 v0 = v[m * sv], v1 = v[(m + 1) * sv], v2 = v[(m + 2) * sv], v3 = v[(m + 3) * sv];
        const float2 y0 = df_fma(x0, w, v0), y1 = df_fma(x1, w, v1);
        const float2 y2 = df_fma(x2, w, v2), y3 = df_fma(x3, w, v3);
        x[m * sx] = y0; x[(m + 1) * sx] = y1; x[(m + 2) * sx] = y2; x[(m + 3) * sx] = y3;
    }
    for (; m < n; ++m) x[m * sx] = df_fma(x[m * sx], w, v[m * sv]);
}
// sum over m in [0, n) of a[m * sa] b[m * sb], in four interleaved double-float sums
__device__ __forceinline__ float2 df_dot(const float2 *a, int sa, const float2 *b, int sb, int n)
{
    float2 s0 = make_float2(0.f, 0.f), s1 = s0, s2 = s0, s3 = s0;
    int m = 0;
    for (; m + 3 < n; m += 4) {
        s0 = df_fma(s0, a[m * sa], b[m * sb]);
        s1 = df_fma(s1, a[(m + 1) * sa], b[(m + 1) * sb]);
        s2 = df_fma(s2, a[(m + 2) * sa], b[(m + 2) * sb]);
        s3 = df_fma(s3, a[(m + 3) * sa], b[(m + 3) * sb]);
    }
    for (; m < n; ++m) s0 = df_fma(s0, a[m * sa], b[m * sb]);
    return df_add(df_add(s0, s1), df_add(s2, s3));
}
// sqrt(q), q > 0: the correctly rounded FP32 root refined by one Newton step (Karp's form,
// s + (q - s^2) / (2 s), with s^2 split exactly): about 48 bits
__device__ __forceinline__ float2 df_sqrt(float2 q)
{
    const float sr = __fsqrt_rn(q.x);
    const float p = __fmul_rn(sr, sr), e = __fmaf_rn(sr, sr, -p);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(q.x, p), e), q.y);
    return df_fast_two_sum(sr, __fmul_rn(r, __fdividef(0.5f, sr)));
}
// 1 / b, b != 0: the correctly rounded FP32 reciprocal refined by one Newton step,
// x + x (1 - b x) with b x split exactly
__device__ __forceinline__ float2 df_rcp(float2 b)
{
    const float x = __frcp_rn(b.x);
    const float p = __fmul_rn(b.x, x), e = __fmaf_rn(b.x, x, -p);
    const float r = __fsub_rn(__fsub_rn(__fsub_rn(1.f, p), e), __fmul_rn(b.y, x));
    return df_fast_two_sum(x, __fmul_rn(x, r));
}
// make_reflector in double-float: [alpha; x] -> [beta; 0] by I - tau [1; v][1; v]^T,
// v = x * scale, from alpha and ||x||^2
__device__ __forceinline__ void make_reflector_df(float2 alpha, float2 xn2, float2 &beta,
                                                  float2 &tau, float2 &scale)
{
    if (xn2.x == 0.f) { beta = alpha; tau = make_float2(0.f, 0.f); scale = tau; return; }
    const float2 nrm = df_sqrt(df_fma(xn2, alpha, alpha));
    beta = (alpha.x >= 0.f) ? df_neg(nrm) : nrm;
    tau = df_mul(df_add(beta, df_neg(alpha)), df_rcp(beta));
    scale = df_rcp(df_add(alpha, df_neg(beta)));
}
__device__ __forceinline__ float2 warp_sum_df(float2 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = df_add(v, make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)));
    return v;
}

// Implicit-shift QR on the upper bidiagonal (d, e), left rotations applied to g.  One thread.
__device__ int bidiag_svd_serial(double *d, double *e, double *g, int n)
{
    const double eps = 2.220446049250313e-16;
    double bnorm = 0.0;
    for (int i = 0; i < n; ++i) bnorm = fmax(bnorm, fabs(d[i]) + (i < n - 1 ? fabs(e[i]) : 0.0));
    if (bnorm == 0.0) return 0;
    int iter = 0;
    const int max_iter = 60 * n + 60;
    int q = n - 1;
    while (q > 0 && iter < max_iter) {
        for (int i = 0; i < q; ++i)
            if (fabs(e[i]) <= eps * (fabs(d[i]) + fabs(d[i + 1]))) e[i] = 0.0;
        while (q > 0 && e[q - 1] == 0.0) --q;
        if (q == 0) break;
        int p = q - 1;
        while (p > 0 && e[p - 1] != 0.0) --p;
        int zi = -1;
        for (int i = p; i <= q; ++i)
            if (fabs(d[i]) <= eps * bnorm) { zi = i; break; }
        if (zi >= 0) {
            d[zi] = 0.0;
            if (zi < q) {   // chase row zi's superdiagonal to the right with left rotations
                double f = e[zi];
                e[zi] = 0.0;
                for (int j = zi + 1; j <= q && f != 0.0; ++j) {
                    double c, s, r;
                    givens(d[j], f, c, s, r);
                    d[j] = r;
                    double gj = g[j], gz = g[zi];
                    g[j] = c * gj + s * gz;
                    g[zi] = -s * gj + c * gz;
                    if (j < q) { f = -s * e[j]; e[j] = c * e[j]; }
                }
            } else {        // d[q] = 0: chase column q's entry upwards with right rotations
                double f = e[q - 1];
                e[q - 1] = 0.0;
                for (int j = q - 1; j >= p && f != 0.0; --j) {
                    double c, s, r;
                    givens(d[j], f, c, s, r);
                    d[j] = r;
                    if (j > p) { f = -s * e[j - 1]; e[j - 1] = c * e[j - 1]; }
                }
            }
            ++iter;
            continue;
        }
        double t11 = d[q - 1] * d[q - 1] + (q - 1 > p ? e[q - 2] * e[q - 2] : 0.0);
        double t12 = d[q - 1] * e[q - 1];
        double t22 = d[q] * d[q] + e[q - 1] * e[q - 1];
        double delta = 0.5 * (t11 - t22);
        double den = delta + (delta >= 0.0 ? 1.0 : -1.0) * hypot(delta, t12);
        double mu = (den == 0.0) ? t22 : t22 - t12 * t12 / den;
        double y = d[p] * d[p] - mu, z = d[p] * e[p];
        for (int j = p; j < q; ++j) {
            double c, s, r;
            givens(y, z, c, s, r);
            if (j > p) e[j - 1] = r;
            y = c * d[j] + s * e[j];
            e[j] = -s * d[j] + c * e[j];
            z = s * d[j + 1];
            d[j + 1] = c * d[j + 1];
            givens(y, z, c, s, r);
            d[j] = r;
            y = c * e[j] + s * d[j + 1];
            d[j + 1] = -s * e[j] + c * d[j + 1];
            double gj = g[j], gj1 = g[j + 1];
            g[j] = c * gj + s * gj1;
            g[j + 1] = -s * gj + c * gj1;
            if (j < q - 1) { z = s * e[j + 1]; e[j + 1] = c * e[j + 1]; }
        }
        e[q - 1] = y;
        ++iter;
    }
    return iter >= max_iter ? -1 : 0;
}

constexpr int kHi2p400 = 0x58f00000;    // high word of 2^400
constexpr int kHi2m400 = 0x26f00000;    // high word of 2^-400
// outside [2^-400, 2^400] (by the high word; a zero high word is an exact zero here: the
// recurrences never get near the subnormal range)
__device__ __forceinline__ bool needs_rescale(int mag)
{
    return mag > kHi2p400 || (mag < kHi2m400 && mag != 0);
}

// det(theta I - T_{first..n-1}) and its derivative by the three-term recurrence, value * 2^ex.
// The scale is checked every fourth step (integer compares of the bit patterns): with the
// scaled T (squared off-diagonals <= 1) and theta <= 2 four steps grow the magnitudes by at
// most 4^4, so values rescaled beyond 2^(+-400) stay far from overflow and underflow.
__device__ void charpoly(const double *t2, int first, int n, double th, double &p, double &dp, int &ex)
{
    double pm2 = 1.0, pm1 = th, qm2 = 0.0, qm1 = 1.0;   // size-1 block: det = theta, d/dth = 1
    int e = 0;
    for (int j = first + 1; j < n; ++j) {
        const double a = t2[j - 1];
        const double pj = th * pm1 - a * pm2;
        const double qj = pm1 + th * qm1 - a * qm2;
        pm2 = pm1; pm1 = pj; qm2 = qm1; qm1 = qj;
        if (((j - first) & 3) == 0) {
            const int mag = max(max(abs_hi(pm1), abs_hi(pm2)), max(abs_hi(qm1), abs_hi(qm2)));
            if (needs_rescale(mag)) {
                const int sh = (mag > kHi2p400) ? -400 : 400;
                pm1 = ldexp(pm1, sh); pm2 = ldexp(pm2, sh);
                qm1 = ldexp(qm1, sh); qm2 = ldexp(qm2, sh);
                e -= sh;
            }
        }
    }
    p = pm1; dp = qm1; ex = e;
}

// Sturm count: number of eigenvalues of the zero-diagonal tridiagonal (squared off-diagonals
// t2[0..n-2]) below x, as the number of sign changes along the leading minors
// p_0 = 1, p_1 = -x, p_j = -x p_{j-1} - t2[j-2] p_{j-2} of T - x I (Sylvester: the pivots of
// T - x I = L D L^T are p_j / p_{j-1}).  Division-free; a zero minor takes the sign opposite to
// its predecessor (as a zero pivot replaced by a tiny negative one would).  Rescaled by powers
// of two every fourth step as in charpoly (x <= 2).
// negative, or zero after a positive predecessor (sprev = false)
__device__ __forceinline__ bool sturm_neg(double v, bool sprev)
{
    const int hi = __double2hiint(v);
    return ((hi << 1) == 0) ? !sprev : (hi < 0);
}

__device__ int count64(const double *t2, int n, double x)
{
    double pm2 = 1.0, pm1 = -x;
    bool sprev = sturm_neg(pm1, false);
    int cnt = sprev;
    for (int j = 2; j <= n; ++j) {
        const double pj = -x * pm1 - t2[j - 2] * pm2;
        const bool sj = sturm_neg(pj, sprev);
        cnt += sj != sprev;
        sprev = sj;
        pm2 = pm1; pm1 = pj;
        if ((j & 3) == 0) {
            const int mag = max(abs_hi(pm1), abs_hi(pm2));
            if (needs_rescale(mag)) {
                const int sh = (mag > kHi2p400) ? -400 : 400;
                pm1 = ldexp(pm1, sh); pm2 = ldexp(pm2, sh);
            }
        }
    }
    return cnt;
}

// det(z I - T) for complex z (rows first..n-1), power-of-two rescaled every fourth step (|z|
// stays below 3, so four steps grow the magnitudes by at most 4^4): value * 2^ex.
__device__ void charpoly_c(const double *t2, int first, int n, double zr, double zi,
                           double &pr, double &pi, int &ex)
{
    double ar = 1.0, ai = 0.0, br = zr, bi = zi;   // p_{j-2}, p_{j-1}
    int e = 0;
    for (int j = first + 1; j < n; ++j) {
        const double a = t2[j - 1];
        double cr = zr * br - zi * bi - a * ar;
        double ci = zr * bi + zi * br - a * ai;
        ar = br; ai = bi; br = cr; bi = ci;
        if (((j - first) & 3) != 0) continue;
        const int mag = max(max(abs_hi(ar), abs_hi(ai)), max(abs_hi(br), abs_hi(bi)));
        if (needs_rescale(mag)) {
            const int sh = (mag > kHi2p400) ? -400 : 400;
            ar = ldexp(ar, sh); ai = ldexp(ai, sh); br = ldexp(br, sh); bi = ldexp(bi, sh);
            e -= sh;
        }
    }
    pr = br; pi = bi; ex = e;
}

// x[m * sx] -= w * v[m * sv] for m in [0, n): four loads of each operand first, then the four
// FP64 multiply-adds, then the four stores, so that a store waits for an FP64 result once per
// four elements (with one element at a time every store waited for its multiply-add, about 67
// cycles on GB300's FP64 pipe)
__device__ __forceinline__ void axpy_sub(double *x, int sx, const double *v, int sv, int n, double w)
{
    int m = 0;
    for (; m + 3 < n; m += 4) {
        const double x0 = x[m * sx], x1 = x[(m + 1) * sx], x2 = x[(m + 2) * sx], x3 = x[(m + 3) * sx];
        const double v0 = v[m * sv], v1 = v[(m + 1) * sv], v2 = v[(m + 2) * sv], v3 = v[(m + 3) * sv];
        const double y0 = fma(-w, v0, x0), y1 = fma(-w, v1, x1);
        const double y2 = fma(-w, v2, x2), y3 = fma(-w, v3, x3);
        x[m * sx] = y0; x[(m + 1) * sx] = y1; x[(m + 2) * sx] = y2; x[(m + 3) * sx] = y3;
    }
    for (; m < n; ++m) x[m * sx] = fma(-w, v[m * sv], x[m * sx]);
}

size_t small_solve_smem_bytes(int k)
{
    size_t nd = (size_t)((k + 1) | 1) * k + 16 * (size_t)(k + 1) + kGcvGrid + 64;
    return nd * sizeof(double);
}

__global__ void __launch_bounds__(kSSThreads, 1) small_solve_kernel(SmallSolveParams P, int batched)
{
    if (batched) {
        // block b solves step k = kfirst + (count - b): the largest problems (longest blocks)
        // start first, on separate SMs, and the short ones fill in behind them
        const int kk = P.kfirst + (int)(gridDim.x - blockIdx.x);
        P.k = kk;
        P.y += (size_t)(kk - 1) * P.ystride;
        P.lambda_out += kk - 1;
        P.resid_out += kk - 1;
        if (P.path) P.path += kk - 1;
    }
    const int k = P.k;
    int stop_now = 0;
    if (P.stop) {
        int st = P.stop[0];
        if (st < 0 || (st > 0 && k > st)) return;
        stop_now = (st == k);
    }
    if (P.only_y) {
        const int target = (P.stop && P.stop[0] > 0) ? P.stop[0] : P.kmax;
        if (k != target) return;
    }
    const bool need_y = P.always_y || k == P.kmax || stop_now || P.only_y || k == P.y_at;
    extern __shared__ double sd[];
    // (k+1) x k, column-major, leading dimension odd: a warp's threads walking columns at once
    // (one column each) then touch 8-byte words lda apart, which an even lda would put in one
    // shared-memory bank
    const int lda = (k + 1) | 1;
    double *A = sd;
    double *g = A + (size_t)lda * k;      // k+1
    double *d = g + (k + 1);              // k
    double *e = d + (k + 1);              // k
    double *tauR = e + (k + 1);           // k
    double *dsv = tauR + (k + 1);
    double *esv = dsv + (k + 1);
    double *gsv = esv + (k + 1);          // k+1
    double *sig = gsv + (k + 1);
    double *cv = sig + (k + 1);           // k+1
    double *z = cv + (k + 1);
    double *rot = z + (k + 1);            // 2(k+1)
    double *t2 = rot + 2 * (k + 1);       // 2(k+1): squared tridiagonal off-diagonals
    float *lo32 = (float *)(t2 + 2 * (k + 1));   // k floats
    float *hi32 = lo32 + (k + 1);                // k floats
    float *t2f = hi32 + (k + 1);                 // 2(k+1) floats
    double *red = (double *)(t2f + 2 * (k + 1)); // kGcvGrid
    double *misc = red + kGcvGrid;               // 64
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = kSSThreads / 32;
    const double beta = P.betap ? *P.betap : P.beta;

    auto load_H = [&]() {
        for (int t = tid; t < lda * k; t += kSSThreads) {
            int c = t / lda, r = t - c * lda;
            A[t] = (r <= k) ? P.H[(size_t)c * P.ldh + r] : 0.0;   // the padding row is zero
        }
        for (int t = tid; t <= k; t += kSSThreads) g[t] = (t == 0) ? beta : 0.0;
        __syncthreads();
    };
    // Givens QR of the Hessenberg matrix in A, rotations applied to g (columns in parallel)
    auto givens_qr = [&]() {
        for (int j = 0; j < k; ++j) {
            if (tid == 0) {
                double c, s, r;
                givens(A[j * lda + j], A[j * lda + j + 1], c, s, r);
                rot[0] = c; rot[1] = s;
                double gj = g[j], gj1 = g[j + 1];
                g[j] = c * gj + s * gj1;
                g[j + 1] = -s * gj + c * gj1;
            }
            __syncthreads();
            const double c = rot[0], s = rot[1];
            for (int l = j + tid; l < k; l += kSSThreads) {
                double a0 = A[l * lda + j], a1 = A[l * lda + j + 1];
                A[l * lda + j] = c * a0 + s * a1;
                A[l * lda + j + 1] = -s * a0 + c * a1;
            }
            __syncthreads();
        }
    };

    load_H();
    double lam = 0.0;
    if (P.rule == CT_LAMBDA_NONE) {
        // ---------------- Eq. (proj_pbm): Givens QR and back substitution
        givens_qr();
        for (int i = k - 1; i >= 0; --i) {
            if (tid == 0) {
                double rii = A[i * lda + i];
                z[i] = (rii != 0.0) ? g[i] / rii : 0.0;
            }
            __syncthreads();
            const double zi = z[i];
            for (int l = tid; l < i; l += kSSThreads) g[l] -= A[i * lda + l] * zi;
            __syncthreads();
        }
        for (int i = tid; i < k; i += kSSThreads) P.y[i] = z[i];
        if (tid == 0) {
            *P.lambda_out = 0.0;
            *P.resid_out = fabs(g[k]);
        }
        return;
    }

    // ================================================================ fast path
    // lower bidiagonalisation of H_k ((k+1) x k) with e1 fixed: right reflector on row j
    // (columns j..k-1) -> alpha_j = d[j]; left reflector on column j (rows j+1..k) ->
    // beta_{j+1} = e[j].  Rows/columns are applied one per thread (no shuffles).  The matrix is
    // held in double-float in place of its FP64 copy (an element's hi and lo in its 8 bytes) and
    // the updates run in double-float; each reflector is formed in FP64 from its double-float
    // vector (make_reflector), and d, e, tau are kept in FP64.  At the end the matrix, which now
    // holds the scaled right reflectors the y step applies, is turned back into FP64.  Double-
    // float has FP32's exponent range, so the matrix is first scaled by a power of two that
    // brings its largest entry into [1, 2) (the reflectors do not change; d and e are scaled
    // back); the exponents are compared as integers on the high words.
    float2 *Af = reinterpret_cast<float2 *>(A);
    int *emax = reinterpret_cast<int *>(misc + 12);
    if (tid == 0) *emax = 0;
    __syncthreads();
    {
        int em = 0;
        for (int t = tid; t < lda * k; t += kSSThreads) em = max(em, (__double2hiint(A[t]) >> 20) & 0x7ff);
        em = __reduce_max_sync(0xffffffffu, em);
        if (lane == 0) atomicMax(emax, em);
    }
    __syncthreads();
    // 2^(1023 - emax) and its inverse as FP64 bit patterns (a zero or subnormal matrix: 1)
    const int eb = (*emax >= 1 && *emax <= 2045) ? *emax : 1023;
    const double dscale = __hiloint2double((2046 - eb) << 20, 0);
    const double dunscale = __hiloint2double(eb << 20, 0);
    for (int t = tid; t < lda * k; t += kSSThreads) Af[t] = df_from(A[t] * dscale);
    __syncthreads();
    // reflector constants (beta, tau, scale) in double-float, and d, e, tau kept in double-float
    // in their FP64 slots until the end
    float2 *mf = reinterpret_cast<float2 *>(misc + 16);
    float2 *dF = reinterpret_cast<float2 *>(d), *eF = reinterpret_cast<float2 *>(e);
    float2 *tF = reinterpret_cast<float2 *>(tauR);
    for (int j = 0; j < k; ++j) {
        if (warp == 0) {
            float2 s2 = make_float2(0.f, 0.f);
            for (int l = j + 1 + lane; l < k; l += 32) s2 = df_fma(s2, Af[l * lda + j], Af[l * lda + j]);
            s2 = warp_sum_df(s2);
            if (lane == 0) make_reflector_df(Af[j * lda + j], s2, mf[0], mf[1], mf[2]);
        }
        __syncthreads();
        {
            const float2 bt = mf[0], tauf = mf[1], scf = mf[2];
            for (int l = j + 1 + tid; l < k; l += kSSThreads) Af[l * lda + j] = df_mul(Af[l * lda + j], scf);
            __syncthreads();
            if (tauf.x != 0.f) {
                for (int i = j + 1 + tid; i <= k; i += kSSThreads) {   // row i
                    const float2 *vj = Af + (size_t)(j + 1) * lda + j;  // v_l, l > j (stride lda)
                    float2 *ri = Af + (size_t)(j + 1) * lda + i;         // A[i][l], l > j
                    const float2 w = df_add(Af[j * lda + i], df_dot(vj, lda, ri, lda, k - j - 1));
                    const float2 nw = df_neg(df_mul(w, tauf));
                    Af[j * lda + i] = df_add(Af[j * lda + i], nw);
                    df_axpy(ri, lda, vj, lda, k - j - 1, nw);
                }
            }
            if (tid == 0) { Af[j * lda + j] = bt; dF[j] = bt; tF[j] = tauf; }
        }
        __syncthreads();
        if (warp == 0) {
            float2 s2 = make_float2(0.f, 0.f);
            for (int i = j + 2 + lane; i <= k; i += 32) s2 = df_fma(s2, Af[j * lda + i], Af[j * lda + i]);
            s2 = warp_sum_df(s2);
            if (lane == 0) make_reflector_df(Af[j * lda + j + 1], s2, mf[0], mf[1], mf[2]);
        }
        __syncthreads();
        {
            const float2 bt = mf[0], tauf = mf[1], scf = mf[2];
            for (int i = j + 2 + tid; i <= k; i += kSSThreads) Af[j * lda + i] = df_mul(Af[j * lda + i], scf);
            __syncthreads();
            if (tauf.x != 0.f) {
                for (int l = j + 1 + tid; l < k; l += kSSThreads) {     // column l
                    float2 *col = Af + (size_t)l * lda;
                    const float2 *vj = Af + (size_t)j * lda + j + 2;     // v_i, i > j + 1
                    const float2 w = df_add(col[j + 1], df_dot(vj, 1, col + j + 2, 1, k - j - 1));
                    const float2 nw = df_neg(df_mul(w, tauf));
                    col[j + 1] = df_add(col[j + 1], nw);
                    df_axpy(col + j + 2, 1, vj, 1, k - j - 1, nw);
                }
            }
            if (tid == 0) { Af[j * lda + j + 1] = bt; eF[j] = bt; }
        }
        __syncthreads();
    }
    // d, e (scaled back) and tau to FP64 in place
    for (int i = tid; i < k; i += kSSThreads) {
        const double di = df_to(dF[i]) * dunscale, ei = df_to(eF[i]) * dunscale, ti = df_to(tF[i]);
        d[i] = di; e[i] = ei; tauR[i] = ti;
    }
    // back to FP64 in place: each thread reads its elements before writing them
    for (int t = tid; t < lda * k; t += kSSThreads) {
        const double v = df_to(Af[t]);
        A[t] = v;
    }
    __syncthreads();
    // Golub-Kahan tridiagonal T (n = 2k+1, zero diagonal) of the (k+1) x k lower bidiagonal:
    // off-diagonals alpha_0, beta_1, alpha_1, ..., alpha_{k-1}, beta_k; eigenvalues +-sigma_i, 0
    const int n = 2 * k + 1;
    if (warp == 0) {
        double mx = 0.0;
        for (int i = lane; i < k; i += 32) mx = fmax(mx, fmax(fabs(d[i]), fabs(e[i])));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) misc[4] = mx;
    }
    __syncthreads();
    const double tscale = misc[4];
    const double inv_ts = (tscale > 0.0) ? 1.0 / tscale : 0.0;
    for (int j = tid; j < n - 1; j += kSSThreads) {
        double t = ((j & 1) == 0 ? d[j >> 1] : e[j >> 1]) * inv_ts;
        t2[j] = t * t;
        t2f[j] = (float)(t * t);
    }
    __syncthreads();
    // sigma_i (i-th largest), one thread each: FP32 bisection with Sturm counts; for x > 0 the
    // count of eigenvalues below x is k + 1 + #{sigma < x}
    for (int i = tid; i < k; i += kSSThreads) {
        // three Sturm counts per step (independent recurrences, interleaved): the bracket
        // shrinks fourfold per step
        float lo = 0.f, hi = 2.f;
        const int target = k - i;               // #{sigma < x} >= target  <=>  sigma_i < x
        for (int it = 0; it < 80 && (hi - lo) > 2e-6f * hi; ++it) {
            const float w = hi - lo;
            const float x1 = lo + 0.25f * w, x2 = lo + 0.5f * w, x3 = lo + 0.75f * w;
            float d1 = -x1, d2 = -x2, d3 = -x3;
            if (fabsf(d1) < 1e-30f) d1 = -1e-30f;
            if (fabsf(d2) < 1e-30f) d2 = -1e-30f;
            if (fabsf(d3) < 1e-30f) d3 = -1e-30f;
            int c1 = d1 < 0.f, c2 = d2 < 0.f, c3 = d3 < 0.f;
            for (int j = 1; j < n; ++j) {
                const float t = t2f[j - 1];
                d1 = -x1 - __fdividef(t, d1);
                d2 = -x2 - __fdividef(t, d2);
                d3 = -x3 - __fdividef(t, d3);
                if (fabsf(d1) < 1e-30f) d1 = -1e-30f;
                if (fabsf(d2) < 1e-30f) d2 = -1e-30f;
                if (fabsf(d3) < 1e-30f) d3 = -1e-30f;
                c1 += d1 < 0.f; c2 += d2 < 0.f; c3 += d3 < 0.f;
            }
            const int off = k + 1;
            if (c1 - off >= target) hi = x1;
            else if (c2 - off >= target) { lo = x1; hi = x2; }
            else if (c3 - off >= target) { lo = x2; hi = x3; }
            else lo = x3;
        }
        lo32[i] = lo;
        hi32[i] = hi;
    }
    __syncthreads();
    // FP64: brackets that overlap a neighbour's are isolated by FP64 Sturm-count multisection,
    // one warp per value: its 32 lanes count at 32 points of the bracket at once (an FP64 warp
    // instruction costs the same with 1 or 32 lanes active), which narrows the bracket 33-fold
    // per round where bisection halves it.  Then safeguarded Newton on det(theta I - T), one
    // thread per value; c_i^2 by the first-component formula.
    double *sblo = dsv, *sbhi = esv;                 // brackets (dsv, esv are free until y)
    int *niso = reinterpret_cast<int *>(gsv);        // the values to isolate, then their count
    for (int i = tid; i < k; i += kSSThreads) {
        const double blo = (double)lo32[i] * (1.0 - 2e-4), bhi = (double)hi32[i] * (1.0 + 2e-4);
        const bool iso = (i == 0 || (double)lo32[i - 1] * (1.0 - 2e-4) > bhi) &&
                         (i == k - 1 || (double)hi32[i + 1] * (1.0 + 2e-4) < blo);
        sblo[i] = blo;
        sbhi[i] = iso ? bhi : -bhi;                  // sign: still to isolate
    }
    __syncthreads();
    if (tid == 0) {
        int m = 0;
        for (int i = 0; i < k; ++i)
            if (sbhi[i] < 0.0) { sbhi[i] = -sbhi[i]; niso[1 + m++] = i; }
        niso[0] = m;
    }
    __syncthreads();
    for (int v = warp; v < niso[0]; v += nwarps) {
        const int i = niso[1 + v], tgt = k - i;
        double blo = sblo[i], bhi = sbhi[i];
        int clo = 0, chi = k;
        // round 0 counts at both ends (lanes 0 and 31) and 30 points between; later rounds at
        // 32 interior points.  Counts grow with x; the first lane with count >= tgt bounds the
        // value from above, the lane before it from below.
        for (int round = 0; round < 40; ++round) {
            const double w = bhi - blo;
            const double x = (round == 0) ? blo + w * ((double)lane * (1.0 / 31.0))
                                          : blo + w * ((double)(lane + 1) * (1.0 / 33.0));
            const int c = count64(t2, n, x) - (k + 1);
            if (round == 0) {
                const int c0 = __shfl_sync(0xffffffffu, c, 0), c31 = __shfl_sync(0xffffffffu, c, 31);
                if (!(c0 <= tgt - 1 && c31 >= tgt)) {     // not a bracket: the whole range
                    blo = 0.0; bhi = 2.0; clo = 0; chi = k;
                    continue;
                }
            }
            const unsigned up = __ballot_sync(0xffffffffu, c >= tgt);
            const int f = up ? __ffs(up) - 1 : 32;
            const double xf = __shfl_sync(0xffffffffu, x, f & 31), xb = __shfl_sync(0xffffffffu, x, (f + 31) & 31);
            const int cf = __shfl_sync(0xffffffffu, c, f & 31), cb = __shfl_sync(0xffffffffu, c, (f + 31) & 31);
            if (f < 32) { bhi = xf; chi = cf; }
            if (f > 0) { blo = xb; clo = cb; }
            if (!(chi - clo > 1 && bhi - blo > 1e-15 * bhi)) break;
        }
        if (lane == 0) { sblo[i] = blo; sbhi[i] = bhi; }
    }
    __syncthreads();
    for (int i = tid; i < k; i += kSSThreads) {
        double blo = sblo[i], bhi = sbhi[i];
        double th = 0.5 * (blo + bhi), th_eval = th;
        double p = 0.0, dp = 0.0;
        int ex = 0;
        // just below sigma_i, i+1 eigenvalues of T lie above theta: det(theta I - T) has sign (-1)^(i+1)
        const bool neg_lo = (i % 2 == 0);
        for (int it = 0; it < 12; ++it) {
            charpoly(t2, 0, n, th, p, dp, ex);
            th_eval = th;
            if (p == 0.0) break;
            if ((p < 0.0) == neg_lo) blo = th; else bhi = th;
            const double delta = p / dp;
            if (fabs(delta) <= 2e-16 * fabs(th)) break;          // converged at th_eval
            double nt = th - delta;
            if (!(nt > blo && nt < bhi)) nt = 0.5 * (blo + bhi);   // safeguard: bisect
            th = nt;
            if (bhi - blo <= 4e-16 * bhi) break;
        }
        // first component of the eigenvector: z1^2 = det(th I - T_{2:n}) / p'(th), both at the
        // last evaluation point (within a rounding error of the root); c_i^2 = 2 beta^2 z1^2
        int ex2;
        double p2, dp2;
        charpoly(t2, 1, n, th_eval, p2, dp2, ex2);
        double z1sq = (dp != 0.0) ? ldexp(p2 / dp, ex2 - ex) : -1.0;
        sig[i] = th;                               // scaled units until the end of this block
        double c2 = 2.0 * beta * beta * z1sq;
        cv[i] = (c2 >= 0.0 && isfinite(c2)) ? c2 : -1.0;   // c_i^2 for now
    }
    __syncthreads();
    // clusters (relative gap < 1e-6): the first-component formula is ill-conditioned there, but
    // lambda rules only see a cluster's total weight sum c_i^2, a contour integral of the
    // resolvent entry r(z) = e1^T (z I - T)^{-1} e1 = det(zI - T_{2:n}) / det(zI - T) around it
    // (32-point trapezoidal rule on a circle of a third of the distance to the next eigenvalue)
    int *clist = reinterpret_cast<int *>(rot);
    if (tid == 0) {
        int nc = 0;
        for (int i = 0; i < k;) {
            int b = i;
            while (b + 1 < k && sig[b] - sig[b + 1] < 1e-6 * sig[b]) ++b;
            if (b > i) { clist[2 * nc] = i; clist[2 * nc + 1] = b; ++nc; }
            i = b + 1;
        }
        misc[7] = (double)nc;
        // c_{k+1}: the left null vector of the lower bidiagonal (u_1 = 1,
        // u_{i+1} = -alpha_i u_i / beta_{i+1}) gives c_{k+1}^2 = beta^2 / ||u||^2
        double sq = 1.0, uu = 1.0;
        int exs = 0;
        bool exact = false;
        for (int i = 0; i < k; ++i) {
            if (e[i] == 0.0) { exact = true; break; }
            uu *= -d[i] / e[i];
            sq += uu * uu;
            if (sq > 0x1p+500) { sq = ldexp(sq, -500); uu = ldexp(uu, -250); exs += 500; }
        }
        misc[3] = exact ? 0.0 : fabs(beta) / sqrt(ldexp(sq, 0)) * ldexp(1.0, -exs / 2);
    }
    __syncthreads();
    {
        const int nc = (int)misc[7];
        for (int q = warp; q < nc; q += nwarps) {
            const int a = clist[2 * q], b = clist[2 * q + 1];
            const double c = 0.5 * (sig[a] + sig[b]), half = 0.5 * (sig[a] - sig[b]);
            double R = c;                                           // the eigenvalue 0 of T
            if (a > 0) R = fmin(R, sig[a - 1] - c);
            if (b + 1 < k) R = fmin(R, c - sig[b + 1]);
            const double rho = fmax(R / 3.0, 10.0 * half);
            const double ph = 2.0 * 3.141592653589793 * (lane + 0.5) / 32.0;
            double sn, cs;
            sincos(ph, &sn, &cs);
            const double zr = c + rho * cs, zi = rho * sn;
            double pr, pi, p2r, p2i;
            int ex, ex2;
            charpoly_c(t2, 0, n, zr, zi, pr, pi, ex);
            charpoly_c(t2, 1, n, zr, zi, p2r, p2i, ex2);
            const double den = pr * pr + pi * pi;
            double rr = (p2r * pr + p2i * pi) / den, ri = (p2i * pr - p2r * pi) / den;
            rr = ldexp(rr, ex2 - ex); ri = ldexp(ri, ex2 - ex);
            double w = rho * (cs * rr - sn * ri);                   // Re(rho e^{i ph} r(z))
            w = warp_sum_d(w) / 32.0;
            if (lane == 0) {
                const double each = 2.0 * beta * beta * w / (double)(b - a + 1);
                for (int j = a; j <= b; ++j) cv[j] = (each >= 0.0 && isfinite(each)) ? each : -1.0;
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < k; i += kSSThreads) {
        sig[i] *= tscale;
        cv[i] = (cv[i] >= 0.0) ? sqrt(cv[i]) : -1.0;
    }
    if (tid == 0) cv[k] = misc[3];
    __syncthreads();
    // self-check: sum c_i^2 = beta^2 (U orthogonal) and the sigma non-increasing
    if (warp == 0) {
        double s = 0.0;
        int bad = 0;
        for (int i = lane; i <= k; i += 32) {
            if (cv[i] < 0.0 || !isfinite(cv[i]) || (i < k && !isfinite(sig[i]))) bad = 1;
            else s += cv[i] * cv[i];
            if (i + 1 < k && !(sig[i] >= sig[i + 1])) bad = 1;
        }
        s = warp_sum_d(s);
        bad = __any_sync(0xffffffffu, bad);
        if (lane == 0) {
            double ref = beta * beta;
            misc[6] = (bad || !(fabs(s - ref) <= 1e-10 * ref)) ? 1.0 : 0.0;
            misc[8] = sig[0];
        }
    }
    __syncthreads();
    const bool fast = misc[6] == 0.0;
    if (tid == 0 && P.path) *P.path = fast ? 1 : 0;

    if (!fast) {
        // ================================================================ exact sequential path
        __syncthreads();
        load_H();
        for (int j = 0; j < k; ++j) {
            if (warp == 0) {
                double s2 = 0.0;
                for (int i = j + 1 + lane; i <= k; i += 32) s2 += A[j * lda + i] * A[j * lda + i];
                s2 = warp_sum_d(s2);
                if (lane == 0) {
                    double bt, tau, sc;
                    make_reflector(A[j * lda + j], s2, bt, tau, sc);
                    misc[0] = bt; misc[1] = tau; misc[2] = sc;
                }
            }
            __syncthreads();
            {
                const double bt = misc[0], tau = misc[1], sc = misc[2];
                for (int i = j + 1 + tid; i <= k; i += kSSThreads) A[j * lda + i] *= sc;
                __syncthreads();
                if (tid == 0) { A[j * lda + j] = bt; d[j] = bt; }
                if (tau != 0.0) {
                    for (int l = j + 1 + warp; l <= k; l += nwarps) {
                        double *col = (l < k) ? A + (size_t)l * lda : g;
                        const double cj = col[j];
                        double w = 0.0;
                        for (int i = j + 1 + lane; i <= k; i += 32) w += A[j * lda + i] * col[i];
                        w = (warp_sum_d(w) + cj) * tau;
                        __syncwarp();
                        if (lane == 0) col[j] -= w;
                        for (int i = j + 1 + lane; i <= k; i += 32) col[i] -= w * A[j * lda + i];
                    }
                }
            }
            __syncthreads();
            if (j < k - 1) {
                if (warp == 0) {
                    double s2 = 0.0;
                    for (int l = j + 2 + lane; l < k; l += 32) s2 += A[l * lda + j] * A[l * lda + j];
                    s2 = warp_sum_d(s2);
                    if (lane == 0) {
                        double bt, tau, sc;
                        make_reflector(A[(j + 1) * lda + j], s2, bt, tau, sc);
                        misc[0] = bt; misc[1] = tau; misc[2] = sc;
                    }
                }
                __syncthreads();
                const double bt = misc[0], tau = misc[1], sc = misc[2];
                for (int l = j + 2 + tid; l < k; l += kSSThreads) A[l * lda + j] *= sc;
                __syncthreads();
                if (tid == 0) { A[(j + 1) * lda + j] = bt; e[j] = bt; tauR[j] = tau; }
                if (tau != 0.0) {
                    for (int i = j + 1 + warp; i <= k; i += nwarps) {
                        const double ai = A[(j + 1) * lda + i];
                        double w = 0.0;
                        for (int l = j + 2 + lane; l < k; l += 32) w += A[l * lda + j] * A[l * lda + i];
                        w = (warp_sum_d(w) + ai) * tau;
                        __syncwarp();
                        if (lane == 0) A[(j + 1) * lda + i] -= w;
                        for (int l = j + 2 + lane; l < k; l += 32) A[l * lda + i] -= w * A[l * lda + j];
                    }
                }
                __syncthreads();
            }
        }
        for (int i = tid; i <= k; i += kSSThreads) {
            if (i < k) { dsv[i] = d[i]; esv[i] = (i < k - 1) ? e[i] : 0.0; }
            gsv[i] = g[i];
        }
        __syncthreads();
        if (tid == 0) {
            bidiag_svd_serial(d, e, g, k);
            double s1 = 0.0;
            for (int i = 0; i < k; ++i) {
                sig[i] = fabs(d[i]);
                cv[i] = g[i];
                s1 = fmax(s1, sig[i]);
            }
            cv[k] = g[k];
            misc[8] = s1;
        }
    }
    __syncthreads();
    const double s1 = misc[8];

    // ---------------- features of the projected problem (learned lambda rule; training data):
    // k / K, then for the 32 largest sigma_i log10(sigma_i / sigma_1) (pad -16) and |c_i| / beta
    // (pad 0), |c_{k+1}| / beta, log10 sigma_1, log10 beta, zeros to 80 entries
    float *feat = reinterpret_cast<float *>(red);    // red is free until the lambda search
    float *hbuf = feat + mlp::kIn;                   // 128 floats of network scratch
    const bool learned = P.rule == CT_LAMBDA_LEARNED && P.net != nullptr;
    if (P.features || learned) {
        if (!fast && tid == 0) {
            // the exact path leaves sigma unsorted: order (sigma_i, c_i) by decreasing sigma
            for (int i = 1; i < k; ++i) {
                const double sv = sig[i], cw = cv[i];
                int j = i - 1;
                while (j >= 0 && sig[j] < sv) { sig[j + 1] = sig[j]; cv[j + 1] = cv[j]; --j; }
                sig[j + 1] = sv;
                cv[j + 1] = cw;
            }
        }
        __syncthreads();
        const bool ok = s1 > 0.0 && beta > 0.0;
        for (int i = tid; i < mlp::kIn; i += kSSThreads) {
            float v = 0.f;
            if (ok) {
                if (i == 0) v = (float)((double)k / (double)P.kmax);
                else if (i <= 32) v = (i - 1 < k) ? (float)fmax(log10(sig[i - 1] / s1), -16.0) : -16.f;
                else if (i <= 64) v = (i - 33 < k) ? (float)(fabs(cv[i - 33]) / beta) : 0.f;
                else if (i == 65) v = (float)(fabs(cv[k]) / beta);
                else if (i == 66) v = (float)log10(s1);
                else if (i == 67) v = (float)log10(beta);
            }
            feat[i] = v;
            if (P.features) P.features[(size_t)(k - 1) * mlp::kIn + i] = v;
        }
        __syncthreads();
    }

    // ---------------- lambda
    // rho^2(lambda) and trace(lambda) are evaluated by the whole block: threads 0-127 take
    // lambda_A, 128-255 lambda_B, one term each (k <= 160 < 2 * 128)
    double *sig2 = rot;                  // sigma_i^2 (rot is free after the cluster pass)
    for (int i = tid; i < k; i += kSSThreads) sig2[i] = sig[i] * sig[i];
    __syncthreads();
    auto eval2 = [&](double lamA, double lamB, double &rA, double &tA, double &rB, double &tB) {
        const int half = tid >> 7, t = tid & 127;
        const double l2 = half ? lamB * lamB : lamA * lamA;
        double r = 0.0, tr = 0.0;
        for (int i = t; i < k; i += 128) {
            const double inv = rcp64(sig2[i] + l2);
            double fc = l2 * inv * cv[i];
            r += fc * fc;
            tr += sig2[i] * inv;
        }
        r = warp_sum_d(r);
        tr = warp_sum_d(tr);
        __syncthreads();                                 // misc[16..31] free from earlier use
        if (lane == 0) { misc[16 + 2 * warp] = r; misc[17 + 2 * warp] = tr; }
        __syncthreads();
        double s0 = 0, s1_ = 0, s2_ = 0, s3 = 0;
        for (int w = 0; w < 4; ++w) {
            s0 += misc[16 + 2 * w]; s1_ += misc[17 + 2 * w];
            s2_ += misc[24 + 2 * w]; s3 += misc[25 + 2 * w];
        }
        const double ck = cv[k] * cv[k];
        rA = s0 + ck; tA = (double)(k + 1) - s1_;
        rB = s2_ + ck; tB = (double)(k + 1) - s3;
    };
    bool have_lam = true;
    if (P.rule == CT_LAMBDA_FIXED) {
        lam = P.lambda_fixed;
    } else if (!(s1 > 0.0)) {
        lam = 0.0;
    } else if (learned) {
        // the network's output is log10(lambda / sigma_1), kept inside the GCV search range;
        // a non-finite output falls back to GCV
        if (warp == 0) {
            const float o = mlp::infer_row_bf16(P.net, feat, hbuf);
            if (lane == 0) misc[14] = (double)o;
        }
        __syncthreads();
        const double o = misc[14];
        if (isfinite(o)) {
            lam = s1 * pow(10.0, fmin(fmax(o, -8.0), 0.0));
        } else {
            have_lam = false;
            if (tid == 0 && P.path) *P.path |= 2;
        }
    } else {
        have_lam = false;
    }
    if (have_lam) {
    } else if (P.rule == CT_LAMBDA_LCURVE) {
        // L-curve corner (Sec. 3.1): maximum curvature of (log ||H y - beta e1||, log ||y||).
        // With inv_i = 1/(sigma_i^2 + lambda^2): eta = ||y||^2 = sum (sigma_i c_i inv_i)^2,
        // rho = sum (lambda^2 c_i inv_i)^2 + c_{k+1}^2, eta' = -4 lambda D with
        // D = sum sigma_i^2 c_i^2 inv_i^3, and the curvature of the log-log curve is
        //   kappa = eta rho (eta rho - 2 lambda^2 D (rho + lambda^2 eta))
        //           / (D (lambda^4 eta^2 + rho^2)^(3/2)).
        auto kappa = [&](double l, double eta, double rho, double D) {
            if (!(eta > 0.0) || !(rho > 0.0) || !(D > 0.0)) return 0.0;
            const double l2 = l * l;
            const double q = l2 * l2 * eta * eta + rho * rho;
            return eta * rho * (eta * rho - 2.0 * l2 * D * (rho + l2 * eta)) / (D * q * sqrt(q));
        };
        auto gridlam = [&](int t) {
            double expo = (t == kGcvGrid - 1) ? 0.0 : -8.0 + t * (8.0 / (kGcvGrid - 1));
            return s1 * pow(10.0, expo);
        };
        const double ck2 = cv[k] * cv[k];
        for (int t = tid; t < kGcvGrid; t += kSSThreads) {
            const double lt = gridlam(t), l2 = lt * lt;
            double eta = 0.0, rho = 0.0, D = 0.0;
            for (int i = 0; i < k; ++i) {
                const double inv = rcp64(sig2[i] + l2);
                const double a = sig[i] * cv[i] * inv;
                const double r = l2 * cv[i] * inv;
                eta += a * a;
                rho += r * r;
                D += a * a * inv;
            }
            red[t] = kappa(lt, eta, rho + ck2, D);
        }
        __syncthreads();
        if (tid == 0) {
            int ibest = 0;
            double best = red[0];
            for (int t = 1; t < kGcvGrid; ++t)
                if (red[t] > best) { best = red[t]; ibest = t; }
            misc[12] = (double)ibest;
            misc[13] = best;
        }
        __syncthreads();
        const int ibest = (int)misc[12];
        const double kbest = misc[13];
        // two lambdas per block pass: threads 0-127 take lamA, 128-255 lamB
        auto evalk2 = [&](double lamA, double lamB, double &kA, double &kB) {
            const int half = tid >> 7, t = tid & 127;
            const double l = half ? lamB : lamA, l2 = l * l;
            double eta = 0.0, rho = 0.0, D = 0.0;
            for (int i = t; i < k; i += 128) {
                const double inv = rcp64(sig2[i] + l2);
                const double a = sig[i] * cv[i] * inv;
                const double r = l2 * cv[i] * inv;
                eta += a * a;
                rho += r * r;
                D += a * a * inv;
            }
            eta = warp_sum_d(eta);
            rho = warp_sum_d(rho);
            D = warp_sum_d(D);
            __syncthreads();
            if (lane == 0) {
                misc[16 + 3 * warp] = eta;
                misc[17 + 3 * warp] = rho;
                misc[18 + 3 * warp] = D;
            }
            __syncthreads();
            double e0 = 0, r0 = 0, d0 = 0, e1 = 0, r1 = 0, d1 = 0;
            for (int w = 0; w < 4; ++w) {
                e0 += misc[16 + 3 * w]; r0 += misc[17 + 3 * w]; d0 += misc[18 + 3 * w];
                e1 += misc[28 + 3 * w]; r1 += misc[29 + 3 * w]; d1 += misc[30 + 3 * w];
            }
            kA = kappa(lamA, e0, r0 + ck2, d0);
            kB = kappa(lamB, e1, r1 + ck2, d1);
        };
        double a = log(gridlam(ibest > 0 ? ibest - 1 : 0));
        double b = log(gridlam(ibest < kGcvGrid - 1 ? ibest + 1 : kGcvGrid - 1));
        const double invphi = 0.6180339887498949;
        for (int it = 0; it < 40; ++it) {
            const double x1 = b - invphi * (b - a), x2 = a + invphi * (b - a);
            double k1, k2;
            evalk2(exp(x1), exp(x2), k1, k2);
            if (k1 >= k2) b = x2; else a = x1;
        }
        double lr = exp(0.5 * (a + b)), kr, kdum;
        evalk2(lr, lr, kr, kdum);
        if (kr < kbest) lr = gridlam(ibest);
        lam = lr;
    } else if (P.rule != CT_LAMBDA_DP) {   // GCV, and the learned rule's fallback
        for (int t = tid; t < kGcvGrid; t += kSSThreads) {
            double expo = (t == kGcvGrid - 1) ? 0.0 : -8.0 + t * (8.0 / (kGcvGrid - 1));
            double lt = s1 * pow(10.0, expo);
            double l2 = lt * lt, r = 0.0, tr = 0.0;
            for (int i = 0; i < k; ++i) {
                double s2 = sig2[i];
                double inv = rcp64(s2 + l2);
                double f = l2 * inv;
                r += (f * cv[i]) * (f * cv[i]);
                tr += s2 * inv;
            }
            r += cv[k] * cv[k];
            tr = (double)(k + 1) - tr;
            red[t] = r / (tr * tr);
        }
        __syncthreads();
        if (tid == 0) {
            int ibest = 0;
            double best = red[0];
            for (int t = 1; t < kGcvGrid; ++t)
                if (red[t] < best) { best = red[t]; ibest = t; }
            misc[12] = (double)ibest;
            misc[13] = best;
        }
        __syncthreads();
        const int ibest = (int)misc[12];
        const double gbest = misc[13];
        auto gridlam = [&](int t) {
            double expo = (t == kGcvGrid - 1) ? 0.0 : -8.0 + t * (8.0 / (kGcvGrid - 1));
            return s1 * pow(10.0, expo);
        };
        double a = log(gridlam(ibest > 0 ? ibest - 1 : 0));
        double b = log(gridlam(ibest < kGcvGrid - 1 ? ibest + 1 : kGcvGrid - 1));
        const double invphi = 0.6180339887498949;
        for (int it = 0; it < 40; ++it) {
            double x1 = b - invphi * (b - a), x2 = a + invphi * (b - a);
            double r1, t1, r2, t2_;
            eval2(exp(x1), exp(x2), r1, t1, r2, t2_);
            if (r1 / (t1 * t1) <= r2 / (t2_ * t2_)) b = x2; else a = x1;
        }
        double lr = exp(0.5 * (a + b)), rr, tt, rdum, tdum;
        eval2(lr, lr, rr, tt, rdum, tdum);
        if (rr / (tt * tt) > gbest) lr = gridlam(ibest);
        lam = lr;
    } else {  // CT_LAMBDA_DP
        // the root of rho(lambda) = target in u = log(lambda) on [log(sigma_1 1e-8), log sigma_1]
        // (rho increases with lambda, so the root is unique): safeguarded Newton on
        // rho^2 - target^2, bisecting whenever a step leaves the bracket.  The bracket halves at
        // least at every bisection, so the 60 steps that plain bisection takes bound the
        // iteration, and the root agrees with the bisection's to rounding.  Each step is one
        // block pass in FP64 (about 70 dependent FP64 instructions on GB300, 2-4 us), so
        // Newton's 5-10 passes replace the bisection's 60.
        const double target = P.dp_target;
        double lo = log(s1 * 1e-8), hi = log(s1);
        double rlo, tlo, rhi, thi;
        eval2(exp(lo), exp(hi), rlo, tlo, rhi, thi);
        if (sqrt(rlo) >= target) {
            lam = exp(lo);
        } else if (sqrt(rhi) <= target) {
            lam = exp(hi);
        } else {
            // rho^2 at lambda and its derivative in log(lambda),
            // d rho^2 / d log(lambda) = 4 sum_i (f_i c_i)^2 sigma_i^2 / (sigma_i^2 + lambda^2),
            // f_i = lambda^2 / (sigma_i^2 + lambda^2); the whole block, one term per thread
            auto eval_dp = [&](double l, double &r2, double &dr2) {
                const double l2 = l * l;
                double r = 0.0, dr = 0.0;
                for (int i = tid; i < k; i += kSSThreads) {
                    const double inv = rcp64(sig2[i] + l2);
                    const double fc = l2 * inv * cv[i];
                    r += fc * fc;
                    dr += fc * fc * (sig2[i] * inv);
                }
                r = warp_sum_d(r);
                dr = warp_sum_d(dr);
                __syncthreads();
                if (lane == 0) { misc[16 + 2 * warp] = r; misc[17 + 2 * warp] = dr; }
                __syncthreads();
                double sr = 0.0, sd = 0.0;
                for (int w = 0; w < nwarps; ++w) { sr += misc[16 + 2 * w]; sd += misc[17 + 2 * w]; }
                r2 = sr + cv[k] * cv[k];
                dr2 = 4.0 * sd;
            };
            const double t2g = target * target;
            double u = 0.5 * (lo + hi), fprev = 1e300;
            for (int it = 0; it < 60; ++it) {
                double r2, dr2;
                eval_dp(exp(u), r2, dr2);
                const double f = r2 - t2g;
                // u is the root to the rounding of rho^2 (the oracle's bisection ends inside the
                // same interval of u, |du| <= 1e-14 target^2 / (d rho^2 / du))
                if (fabs(f) <= 1e-14 * t2g) break;
                if (f < 0.0) lo = u; else hi = u;
                // Newton, or bisection where the step leaves the bracket or |f| did not halve
                double nu = (dr2 > 0.0) ? u - f / dr2 : 0.5 * (lo + hi);
                if (!(nu > lo && nu < hi) || fabs(f) > 0.5 * fprev) nu = 0.5 * (lo + hi);
                fprev = fabs(f);
                const double step = fabs(nu - u);
                u = nu;
                if (step <= 1e-14 * fmax(1.0, fabs(u)) || hi - lo <= 1e-14 * fmax(1.0, fabs(u)))
                    break;
            }
            lam = exp(u);
        }
    }

    // ---------------- projected residual and y
    {
        double r, t, rd, td;
        eval2(lam, lam, r, t, rd, td);
        if (tid == 0) misc[11] = r;
    }
    __syncthreads();
    if (need_y) {
        if (tid == 0) {
            if (fast) {
                // min || Bd z - beta e1 ||^2 + lambda^2 ||z||^2 for the (k+1) x k lower
                // bidiagonal (alpha = d, beta_{i+1} = e[i]): per column one rotation removes the
                // lambda row, one the subdiagonal beta (the damped Golub-Kahan QR), then back
                // substitution on the upper bidiagonal (rho = dsv, theta = esv, rhs z)
                double rb = d[0], phib = beta;
                for (int i = 0; i < k; ++i) {
                    double c1, s1r, r;
                    givens(rb, lam, c1, s1r, r);
                    const double ph = c1 * phib;
                    double cc, ss, rr;
                    givens(r, e[i], cc, ss, rr);
                    dsv[i] = rr;
                    z[i] = cc * ph;
                    if (i + 1 < k) { esv[i] = ss * d[i + 1]; rb = cc * d[i + 1]; }
                    else esv[i] = 0.0;
                    phib = -ss * ph;
                }
            } else {
                // Elden: eliminate lambda I of [Bd; lambda I] (upper bidiagonal) with 2k rotations
                double mu = lam, rr = 0.0;
                for (int i = 0; i < k; ++i) {
                    double a = dsv[i], b = (i < k - 1) ? esv[i] : 0.0, gi = gsv[i];
                    double c, s, r;
                    givens(a, mu, c, s, r);
                    dsv[i] = r;
                    esv[i] = c * b;
                    z[i] = c * gi + s * rr;
                    double f = -s * b;
                    double t = -s * gi + c * rr;
                    if (i < k - 1) {
                        double c2, s2, r2;
                        givens(lam, f, c2, s2, r2);
                        mu = r2;
                        rr = s2 * t;
                    }
                }
            }
            for (int i = k - 1; i >= 0; --i) {
                double num = z[i] - ((i < k - 1) ? esv[i] * z[i + 1] : 0.0);
                z[i] = (dsv[i] != 0.0) ? num * rcp64(dsv[i]) : 0.0;
            }
        }
        __syncthreads();
        // y = Q z with the stored right reflectors: fast-path reflector j acts on coordinates
        // j..k-1 (vector in row j of A), the exact path's on j+1..k-1 (row j, columns j+2..)
        if (warp == 0) {
            const int first = fast ? k - 1 : k - 3;
            for (int j = first; j >= 0; --j) {
                const double tau = tauR[j];
                if (tau == 0.0) continue;
                const int c0 = fast ? j : j + 1;
                const double zj = z[c0];
                double w = 0.0;
                for (int l = c0 + 1 + lane; l < k; l += 32) w += A[l * lda + j] * z[l];
                w = (warp_sum_d(w) + zj) * tau;
                __syncwarp();
                if (lane == 0) z[c0] -= w;
                for (int l = c0 + 1 + lane; l < k; l += 32) z[l] -= w * A[l * lda + j];
                __syncwarp();
            }
        }
        __syncthreads();
        for (int i = tid; i < k; i += kSSThreads) P.y[i] = z[i];
    }
    if (tid == 0) {
        *P.lambda_out = lam;
        *P.resid_out = sqrt(misc[11]);
    }
}

static cudaError_t set_smem_attr();

cudaError_t launch_small_solve(const SmallSolveParams &p, cudaStream_t s)
{
    size_t smem = small_solve_smem_bytes(p.k);
    cudaError_t e = set_smem_attr();
    if (e != cudaSuccess) return e;
    small_solve_kernel<<<1, kSSThreads, smem, s>>>(p, 0);
    return cudaGetLastError();
}

static cudaError_t set_smem_attr()
{
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        e = cudaFuncSetAttribute(small_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)small_solve_smem_bytes(kMaxSmallK));
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    return cudaSuccess;
}

cudaError_t small_solve_prepare() { return set_smem_attr(); }

cudaError_t launch_small_solve_batched(const SmallSolveParams &p, cudaStream_t s)
{
    cudaError_t e = set_smem_attr();
    if (e != cudaSuccess) return e;
    if (p.k < 1) return cudaSuccess;
    // at most one CTA per SM: the FP64 pipe (two lanes per clock per SM on GB300) is the bound,
    // so two projected problems sharing an SM would each run at half speed
    const size_t smem = std::max(small_solve_smem_bytes(p.kfirst + p.k), (size_t)(116 * 1024));
    small_solve_kernel<<<p.k, kSSThreads, smem, s>>>(p, 1);
    return cudaGetLastError();
}

// rule 1: discrepancy principle, rho_k <= target; rule 2: residual norm stagnation,
// |rho_{k-1} - rho_k| < tol rho_{k-1} (k >= 2)
__global__ void stop_check_kernel(const double *__restrict__ res, int k0, int k1, int rule,
                                  double target, double tol, int *stop)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (stop[0] != 0) return;
    for (int k = k0 + 1; k <= k1; ++k) {
        bool hit = false;
        if (rule == CT_STOP_DP) hit = res[k - 1] <= target;
        else if (rule == CT_STOP_RNS && k >= 2) hit = fabs(res[k - 2] - res[k - 1]) < tol * res[k - 2];
        if (hit) {
            stop[1] = CT_OK;
            stop[0] = k;
            return;
        }
    }
}

cudaError_t launch_stop_check(const double *res, int k0, int k1, int rule, double target,
                              double tol, int *stop, cudaStream_t s)
{
    stop_check_kernel<<<1, 32, 0, s>>>(res, k0, k1, rule, target, tol, stop);
    return cudaGetLastError();
}

}  // namespace ct
