// The hybrid step of Algorithms 1 and 2 (lines 12-13) on the device, in FP64:
// choose lambda for the (k+1) x k Hessenberg matrix H_k and solve Eq. (hybrid_proj)
//     y = argmin || [H_k; lambda I] y - beta [e1; 0] ||.
//
// lambda = 0 (plain AB/BA-GMRES, Eq. (proj_pbm)): Givens QR of H_k and back substitution.
// lambda > 0: Householder bidiagonalisation P^T H_k Q = [Bd; 0] (Bd upper bidiagonal),
// g = P^T beta e1; implicit-shift Golub-Kahan QR on Bd gives the singular values sigma_i and,
// through the left rotations applied to g, the coordinates c = U^T beta e1 that GCV (Sec. 3.1)
// and the discrepancy principle (Sec. 3.2) need:
//     rho^2(lambda) = sum_i (lambda^2 c_i / (sigma_i^2 + lambda^2))^2 + c_{k+1}^2,
//     trace(I - H H_lambda) = (k+1) - sum_i sigma_i^2 / (sigma_i^2 + lambda^2).
// y follows from the bidiagonal Tikhonov problem min ||Bd z - g||^2 + lambda^2 ||z||^2,
// eliminated with 2k Givens rotations (O(k)), and y = Q z (stored right reflectors).
//
// Parameter readings shared with the FP64 CPU oracle: GCV is evaluated on 256 log-spaced
// lambda in [sigma_1 1e-8, sigma_1], the first grid minimum is refined by 40 golden-section
// steps in log lambda on the neighbouring bracket (kept only if not worse); DP solves
// rho(lambda) = tau ||e|| by 60 bisection steps in log lambda over the same range.
#include "ct_internal.h"

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
    r = hypot(a, b);
    c = a / r;
    s = b / r;
}

// Householder vector (LAPACK dlarfg convention): returns beta, tau; x scaled in place so that
// H = I - tau [1; x][1; x]^T maps [alpha; x] to [beta; 0].
__device__ void make_reflector(double alpha, double xnorm2, double &beta, double &tau, double &scale)
{
    if (xnorm2 == 0.0) { beta = alpha; tau = 0.0; scale = 0.0; return; }
    double nrm = sqrt(alpha * alpha + xnorm2);
    beta = (alpha >= 0.0) ? -nrm : nrm;
    tau = (beta - alpha) / beta;
    scale = 1.0 / (alpha - beta);
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
        // a zero on the diagonal of the block: split with rotations
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
        // Wilkinson shift from the trailing 2x2 of Bd^T Bd
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

size_t small_solve_smem_bytes(int k)
{
    size_t nd = (size_t)(k + 1) * k + 12 * (size_t)(k + 1) + kGcvGrid + 64;
    return nd * sizeof(double);
}

__global__ void __launch_bounds__(kSSThreads) small_solve_kernel(SmallSolveParams P)
{
    const int k = P.k;
    if (P.stop) {
        int st = P.stop[0];
        if (st < 0 || (st > 0 && k > st)) return;
    }
    extern __shared__ double sd[];
    const int lda = k + 1;
    double *A = sd;                       // (k+1) x k, column-major
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
    double *rot = z + (k + 1);            // 2(k+1): Givens c, s
    double *red = rot + 2 * (k + 1);      // kGcvGrid
    double *misc = red + kGcvGrid;        // 64
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = kSSThreads / 32;
    const double beta = P.betap ? *P.betap : P.beta;

    for (int t = tid; t < lda * k; t += kSSThreads) {
        int c = t / lda, r = t - c * lda;
        A[t] = P.H[(size_t)c * P.ldh + r];
    }
    for (int t = tid; t <= k; t += kSSThreads) g[t] = (t == 0) ? beta : 0.0;
    __syncthreads();

    double lam = 0.0, rho2 = 0.0;
    if (P.rule == CT_LAMBDA_NONE) {
        // ---------------- Givens QR of H_k, back substitution (Eq. (proj_pbm))
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
        for (int i = k - 1; i >= 0; --i) {   // column-oriented back substitution
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
            rho2 = g[k] * g[k];
            *P.lambda_out = 0.0;
            *P.resid_out = fabs(g[k]);
        }
        return;
    }

    // ---------------- Householder bidiagonalisation of H_k ((k+1) x k)
    for (int j = 0; j < k; ++j) {
        // left reflector on column j, rows j..k
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
            // apply to columns j+1..k-1 and to g (index k as an extra column)
            if (tau != 0.0) {
                for (int l = j + 1 + warp; l <= k; l += nwarps) {
                    double *col = (l < k) ? A + (size_t)l * lda : g;
                    const double cj = col[j];
                    double w = 0.0;
                    for (int i = j + 1 + lane; i <= k; i += 32) w += A[j * lda + i] * col[i];
                    w = warp_sum_d(w) + cj;
                    w *= tau;
                    if (lane == 0) col[j] -= w;
                    for (int i = j + 1 + lane; i <= k; i += 32) col[i] -= w * A[j * lda + i];
                }
            }
        }
        __syncthreads();
        // right reflector on row j, columns j+1..k-1
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
                    w = warp_sum_d(w) + ai;
                    w *= tau;
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

    // ---------------- singular values and c = U^T g (one thread)
    if (tid == 0) {
        int st = bidiag_svd_serial(d, e, g, k);
        double s1 = 0.0;
        for (int i = 0; i < k; ++i) {
            sig[i] = fabs(d[i]);
            cv[i] = g[i];
            s1 = fmax(s1, sig[i]);
        }
        cv[k] = g[k];
        misc[8] = s1;
        misc[9] = (double)st;
    }
    __syncthreads();
    const double s1 = misc[8];

    // ---------------- lambda
    if (P.rule == CT_LAMBDA_FIXED) {
        lam = P.lambda_fixed;
    } else if (s1 == 0.0) {
        lam = 0.0;
    } else if (P.rule == CT_LAMBDA_GCV) {
        // grid: lambda_t = s1 10^(-8 + 8 t / 255)
        for (int t = tid; t < kGcvGrid; t += kSSThreads) {
            double expo = -8.0 + t * (8.0 / (kGcvGrid - 1));
            if (t == kGcvGrid - 1) expo = 0.0;
            double lt = s1 * pow(10.0, expo);
            double l2 = lt * lt, r = 0.0, tr = 0.0;
            for (int i = 0; i < k; ++i) {
                double s2 = sig[i] * sig[i];
                double f = l2 / (s2 + l2);
                r += (f * cv[i]) * (f * cv[i]);
                tr += s2 / (s2 + l2);
            }
            r += cv[k] * cv[k];
            tr = (double)(k + 1) - tr;
            red[t] = r / (tr * tr);
        }
        __syncthreads();
        if (warp == 0) {
            int ibest = 0;
            if (lane == 0) {
                double best = red[0];
                for (int t = 1; t < kGcvGrid; ++t)
                    if (red[t] < best) { best = red[t]; ibest = t; }
            }
            ibest = __shfl_sync(0xffffffffu, ibest, 0);
            const double gbest = red[ibest];
            auto gridlog = [&](int t) {
                double expo = (t == kGcvGrid - 1) ? 0.0 : -8.0 + t * (8.0 / (kGcvGrid - 1));
                return log(s1 * pow(10.0, expo));
            };
            double a = gridlog(ibest > 0 ? ibest - 1 : 0);
            double b = gridlog(ibest < kGcvGrid - 1 ? ibest + 1 : kGcvGrid - 1);
            const double invphi = 0.6180339887498949;
            for (int it = 0; it < 40; ++it) {
                double x1 = b - invphi * (b - a), x2 = a + invphi * (b - a);
                double r1, t1, r2, t2;
                eval_lambda_warp(exp(x1), sig, cv, k, r1, t1);
                eval_lambda_warp(exp(x2), sig, cv, k, r2, t2);
                if (r1 / (t1 * t1) <= r2 / (t2 * t2)) b = x2; else a = x1;
            }
            double lr = exp(0.5 * (a + b)), rr, tt;
            eval_lambda_warp(lr, sig, cv, k, rr, tt);
            if (rr / (tt * tt) > gbest) {
                double expo = (ibest == kGcvGrid - 1) ? 0.0 : -8.0 + ibest * (8.0 / (kGcvGrid - 1));
                lr = s1 * pow(10.0, expo);
            }
            if (lane == 0) misc[10] = lr;
        }
        __syncthreads();
        lam = misc[10];
    } else {  // CT_LAMBDA_DP
        if (warp == 0) {
            const double target = P.dp_target;
            double lo = log(s1 * 1e-8), hi = log(s1);
            double r, t, out;
            eval_lambda_warp(exp(lo), sig, cv, k, r, t);
            if (sqrt(r) >= target) {
                out = exp(lo);
            } else {
                eval_lambda_warp(exp(hi), sig, cv, k, r, t);
                if (sqrt(r) <= target) {
                    out = exp(hi);
                } else {
                    for (int it = 0; it < 60; ++it) {
                        double mid = 0.5 * (lo + hi);
                        eval_lambda_warp(exp(mid), sig, cv, k, r, t);
                        if (sqrt(r) < target) lo = mid; else hi = mid;
                    }
                    out = exp(0.5 * (lo + hi));
                }
            }
            if (lane == 0) misc[10] = out;
        }
        __syncthreads();
        lam = misc[10];
    }

    // ---------------- projected residual and y
    if (warp == 0) {
        double r, t;
        eval_lambda_warp(lam, sig, cv, k, r, t);
        if (lane == 0) misc[11] = r;
    }
    if (tid == 0) {
        // Elden: eliminate the lambda I block of [Bd; lambda I] with 2k Givens rotations
        double mu = lam, rr = 0.0;   // current lambda-row entry and its right-hand side
        for (int i = 0; i < k; ++i) {
            double a = dsv[i], b = (i < k - 1) ? esv[i] : 0.0, gi = gsv[i];
            double c, s, r;
            givens(a, mu, c, s, r);
            dsv[i] = r;                 // new diagonal
            esv[i] = c * b;             // new superdiagonal
            z[i] = c * gi + s * rr;     // new right-hand side
            double f = -s * b;          // fill in the lambda row at column i+1
            double t = -s * gi + c * rr;
            if (i < k - 1) {
                double c2, s2, r2;
                givens(lam, f, c2, s2, r2);
                mu = r2;
                rr = s2 * t;
            }
        }
        for (int i = k - 1; i >= 0; --i) {
            double num = z[i] - ((i < k - 1) ? esv[i] * z[i + 1] : 0.0);
            z[i] = (dsv[i] != 0.0) ? num / dsv[i] : 0.0;
        }
    }
    __syncthreads();
    // y = Q z: right reflectors j = k-3 .. 0 act on coordinates j+1..k-1
    if (warp == 0) {
        for (int j = k - 3; j >= 0; --j) {
            const double tau = tauR[j];
            if (tau == 0.0) continue;
            const double zj = z[j + 1];
            double w = 0.0;
            for (int l = j + 2 + lane; l < k; l += 32) w += A[l * lda + j] * z[l];
            w = warp_sum_d(w) + zj;
            w *= tau;
            __syncwarp();
            if (lane == 0) z[j + 1] -= w;
            for (int l = j + 2 + lane; l < k; l += 32) z[l] -= w * A[l * lda + j];
            __syncwarp();
        }
    }
    __syncthreads();
    for (int i = tid; i < k; i += kSSThreads) P.y[i] = z[i];
    if (tid == 0) {
        *P.lambda_out = lam;
        *P.resid_out = sqrt(misc[11]);
    }
}

cudaError_t launch_small_solve(const SmallSolveParams &p, cudaStream_t s)
{
    size_t smem = small_solve_smem_bytes(p.k);
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
    small_solve_kernel<<<1, kSSThreads, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace ct
