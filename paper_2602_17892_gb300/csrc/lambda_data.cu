// Training labels of the learned lambda rule (not in the paper).
//
// For a hybrid AB-GMRES solve with u0 = 0 the iterate of step k at parameter lambda is
// x_k(lambda) = B W_k y_k(lambda) = Z_k y_k(lambda), Z = B W.  With x_true known,
//     ||x_k(lambda) - x_true||^2 = y^T G_k y - 2 g_k^T y + ||x_true||^2,
// G = Z^T Z and g = Z^T x_true (leading k x k block and k entries for step k).  Writing
// H_k = U diag(sigma) V^T, the Tikhonov solution of Eq. (hybrid_proj) is y = V f with
// f_j = sigma_j c_j / (sigma_j^2 + lambda^2) and sigma_j c_j = beta (H_k V)_{1j}, so the error is
// f^T (V^T G_k V) f - 2 (V^T g_k)^T f + const, O(k^2) per lambda once V is known.
//
// gram_kernel forms G and g in FP64 (one CTA per entry, fixed-order reduction).
// lambda_label_kernel takes one warp per step k: one-sided Jacobi SVD of H_k in FP64
// (Hestenes; round-robin pairs, one pair per lane), then the GCV-style search of lambda over
// 256 log-spaced points on [1e-8 sigma_1, sigma_1] and 40 golden-section steps in log lambda.
#include "ct_internal.h"

namespace ct {

constexpr int kGramThreads = 256;

// blockIdx.x = i, blockIdx.y = j: G[i][j] = <z_i, z_j> for i <= j < K (mirrored), and for
// j == K: g[i] = <z_i, x_true>.  Z column i at Z + i * ldz (n floats).
__global__ void __launch_bounds__(kGramThreads) gram_kernel(const float *__restrict__ Z,
                                                            int64_t ldz, int64_t n, int K,
                                                            const float *__restrict__ xt,
                                                            double *__restrict__ G,
                                                            double *__restrict__ gv)
{
    const int i = blockIdx.x, j = blockIdx.y;
    if (j < K && j < i) return;
    const float *a = Z + (int64_t)i * ldz;
    const float *b = (j < K) ? Z + (int64_t)j * ldz : xt;
    double s = 0.0;
    for (int64_t t = threadIdx.x; t < n; t += kGramThreads) s += (double)a[t] * (double)b[t];
    __shared__ double red[kGramThreads];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kGramThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (j == K) {
            gv[i] = red[0];
        } else {
            G[(int64_t)j * K + i] = red[0];
            G[(int64_t)i * K + j] = red[0];
        }
    }
}

__device__ __forceinline__ double warp_sum_ld(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max_ld(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

constexpr int kLabelMaxK = 64;

size_t label_smem_bytes(int K)
{
    return ((size_t)(K + 1) * K + 2 * (size_t)K * K + 4 * (size_t)K) * sizeof(double);
}

// Block b (32 threads) labels step k = b + 1.  H: FP64 column-major, leading dimension ldh;
// G: K x K column-major; gv: K entries.
__global__ void __launch_bounds__(32) lambda_label_kernel(const double *__restrict__ H, int ldh,
                                                          const double *__restrict__ betap,
                                                          const double *__restrict__ G, int K,
                                                          const double *__restrict__ gv,
                                                          float *__restrict__ labels)
{
    const int k = blockIdx.x + 1, lane = threadIdx.x;
    extern __shared__ double sm[];
    const int ldm = k + 1;
    double *M = sm;                    // (k+1) x k: H_k, rotated into U diag(sigma)
    double *V = M + (size_t)ldm * k;   // k x k, column-major
    double *Gt = V + (size_t)k * k;    // V^T G_k V
    double *sg = Gt + (size_t)k * k;   // sigma_j
    double *sc = sg + k;               // sigma_j c_j = beta (H_k V)_{1j}
    double *gt = sc + k;               // V^T g_k
    double *f = gt + k;
    double *T = M;                     // G_k V (M is free once sigma and sc are taken)
    const double beta = *betap;

    for (int t = lane; t < ldm * k; t += 32) {
        const int c = t / ldm, r = t - c * ldm;
        M[t] = H[(size_t)c * ldh + r];
    }
    for (int t = lane; t < k * k; t += 32) V[t] = (t / k == t % k) ? 1.0 : 0.0;
    __syncwarp();

    // one-sided Jacobi: rotate column pairs (p, q) of M until all are orthogonal; pairs follow
    // the circle schedule (player kk-1 fixed), so the pairs of one round are disjoint
    const int kk = k + (k & 1);
    for (int sweep = 0; sweep < 60 && k > 1; ++sweep) {
        int rotated = 0;
        for (int r = 0; r < kk - 1; ++r) {
            for (int pi = lane; pi < kk / 2; pi += 32) {
                int p, q;
                if (pi == 0) { p = kk - 1; q = r; }
                else { p = (r + pi) % (kk - 1); q = (r - pi + kk - 1) % (kk - 1); }
                if (p >= k || q >= k) continue;
                double a = 0.0, b = 0.0, c = 0.0;
                for (int i = 0; i <= k; ++i) {
                    const double x = M[p * ldm + i], y = M[q * ldm + i];
                    a += x * x; b += y * y; c += x * y;
                }
                if (c != 0.0 && fabs(c) > 1e-13 * sqrt(a * b)) {
                    const double zeta = (b - a) / (2.0 * c);
                    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                    for (int i = 0; i <= k; ++i) {
                        const double x = M[p * ldm + i], y = M[q * ldm + i];
                        M[p * ldm + i] = cs * x - sn * y;
                        M[q * ldm + i] = sn * x + cs * y;
                    }
                    for (int i = 0; i < k; ++i) {
                        const double x = V[p * k + i], y = V[q * k + i];
                        V[p * k + i] = cs * x - sn * y;
                        V[q * k + i] = sn * x + cs * y;
                    }
                    rotated = 1;
                }
            }
            __syncwarp();
        }
        if (!__any_sync(0xffffffffu, rotated)) break;
    }
    double smax = 0.0;
    for (int j = lane; j < k; j += 32) {
        double s2 = 0.0;
        for (int i = 0; i <= k; ++i) s2 += M[j * ldm + i] * M[j * ldm + i];
        sg[j] = sqrt(s2);
        sc[j] = beta * M[j * ldm];
        smax = fmax(smax, sg[j]);
    }
    const double s1 = warp_max_ld(smax);
    __syncwarp();
    if (!(s1 > 0.0)) {
        if (lane == 0) labels[k - 1] = __int_as_float(0x7fc00000);   // NaN
        return;
    }
    // T = G_k V, Gt = V^T T, gt = V^T g_k
    for (int t = lane; t < k * k; t += 32) {
        const int j = t / k, i = t - j * k;
        double s = 0.0;
        for (int l = 0; l < k; ++l) s += G[(size_t)l * K + i] * V[j * k + l];
        T[t] = s;
    }
    __syncwarp();
    for (int t = lane; t < k * k; t += 32) {
        const int j = t / k, i = t - j * k;
        double s = 0.0;
        for (int l = 0; l < k; ++l) s += V[i * k + l] * T[j * k + l];
        Gt[t] = s;
    }
    for (int i = lane; i < k; i += 32) {
        double s = 0.0;
        for (int l = 0; l < k; ++l) s += V[i * k + l] * gv[l];
        gt[i] = s;
    }
    __syncwarp();
    // error(lambda) - ||x_true||^2 = f^T Gt f - 2 gt^T f
    auto err = [&](double lam) {
        const double l2 = lam * lam;
        for (int j = lane; j < k; j += 32) f[j] = sc[j] / (sg[j] * sg[j] + l2);
        __syncwarp();
        double acc = 0.0;
        for (int i = lane; i < k; i += 32) {
            double r = 0.0;
            for (int j = 0; j < k; ++j) r += Gt[j * k + i] * f[j];
            acc += f[i] * (r - 2.0 * gt[i]);
        }
        acc = warp_sum_ld(acc);
        __syncwarp();
        return acc;
    };
    auto gridlam = [&](int t) {
        const double expo = (t == 255) ? 0.0 : -8.0 + t * (8.0 / 255.0);
        return s1 * pow(10.0, expo);
    };
    int ibest = 0;
    double best = err(gridlam(0));
    for (int t = 1; t < 256; ++t) {
        const double e = err(gridlam(t));
        if (e < best) { best = e; ibest = t; }
    }
    double a = log(gridlam(ibest > 0 ? ibest - 1 : 0));
    double b = log(gridlam(ibest < 255 ? ibest + 1 : 255));
    const double invphi = 0.6180339887498949;
    for (int it = 0; it < 40; ++it) {
        const double x1 = b - invphi * (b - a), x2 = a + invphi * (b - a);
        if (err(exp(x1)) <= err(exp(x2))) b = x2; else a = x1;
    }
    double lam = exp(0.5 * (a + b));
    if (err(lam) > best) lam = gridlam(ibest);
    if (lane == 0) labels[k - 1] = (float)log10(lam / s1);
}

cudaError_t launch_gram(const float *Z, int64_t ldz, int64_t n, int K, const float *xt,
                        double *G, double *gv, cudaStream_t s)
{
    gram_kernel<<<dim3(K, K + 1), kGramThreads, 0, s>>>(Z, ldz, n, K, xt, G, gv);
    return cudaGetLastError();
}

cudaError_t launch_lambda_labels(const double *H, int ldh, const double *betap, const double *G,
                                 int K, const double *gv, float *labels, cudaStream_t s)
{
    if (K < 1 || K > kLabelMaxK) return cudaErrorInvalidValue;
    const size_t smem = label_smem_bytes(K);
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        e = cudaFuncSetAttribute(lambda_label_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)label_smem_bytes(kLabelMaxK));
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    lambda_label_kernel<<<K, 32, smem, s>>>(H, ldh, betap, G, K, gv, labels);
    return cudaGetLastError();
}

}  // namespace ct
