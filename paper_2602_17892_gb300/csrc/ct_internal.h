// Internal declarations shared by the CUDA translation units of libctabba.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/ctabba.h"

namespace ct {

// ----------------------------------------------------------------------------- errors
void set_error(const std::string &msg);
ct_status cuda_fail(cudaError_t e, const char *what);
#define CT_CUDA(call)                                                        \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return ::ct::cuda_fail(e_, #call);            \
    } while (0)

// ----------------------------------------------------------------------------- geometry
// One Joseph ray in index units, 8 bytes: along the driving axis the sample at integer index t
// lies at fractional index pos = pmid + slope * (t - (n_drive-1)/2) of the other axis.  The
// slope (|slope| <= 1: the driving axis is the ray's longer component) is stored in fixed point,
// round(slope 2^29), shifted left by one with the driving axis (0 = x, 1 = y) in bit 0.  The
// kernels form the FP32 slope, the sample weight h sqrt(1 + slope^2) and the range of t whose
// FP32 positions lie in [-1, n_other] themselves (decode_ray2d), so the table is half the size
// a table of those values would be.
struct __align__(8) Ray2D {
    float pmid;
    int32_t enc;
};

// Per-view constants of the pixel-driven backprojector.
struct __align__(16) ViewBP {
    float cs, sn;   // cos, sin of the view angle
    float a, b;     // parallel: h cos / pitch, h sin / pitch; fan: unused
};

// One (view, detector column u) of a cone geometry.  All rays of the column share their x-y
// projection (the fan ray of that column), so its in-plane Joseph parameters are computed once
// on the host in FP64; the z part depends on the detector row v and is formed per ray.
// D = (detector point - source) in physical units, Da its component on the driving axis.
struct __align__(16) RayXY {
    float bmid, bslope;   // in-plane tap position across the driving axis at its central plane
                          // (index units) and its change per plane
    float dxy2;           // (Dx^2 + Dy^2) / Da^2
    uint32_t packed;      // t_lo (bits 0-14) | t_hi (bits 15-29) | axis (bits 30-31: 0 x, 1 y)
    // the z part in FP32 for the row offset c = iv - (ndv - 1) / 2 (exact in FP32):
    // z slope pitch_v / Da and z at the central plane (nz - 1) / 2 - c pitch_v Sa / (h Da), each
    // factor as an FP32 pair hi + lo of its FP64 value; rows iv in [iv_lo, iv_hi] are driven
    // along x or y (the FP64 test |v| |1 / Da| <= 1, evaluated on the host), the others along z
    float zp_hi, zp_lo, zq_hi, zq_lo;
    int32_t iv_lo, iv_hi, pad0, pad1;
    double rda;           // 1 / Da
    double sa_h;          // source coordinate on the driving axis / h
    double sx_h, sy_h;    // source / h      (rays driven along z)
    double dx, dy;        // Dx, Dy          (rays driven along z)
};

struct DeviceGeom {
    int kind, nx, ny, nz;
    float h;
    int n_views, ndu, ndv;
    float pitch_u, pitch_v, sid, sdd;
    // padded layouts
    int row_pairs_ld;   // P_row row length in float2: >= nx + 3
    int col_pairs_ld;   // P_col row length in float2: >= ny + 3
    int sino_ld;        // padded sinogram row length: ndu + 4 (2 zero bins each side)
    int tune_a_threads; // Joseph A: rays (threads) per block, chosen by ct_geom_autotune
    int tune_a_views;   // 2D Joseph A: views per block (each warp one view)
    int back_adjoint;   // the geometry's backprojector: 0 pixel/voxel-driven B, 1 A^T
    int tune_b_rows;    // pixel-driven B: block of 32 x tune_b_rows pixels
    int tune_b_views;   // 2D pixel-driven B: views per loop iteration (1, or 2 in paired FP32);
                        // 4: the four-fold rotation kernel (b_rot4 geometries only)
    int b_noclamp;      // 2D: every pixel centre projects inside the detector in every view
    int b_rot4;         // fan, square image of even side, views in quadruples 90 degrees apart
                        // (view k + m n/4 at angle theta_k + m pi/2): B may use the rotation
                        // kernel
    int tune_a_slab;    // 3D Joseph A: z slab thickness (tap rows) per launch
    int tune_a_rays;    // 3D Joseph A: detector rows per thread (1, or 2 sharing the in-plane
                        // coordinate)
    int tune_a_wviews;  // 2D Joseph A: views per warp (1, 2, 4, 8; 32 / tune_a_wviews bins each)
    int tune_b_wrows;   // 2D pixel-driven B: pixel (orbit) rows per warp (1, 2, 4)
    int64_t sino_view_ld; // floats per view in the padded sinogram (2D: sino_ld; 3D: (ndv + 2)
                          // rows of sino_ld, detector row 0 at row 1)
    int sino_row0;      // offset of detector row 0 inside a padded view (0 in 2D, sino_ld in 3D)
    int64_t slice_x;    // 3D: pairs per z slice of P_x ((max(nx, ny) + 3) * col_pairs_ld)
    int64_t slice_y;    // 3D: pairs per z slice of P_y ((max(nx, ny) + 3) * row_pairs_ld)
    // tables
    const Ray2D *rays;  // m rays (2D)
    const RayXY *rays_xy; // n_views x ndu (3D)
    const ViewBP *views;
};

}  // namespace ct

struct ct_geom {
    ct_geom_desc desc;
    double *angles_host;
    int64_t n, m;
    int64_t a_samples;   // sum over rays of the clipped Joseph sample counts
    ct::DeviceGeom dg;
    // device allocations owned by the geometry
    ct::Ray2D *rays_dev;
    ct::RayXY *rays_xy_dev;
    ct::ViewBP *views_dev;
    float2 *prow_dev;   // 2D: [ny][row_pairs_ld] pairs along x; 3D: P_y, [nz + 3][slice_y]
    float2 *pcol_dev;   // 2D: [nx][col_pairs_ld] pairs along y; 3D: P_x, [nz + 3][slice_x]
    float *sino_pad_dev;  // [n_views][sino_view_ld]
    float2 *sino_pairs_dev; // [n_views][sino_view_ld] (bin j, bin j + 1 - bin j) pairs read by B
    double *adj_acc_dev;    // n FP64 accumulators of the matched adjoint A^T (2D: from creation;
                            // cone: allocated when the adjoint is first selected)
    // solver workspace (grown on demand)
    struct Workspace *ws;
};

namespace ct {

// Floor by one round-down FP32 addition (projector kernels): for an integer K with
// 2^23 <= K + p < 2^24, K + p rounded towards -infinity is K + floor(p) exactly and its bit
// pattern is the integer 0x4B000000 + (K + floor(p) - 2^23).
constexpr float kFloor2p23 = 8388608.f;   // 2^23
constexpr float kFloorK0 = 8388610.f;     // 2^23 + 2: K + p >= 2^23 for p >= -2
constexpr int kFloorSpan = 1 << 22;       // row (or view) offsets carried in K stay below this
// rows (or views) of `stride` elements per chunk whose offsets K carries
inline int floor_chunk(int64_t stride)
{
    const int64_t s = stride > 0 ? stride : 1;
    return (int)(kFloorSpan / s > 0 ? kFloorSpan / s : 1);
}

// ----------------------------------------------------------------------------- projectors
// Every launcher takes an optional device stop word: when non-null and non-zero at kernel
// start, the kernel returns at once (a solver that met breakdown skips the remaining steps).
// Image x (row-major, n floats) -> the two padded pair layouts used by the Joseph kernels.
cudaError_t launch_image_pairs(const ct_geom *g, const float *x, const int *stop, cudaStream_t s);
// x = A^T y (2D matched adjoint; y with row stride y_ld and bin offset y_off)
cudaError_t launch_adjoint2d(const ct_geom *g, const float *y, int y_ld, int y_off, float *x,
                             const int *stop, cudaStream_t s);
// x = A^T y (cone matched adjoint; y with view stride y_view_ld, row stride y_ld, bin offset
// y_off; acc: n FP64 accumulators)
cudaError_t launch_adjoint3d(const ct_geom *g, const float *y, int64_t y_view_ld, int y_ld,
                             int y_off, double *acc, float *x, const int *stop, cudaStream_t s);
// x[i] = (float)a[i]
cudaError_t launch_round_to_float(const double *a, int64_t n, float *x, const int *stop,
                                  cudaStream_t s);
// y[view][v][u] -> padded sinogram (sino_view_ld floats per view, row length sino_ld, bin u of
// row v at index sino_row0 + v * sino_ld + u + 2).
cudaError_t launch_pad_sino(const ct_geom *g, const float *y, float *ypad, cudaStream_t s);
// y = A x from the pair layouts: padded != 0 writes the padded sinogram layout, else the dense
// [view][v][u] layout.
cudaError_t launch_forward_proj(const ct_geom *g, float *y, bool padded, const int *stop,
                                cudaStream_t s);
// x = B y from a padded sinogram (two launches: the pair layout of y, then B)
cudaError_t launch_back_proj(const ct_geom *g, const float *ypad, float *x, const int *stop,
                             cudaStream_t s);
// kind-specific launchers (2D: proj2d.cu, 3D: proj3d.cu); element (view, v, u) of y at
// view * y_view_ld + v * y_ld + y_off + u
cudaError_t launch_joseph2d(const ct_geom *g, float *y, int y_ld, int y_off, const int *stop,
                            cudaStream_t s);
cudaError_t launch_pixbp2d(const ct_geom *g, const float2 *ypair, float *x, const int *stop,
                           cudaStream_t s);
cudaError_t launch_joseph3d(const ct_geom *g, float *y, int64_t y_view_ld, int y_ld, int y_off,
                            const int *stop, cudaStream_t s);
cudaError_t launch_voxbp3d(const ct_geom *g, const float2 *ypair, float *x, const int *stop,
                           cudaStream_t s);
// kernel launches made by one launch_joseph3d (one per z slab)
int joseph3d_launches(const ct_geom *g);
// total Joseph sample count of a cone geometry (one counting launch, synchronous)
cudaError_t count_joseph3d_samples(const ct_geom *g, int64_t *out);

// ----------------------------------------------------------------------------- Arnoldi
struct ArnoldiScratch {
    double *partial;      // [max_blocks][kmax + 2]
    unsigned *counter;    // block-completion counter (reset by the last block)
    int max_blocks;
    int kmax;
};

// caches the Gram-Schmidt kernels' one-wave grid for the current device (before a capture)
cudaError_t arnoldi_prepare();
// test hook of the bounded TMA waits (see ct_test_drop_tile_copy)
cudaError_t arnoldi_test_drop_tile_copy(int enable, long long wait_cycles);

// ----------------------------------------------------------------------------- small solve
constexpr int kMaxSmallK = 160;   // largest projected problem held in shared memory
struct SmallSolveParams {
    const double *H = nullptr;  int ldh = 0; int k = 0;
    double beta = 0.0; const double *betap = nullptr;   // beta, or read from device when betap != null
    int rule = 0; double lambda_fixed = 0.0; double dp_target = 0.0;
    double *y = nullptr; double *lambda_out = nullptr; double *resid_out = nullptr;
    const int *stop = nullptr;  // solver stop word (may be null)
    int kmax = 0;     // last step of the solve: y is formed there (or at a breakdown step)
    int always_y = 0; // form y at every k
    int *path = nullptr; // optional: 1 where the parallel path was accepted, 0 where the exact
                      // sequential path ran (indexed by k - 1); + 2 where CT_LAMBDA_LEARNED
                      // fell back to GCV
    int ystride = 0;  // batched launch: step k has y at y + (k - 1) * ystride,
                      // lambda_out[k - 1], resid_out[k - 1], path[k - 1]
    const float *net = nullptr;   // CT_LAMBDA_LEARNED: FP32 network parameters (device)
    float *features = nullptr;    // optional: row k - 1 (80 floats) gets the features of H_k
    int kfirst = 0;   // batched launch over k = kfirst + 1 .. kfirst + k (outputs indexed k - 1)
    int only_y = 0;   // batched launch: only the block of the final step (stop[0] when set,
                      // else kmax) runs, and it forms y
    int y_at = 0;     // also form y at this step (the NCP check's iterate)
};
cudaError_t launch_small_solve(const SmallSolveParams &p, cudaStream_t s);
// sets the kernel's shared-memory limit on the current device (call before a stream capture)
cudaError_t small_solve_prepare();
// steps k = p.kfirst + 1 .. p.kfirst + p.k of one solve in one launch (one CTA per k)
cudaError_t launch_small_solve_batched(const SmallSolveParams &p, cudaStream_t s);
// stopping rules (Sec. 3.2) on the residual norms res[k0 .. k1-1] (steps k0+1 .. k1): sets
// stop[0] = the first step that meets the rule (stop[1] = CT_OK) unless stop[0] is already set
cudaError_t launch_stop_check(const double *res, int k0, int k1, int rule, double target,
                              double tol, int *stop, cudaStream_t s);
size_t small_solve_smem_bytes(int k);

// ----------------------------------------------------------------------------- probes
int probe_threads();
int probe_chains();
int probe_blocks_per_sm(int kind);
// kind 0: 8-byte L1 gathers; kind 1: reciprocal + square root pairs; `blocks` x probe_threads()
// threads, each `reps` operations (a multiple of probe_chains()), one float each into out
cudaError_t launch_probe(int kind, int64_t reps, float *out, int blocks, cudaStream_t s);

// ----------------------------------------------------------------------------- NCP stop rule
constexpr int kNcpMaxBins = 8192;   // detector row length the NCP kernels hold in shared memory
size_t ncp_smem_bytes(int n);
cudaError_t ncp_prepare(int n);     // shared-memory limit of the row kernel (before a capture)
// distances[step - 1] = NCP distance of the rows of b - ax (b dense [view][v][u], ax padded);
// stops the solve at `prev` (stop[0] = prev) when the distance grew since that check
cudaError_t launch_ncp_check(const ct_geom *g, const float *b, const float *ax_pad,
                             const float2 *tw, float *part, double *dist, int step, int prev,
                             int *stop, cudaStream_t s);

// ----------------------------------------------------------------------------- learned lambda
// network kernels (mlp.cu): P = FP32 parameter vector, X = n x 80 row-major features
cudaError_t mlp_prepare();
int mlp_num_params();
int mlp_rows_per_block();
cudaError_t launch_mlp_forward(const float *P, const float *X, int n, float *out, bool bf16,
                               cudaStream_t s);
// part: ceil(n / rows_per_block) * num_params floats; lpart: ceil(n / rows_per_block) floats
cudaError_t launch_mlp_grad(const float *P, const float *X, const float *Y, int n, float *part,
                            float *lpart, float *grad, float *loss, bool bf16, cudaStream_t s);
cudaError_t launch_mlp_adam(float *P, const float *G, float *M, float *V, float lr, int t,
                            cudaStream_t s);
// training labels (lambda_data.cu): G = Z^T Z (K x K, FP64) and gv = Z^T x_true for Z = n x K
// (column i at Z + i * ldz); labels[k-1] = log10(lambda*_k / sigma_1(H_k)), K <= 64
cudaError_t launch_gram(const float *Z, int64_t ldz, int64_t n, int K, const float *xt,
                        double *G, double *gv, cudaStream_t s);
cudaError_t launch_lambda_labels(const double *H, int ldh, const double *betap, const double *G,
                                 int K, const double *gv, float *labels, cudaStream_t s);

}  // namespace ct
