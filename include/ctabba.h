/*
 * ctabba — hybrid AB-/BA-GMRES for X-ray CT with an unmatched projector pair, on one
 * NVIDIA GB300 (sm_103a).  C ABI of libctabba.so.
 *
 * The paper (arXiv 2602.17892) poses reconstruction as A x ~= b (Sec. 1, Eq. (1)) with a
 * forward projector A in R^{m x n} and a backprojector B in R^{n x m} that is NOT A^T
 * (Sec. 2, "unmatched projector pairs").  AB-GMRES applies GMRES to A B u = b, x = B u;
 * BA-GMRES applies it to B A x = B b (Sec. 2.1, Eqs. (AB_optimality), (BA_optimality)).
 * The hybrid variants (Sec. 3, Algorithms 1 and 2) replace the projected least-squares
 * problem by its Tikhonov-regularised form (Eq. (hybrid_proj)) with lambda chosen at every
 * iteration by GCV (Sec. 3.1) or by the discrepancy principle (Sec. 3.2).
 *
 * General rules for every entry point:
 *  - Pointers whose names end in _dev are CUDA device pointers on the current device; all
 *    others are host pointers.  The caller owns every buffer it passes; the library never
 *    frees or retains them after the call returns.
 *  - Device arrays are dense FP32, row-major: an image is [ny][nx] (3D: [nz][ny][nx]); a
 *    sinogram is [n_views][n_det_u] (3D: [n_views][n_det_v][n_det_u]).  Device pointers
 *    must be 16-byte aligned.
 *  - Work is enqueued on `stream` (0 = the legacy default stream) and is asynchronous,
 *    except where a function says it synchronises.
 *  - A geometry object owns device tables and scratch buffers.  Calls that use the same
 *    ct_geom must not overlap in time (issue them on one stream, or synchronise).
 *  - Errors are returned as ct_status; nothing is launched when an argument is invalid.
 *    ct_last_error() returns a message for the calling thread's most recent failure.
 *  - There is no CPU fallback: every numerical step runs in this library's CUDA kernels.
 */
#ifndef CTABBA_H
#define CTABBA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void *ct_stream_t; /* a cudaStream_t */

typedef enum {
    CT_OK = 0,
    CT_EINVAL = 1,      /* invalid argument (null pointer, bad size, bad enum)          */
    CT_ENOMEM = 2,      /* device allocation failed                                     */
    CT_ECUDA = 3,       /* a CUDA runtime call failed (message in ct_last_error)         */
    CT_BREAKDOWN = 4,   /* Arnoldi breakdown h_{k+1,k} <= tol ||M w_k||; iterate is valid */
    CT_ETIMEOUT = 5,    /* a bounded device wait expired                                */
    CT_ENONFINITE = 6   /* NaN or Inf met in the data or the projected problem           */
} ct_status;

typedef enum { CT_PARALLEL2D = 0, CT_FANFLAT2D = 1, CT_CONE3D = 2 } ct_geom_kind;

/* Scan geometry (the paper leaves conventions open; Sec. 4 uses parallel and fan-flat 2D):
 *   pixel (r, c) has centre X = (c - (nx-1)/2) h, Y = (r - (ny-1)/2) h;
 *   parallel: ray (theta, s) is { p : p . (cos theta, sin theta) = s },
 *             bin j at s_j = (j - (n_det_u-1)/2) pitch_u;
 *   fan-flat / cone: source at SID (cos, sin), detector centre at -(SDD-SID)(cos, sin),
 *             detector axis (-sin, cos), bin j at u_j = (j - (n_det_u-1)/2) pitch_u, rows
 *             along +z at v_i = (i - (n_det_v-1)/2) pitch_v.
 * `angles` (host, n_views entries, radians) is copied; the array may be freed afterwards. */
typedef struct {
    ct_geom_kind kind;
    int nx, ny, nz;          /* nz = 1 for 2D                                          */
    double pixel;            /* h                                                      */
    int n_views;
    const double *angles;    /* host, n_views                                          */
    int n_det_u, n_det_v;    /* n_det_v = 1 for 2D                                     */
    double pitch_u, pitch_v;
    double sid, sdd;         /* source-isocentre and source-detector distances (fan/cone) */
} ct_geom_desc;

typedef struct ct_geom ct_geom; /* opaque */

/* Validate `d`, build the per-ray and per-view device tables and the projector scratch.
 * Allocates device memory (owned by the object).  2D sizes up to 16384 per side; cone
 * volumes need nx = ny. */
ct_status ct_geom_create(const ct_geom_desc *d, ct_geom **out);
void ct_geom_destroy(ct_geom *g);
/* n = number of unknowns, m = number of measurements. */
ct_status ct_geom_dims(const ct_geom *g, int64_t *n, int64_t *m);
/* Algorithmic work of one projector call: a_samples = Joseph samples whose interpolation
 * position lies inside the image (the samples ct_forward_A computes), b_samples = pixel-view
 * pairs of ct_back_B (n * n_views).  Host-only query. */
ct_status ct_geom_work(const ct_geom *g, int64_t *a_samples, int64_t *b_samples);

/* y = A x (Sec. 1, Eq. (1)): ray-driven Joseph projector.  Every line of the driving axis
 * (the axis with the largest |ray direction| component, ties to x then y) is sampled; the
 * image is interpolated linearly (bilinearly in 3D) between pixel centres, zero outside;
 * each sample is weighted h / |d_drive|.  x_dev: n floats, y_dev: m floats (overwritten). */
ct_status ct_forward_A(ct_geom *g, const float *x_dev, float *y_dev, ct_stream_t stream);

/* x = B y (Sec. 2: B realises A^T approximately and differently): pixel/voxel-driven
 * backprojector.  For every view the ray through the pixel centre is followed to the
 * detector and y is interpolated linearly (bilinearly in 3D) there, zero outside, with
 * weight h^2/(ray spacing at the pixel) so that B has the scale of A^T:
 *   parallel h^2/pitch;  fan h^2 (SDD^2+u^2)/(L pitch SDD);
 *   cone h^3 (SDD^2+u^2+v^2)^{3/2}/(L^2 pitch_u pitch_v SDD), L = |pixel - source|.
 * y_dev: m floats, x_dev: n floats (overwritten).  With ct_geom_set_backprojector(g,
 * CT_BACK_ADJOINT) the geometry's B is A^T instead (here and in the solvers). */
ct_status ct_back_B(ct_geom *g, const float *y_dev, float *x_dev, ct_stream_t stream);

/* x = A^T y, the exact transpose of ct_forward_A (Sec. 2, the matched case; with B = A^T
 * AB-GMRES is LSQR and BA-GMRES is LSMR in exact arithmetic): every ray's samples, at the
 * same FP32 positions as A, add weight (1 - f) y_ray and weight f y_ray to their two taps'
 * pixels by atomic FP64 additions into a scratch image owned by the geometry, rounded to FP32
 * at the end (the arrival order of the rays changes the sums only far below FP32 resolution).
 * Cone geometries: bilinear taps, four per sample; the first call allocates the geometry's n
 * FP64 accumulators.  y_dev: m floats, x_dev: n floats (overwritten). */
ct_status ct_back_AT(ct_geom *g, const float *y_dev, float *x_dev, ct_stream_t stream);

/* The backprojector the solvers (and ct_back_B) use on `g`: CT_BACK_PIXEL (the unmatched
 * pixel/voxel-driven B, the default) or CT_BACK_ADJOINT (A^T: the matched pair, for the
 * LSQR / LSMR comparison of Sec. 2; allocates the accumulators ct_back_AT needs).  Host-only. */
typedef enum { CT_BACK_PIXEL = 0, CT_BACK_ADJOINT = 1 } ct_backprojector;
ct_status ct_geom_set_backprojector(ct_geom *g, ct_backprojector kind);

/* ------------------------------------------------------------------ hybrid solvers */

typedef enum {
    CT_LAMBDA_NONE = 0,   /* lambda = 0: plain AB/BA-GMRES, Eq. (proj_pbm) by Givens rotations */
    CT_LAMBDA_FIXED = 1,  /* lambda = lambda_fixed at every iteration                        */
    CT_LAMBDA_GCV = 2,    /* GCV on the projected problem (Sec. 3.1)                          */
    CT_LAMBDA_DP = 3,     /* discrepancy principle: ||H y - beta e1|| = tau * noise_norm      */
    CT_LAMBDA_LEARNED = 4,/* not in the paper: lambda_k = sigma_1 10^net(features of H_k) from a
                             trained network (see "learned lambda" below); GCV where the
                             network's output is not finite                                  */
    CT_LAMBDA_LCURVE = 5  /* L-curve criterion (Sec. 3.1): the corner (maximum curvature) of
                             (log ||H y - beta e1||, log ||y||), searched on the GCV grid     */
} ct_lambda_rule;

typedef enum { CT_BASIS_F32 = 0, CT_BASIS_BF16 = 1, CT_BASIS_F16 = 2 } ct_basis_dtype;

/* Stopping rules (Sec. 3.2).  DP and RNS use rho_k = ||H_k y_k - beta e1|| (= ||b - A x_k||
 * for AB, ||B (b - A x_k)|| for BA): the solve returns x_k at the first step k that meets the
 * rule (or x_K).  DP: rho_k <= tau * noise_norm (the paper prints the inequality reversed);
 * RNS: |rho_{k-1} - rho_k| < stop_tol * rho_{k-1}, k >= 2.  The rule is checked on the device
 * every stop_every steps, so up to stop_every - 1 steps beyond the stopping step are computed
 * (and discarded); once it fires, the remaining launches of the solve return at once.
 * NCP (normalized cumulative periodogram): at the steps stop_every, 2 stop_every, ... and K the
 * data residual r_k = b - A x_k is formed (one extra B and A per check for AB, one extra A for
 * BA), each detector row's periodogram |DFT|^2 at the frequencies 1..q = n_det_u / 2 is
 * accumulated and normalised, the rows' NCPs are averaged and their distance
 * ||c - (1..q)/q||_2 from the white-noise line is recorded; the solve stops at the first
 * checked step whose distance is larger than at the previous check and returns the iterate of
 * that previous check (iters_done = its step).  Needs 2 <= n_det_u <= 8192. */
typedef enum { CT_STOP_NONE = 0, CT_STOP_DP = 1, CT_STOP_RNS = 2, CT_STOP_NCP = 3 } ct_stop_rule;

typedef struct {
    int max_iters;           /* K >= 1                                                     */
    ct_lambda_rule rule;
    double lambda_fixed;     /* CT_LAMBDA_FIXED                                            */
    double noise_norm;       /* CT_LAMBDA_DP: ||e|| for AB, ||B e|| for BA                  */
    double tau;              /* CT_LAMBDA_DP safety factor (> 0; the paper asks tau > 1)    */
    int reorth;              /* 1 = classical Gram-Schmidt twice (default), 0 = once       */
    ct_basis_dtype basis;    /* storage type of the Krylov basis                           */
    double *lambda_hist;     /* host, max_iters entries, may be NULL: lambda_k              */
    double *resid_hist;      /* host, max_iters entries, may be NULL: ||H_k y_k - beta e1|| */
    const float *lambda_net_dev; /* CT_LAMBDA_LEARNED: the network's CT_MLP_NPARAMS FP32
                                    parameters (device; read during the solve)              */
    float *features_dev;     /* device, max_iters x CT_MLP_NIN floats, may be NULL: row k-1
                                receives the features of H_k (any rule but CT_LAMBDA_NONE)  */
    ct_stop_rule stop_rule;  /* CT_STOP_NONE (default): exactly max_iters steps             */
    double stop_tol;         /* CT_STOP_RNS tolerance (> 0)                                 */
    int stop_every;          /* steps between device-side checks of the rule (>= 1)         */
    double *ncp_hist;        /* host, max_iters entries, may be NULL: the NCP distance of every
                                checked step (CT_STOP_NCP), NaN at the other steps          */
} ct_hybrid_opts;

typedef struct {
    int iters_done;          /* k of the returned iterate (the stopping step under a rule)  */
    double beta;             /* ||r0||                                                     */
    double final_lambda;
    double final_resid;      /* ||H_k y_k - beta e1|| (= ||b - A x_k|| for AB)             */
    ct_status status;        /* CT_OK or CT_BREAKDOWN                                      */
    int fast_path_steps;     /* steps whose hybrid step took the parallel path (the others ran
                                the exact sequential SVD path; diagnostics only)            */
    int lambda_fallback_steps; /* CT_LAMBDA_LEARNED: steps where GCV replaced the network   */
} ct_hybrid_info;

/* Fill `o` with defaults: K = 30, GCV, tau = 1.01, reorth = 1, FP32 basis, no history, no
 * stopping rule (stop_tol = 1e-3, stop_every = 5 for when one is set). */
void ct_hybrid_opts_default(ct_hybrid_opts *o);

/* Hybrid AB-GMRES, Algorithm 1 (Sec. 3): x0 = B u0 (u0 = 0 when u0_dev is NULL),
 * r0 = b - A x0, Arnoldi on A B with classical Gram-Schmidt applied twice, lambda_k by
 * `o->rule`, y_k from Eq. (hybrid_proj) through the SVD of H_k in FP64 (its Householder
 * bidiagonalisation in double-float, pairs of FP32 numbers with about 48 bits), and
 * x_K = x0 + B W_K y_K.  b_dev: m floats; x_dev: n floats (output).  The residual
 * r_k = b - A x_k of Algorithm 1 is not recomputed for the norm-based rules: ||b - A x_k||
 * equals the projected residual.
 * Allocates its workspace on the first call for a geometry (reused while max_iters and
 * basis do not grow).  Synchronises `stream` before returning to fill `info` and the
 * host histories. */
ct_status ab_gmres_hybrid(ct_geom *g, const float *b_dev, const float *u0_dev, float *x_dev,
                          const ct_hybrid_opts *o, ct_hybrid_info *info, ct_stream_t stream);

/* Hybrid BA-GMRES, Algorithm 2 (Sec. 3): r0 = B (b - A x0) (x0 = 0 when x0_dev is NULL),
 * Arnoldi on B A, x_K = x0 + W_K y_K.  Same conventions as ab_gmres_hybrid. */
ct_status ba_gmres_hybrid(ct_geom *g, const float *b_dev, const float *x0_dev, float *x_dev,
                          const ct_hybrid_opts *o, ct_hybrid_info *info, ct_stream_t stream);

/* Restarted hybrid AB-/BA-GMRES (Sec. 3.3, Restarting): `cycles` cycles of o->max_iters = p
 * steps each, every cycle restarting Algorithm 1 / 2 from the iterate of the previous one
 * (AB keeps its iterate as u with x = B u, so its restart r0 = b - A B u equals the restart from
 * x; BA restarts from x).  The Krylov basis holds p + 1 vectors whatever the number of cycles.
 * lambda is chosen per step by o->rule as in the plain solvers.  x_dev (n floats) receives the
 * final iterate (its input content is ignored).  o->lambda_hist / o->resid_hist, when given,
 * need cycles * p entries (cycle-major); o->features_dev is ignored.  info: iters_done sums the
 * cycles, beta is the first cycle's ||r0||, the rest describes the last cycle.  Synchronises
 * `stream` after every cycle.  A cycle that starts from an exact iterate (r0 = 0) ends the
 * solve. */
ct_status ab_gmres_hybrid_restarted(ct_geom *g, const float *b_dev, float *x_dev, int cycles,
                                    const ct_hybrid_opts *o, ct_hybrid_info *info,
                                    ct_stream_t stream);
ct_status ba_gmres_hybrid_restarted(ct_geom *g, const float *b_dev, float *x_dev, int cycles,
                                    const ct_hybrid_opts *o, ct_hybrid_info *info,
                                    ct_stream_t stream);

/* ------------------------------------------------------------------ tile autotuning */

/* Launch shapes of the projector kernels of a geometry. */
typedef struct {
    int a_threads;   /* 2D Joseph A: threads per block                                    */
    int a_views;     /* Joseph A: 2D, views per block (a_threads / a_views consecutive bins of
                        each); 3D, detector rows per block of 32 columns (each warp one row) */
    int a_slab;      /* 3D Joseph A: z-slab thickness (tap rows) of one pass; each pass
                        reads one slab of the volume's pair layouts, so it stays in L2    */
    int b_rows;      /* 2D pixel-driven B: pixel rows per block                           */
    int b_views;     /* 2D pixel-driven B: views per loop iteration (1, or 2 with paired FP32
                        arithmetic, gathers in batches of 8 view pairs, at most 8 rows per
                        block; the same operations, so results do not change).  4: the
                        four-fold kernel, for fan geometries on a square image of even side
                        whose views come in quadruples a quarter turn apart (view k + m n/4 at
                        angle theta_k + m pi/2): a thread takes the four pixels one quarter
                        turn of the image maps onto each other and evaluates the bin position
                        and weight once for the four views that see them alike; each
                        pixel-view pair has the same operations, with view k's cos and sin
                        for the rotated pixel, and the views are summed in another order, so
                        results agree with b_views 1 and 2 to FP32 rounding, not bit for bit
                        (b_rows 4, 8, 16: blocks of 32 x 2, 32 x 4, 32 x 2 orbits with the
                        base views split into 2, 2, 4 parts)                              */
    int a_rays;      /* 3D Joseph A: detector rows per thread, 1 or 2 (two rays of one detector
                        column share their in-plane tap positions; the same operations per
                        sample, so results do not change); ignored in 2D                    */
    int a_warp_views; /* 2D Joseph A: views per warp, 1, 2, 4 or 8 (a warp takes 32 / a_warp_views
                        consecutive bins of each; several views of fewer bins keep a warp's
                        taps on one line within fewer cache lines); divides a_views; 1 in 3D */
    int b_warp_rows; /* 2D pixel-driven B: pixel rows per warp, 1, 2 or 4 (a warp takes a tile
                        of 32 / b_warp_rows columns by b_warp_rows rows; for the four-fold
                        kernel, of orbit positions); at most the block's rows (b_rows, or the
                        orbit rows of the four-fold kernel: 2 for b_rows 4 and 16, 4 for 8);
                        ignored in 3D                                                        */
} ct_launch_shapes;

/* Time the candidate launch shapes of the projectors on this geometry and keep the fastest for
 * later calls on `g`.  2D: Joseph A with (threads, views) per block in (128, 1), (128, 2),
 * (128, 4), (256, 1), (256, 2), (256, 4), (512, 4), (512, 8); pixel-driven B with 4, 8 or 16
 * pixel rows per block and one view per loop iteration, or 4 or 8 rows and two, and for
 * geometries with the four-fold symmetry also the four-fold kernel (b_rows 4, 8, 16), each with
 * warps of 32 x 1 pixels and of the taller tiles its block allows, and the Joseph shapes with
 * several views per warp (threads, views per block, views per warp) in (128, 2, 2), (128, 4, 2),
 * (128, 4, 4), (256, 4, 4), (256, 8, 4), (256, 8, 8), (512, 8, 4).  3D: Joseph
 * (slab thickness, warp rows per block, detector rows per thread) in (16, 1, 1), (16, 4, 1),
 * (16, 8, 1), (64, 4, 1), (64, 8, 1), one pass over the whole volume with 1, 4 or 8 warp rows
 * and one detector row per thread, and (16, 4, 2), (64, 4, 2), one pass with 2 or 4 warp rows
 * and two detector rows per thread (the voxel-driven B has one shape, 32 x 4 columns of 8
 * voxels).  The shapes change only the order of work, not
 * the arithmetic of a sample (the four-fold B: see ct_launch_shapes).  Geometries of the same
 * kind, sizes and symmetry reuse an earlier result.
 * Runs a few dozen projector launches on `stream`, synchronises it, and allocates two temporary
 * device buffers.  The chosen shapes are written to *out (may be NULL). */
ct_status ct_geom_autotune(ct_geom *g, ct_stream_t stream, ct_launch_shapes *out);
/* Set the projectors' launch shapes of `g` explicitly (for instance a shape an earlier autotune
 * found, or a fixed one for timing).  Values: a_threads in {128, 256, 512}, a_views in
 * {1, 2, 4, 8}, a_warp_views in {1, 2, 4, 8} dividing a_views, and a_threads / a_views >=
 * 32 / a_warp_views (2D), a_slab >= 1 (3D; >= nz + 1 is one pass),
 * a_views in 1..8 warp rows (3D), a_rays in {1, 2} (3D), b_rows in {4, 8, 16}, b_views in
 * {1, 2, 4} (b_rows 16 only with b_views 1; b_views 4 only on a geometry with the four-fold
 * symmetry described at ct_launch_shapes), b_warp_rows in {1, 2, 4} up to the block's rows
 * (2D); in 3D a_warp_views and b_warp_rows are not checked and read back as 1; anything else
 * returns CT_EINVAL and leaves `g` unchanged.  Host-only; shapes change the order of work, not a
 * sample's arithmetic. */
ct_status ct_geom_set_launch_shapes(ct_geom *g, const ct_launch_shapes *shapes);
/* The launch shapes `g` uses now. */
ct_status ct_geom_get_launch_shapes(const ct_geom *g, ct_launch_shapes *out);

/* ------------------------------------------------------------------ batched solves */

/* Many independent problems (for instance CT slices of uneven size and geometry) solved
 * together.  The first ct_batch_solve captures every problem's whole solve (Algorithm 1 or 2:
 * all iterations, the hybrid steps and the final iterate) into one CUDA graph whose branches are
 * independent, so the GPU runs the problems concurrently; later calls with the same buffers and
 * noise norms replay that graph with a single launch.  Each problem needs its own ct_geom (the
 * geometry owns the problem's workspace; ct_batch_create allocates it).
 * methods[i]: 0 = hybrid AB-GMRES, 1 = hybrid BA-GMRES, 2 = AB when m < n, else BA (Sec. 2.1:
 * AB-GMRES for underdetermined, BA-GMRES for overdetermined systems).  All problems share `o`
 * (its history pointers must be NULL) except the discrepancy-principle noise norms, which
 * ct_batch_solve takes per problem.  autotune != 0 runs ct_geom_autotune on every geometry. */
typedef struct ct_batch ct_batch;
ct_status ct_batch_create(int n_prob, ct_geom *const *geoms, const int *methods,
                          const ct_hybrid_opts *o, int autotune, ct_batch **out);
/* b_dev[i]: m_i floats, x_dev[i]: n_i floats (device pointers in host arrays of n_prob
 * entries); noise_norms: host array (used by CT_LAMBDA_DP, may be NULL otherwise); info: host
 * array of n_prob entries (may be NULL).  Initial guesses are zero.  Synchronises `stream`.
 * Calls on one batch must not overlap. */
ct_status ct_batch_solve(ct_batch *bt, const float *const *b_dev, float *const *x_dev,
                         const double *noise_norms, ct_hybrid_info *info, ct_stream_t stream);
/* Kernel launches one replay of the batch's graph performs (0 before the first solve). */
int64_t ct_batch_launches(const ct_batch *bt);
void ct_batch_destroy(ct_batch *bt);
/* One call: create a batch (with autotuning), solve it once, destroy it. */
ct_status abba_solve(int n_prob, ct_geom *const *geoms, const float *const *b_dev,
                     float *const *x_dev, const int *methods, const ct_hybrid_opts *o,
                     const double *noise_norms, ct_hybrid_info *info, ct_stream_t stream);

/* ------------------------------------------------------------------ building blocks */

/* One Arnoldi orthogonalisation step (Sec. 2.1, Eq. (Hessenberg)).
 * Allocates its scratch with stream-ordered cudaMallocAsync/cudaFreeAsync on every call.
 * given k+1 orthonormal rows W[0..k] (each `len` floats, row stride `ld` floats) and
 * q = M w_k, compute h[i] = <q, w_i> by classical Gram-Schmidt applied twice (the second
 * pass's coefficients added), h[k+1] = ||q||, and W[k+1] = q / h[k+1].  W_dev must have
 * room for k+2 rows; q_dev (len floats) is overwritten; h_dev receives k+2 doubles. */
ct_status ct_arnoldi_step(float *W_dev, int64_t len, int64_t ld, int k, float *q_dev,
                          double *h_dev, ct_stream_t stream);

/* ct_arnoldi_step without any device allocation.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate GPU memory while they run.  cudaFree
 * synchronises the whole device, which would stall acquisition or other work that the caller
 * keeps running on other streams, and an application that reserves the GPU's memory through its
 * own pool cannot let a library take more.  ct_arnoldi_step allocates and frees its scratch
 * (per-block partial sums, counters) on every call; this variant keeps that scratch in one
 * static device array of about 1.3 MB in the library, which every GPU that loads the library
 * holds until the process exits.
 *   - Same arguments, results and layout rules as ct_arnoldi_step.
 *   - Limit: k <= 126 (h has at most 128 entries); larger k returns CT_EINVAL with a message,
 *     and nothing is launched.
 *   - The first call on a device, with that device current, looks up the array's device
 *     address (cudaGetSymbolAddress) once; make that first call before any stream capture.
 *   - Every call uses the same array and the array keeps the previous call's contents (the
 *     call clears what must start at zero), so calls that overlap on the GPU (different
 *     streams, or concurrent host threads) race: serialise them.
 *   - Calls no cudaMalloc, cudaFree or allocating library routine. */
ct_status ct_arnoldi_step_noalloc(float *W_dev, int64_t len, int64_t ld, int k, float *q_dev,
                                  double *h_dev, ct_stream_t stream);

/* The hybrid step on the device (Sec. 3, Eq. (hybrid_proj); Sec. 3.1/3.2): for the
 * (k+1) x k Hessenberg matrix H (FP64, column-major, leading dimension ldh >= k+1) and
 * beta = ||r0||, choose lambda by `rule` and return y (k doubles), lambda and the projected
 * residual ||H y - beta e1||.  All pointers are device pointers.  1 <= k <= 160;
 * any rule but CT_LAMBDA_LEARNED.  The singular values and first components come from a
 * bidiagonal form computed in double-float (about 48 bits) and FP64 Sturm counts and Newton
 * steps; if their Parseval check fails, the solve falls back to a sequential FP64 SVD. */
ct_status ct_projected_solve(const double *H_dev, int ldh, int k, double beta,
                             ct_lambda_rule rule, double lambda_fixed, double dp_target,
                             double *y_dev, double *lambda_dev, double *resid_dev,
                             ct_stream_t stream);

/* ------------------------------------------------------------------ learned lambda */

/* Not in the paper.  A 3-layer perceptron predicts log10(lambda_k / sigma_1(H_k)) from
 * features of the projected problem; CT_LAMBDA_LEARNED uses it in place of GCV or the
 * discrepancy principle, which stay the fallback and the measure of its reconstruction error.
 *
 * Features of H_k (CT_MLP_NIN = 80 floats, computed by the hybrid step from the SVD of H_k,
 * H_k = U diag(sigma) V^T, c = beta U^T e1 with c_{k+1} the component outside range(H_k)):
 *   [0] k / max_iters; [1..32] log10(sigma_i / sigma_1) for the 32 largest sigma_i (pad -16);
 *   [33..64] |c_i| / beta for the same i (pad 0); [65] |c_{k+1}| / beta; [66] log10 sigma_1;
 *   [67] log10 beta; [68..79] 0.
 * Network: the features standardised in FP32, f' = (f - mu) * isd, then 80 -> 64 -> 64 -> 1
 * with GELU (tanh form) after both hidden layers.  Parameters, one FP32 vector of
 * CT_MLP_NPARAMS entries in this order: W1[64][80], b1[64], W2[64][64], b2[64], w3[64], b3,
 * mu[80], isd[80] (mu and isd are set before training and get zero gradient).  bf16 != 0:
 * weights, standardised inputs and both hidden activations are rounded to BF16 and the
 * products accumulate in FP32 on the tensor cores (the solver's inference always works this
 * way); bf16 == 0: the same arithmetic in FP32 on the CUDA cores. */
#define CT_MLP_NIN 80
#define CT_MLP_NPARAMS 9569

/* out_dev[i] = net(X_dev[i][0..79]) for i < n.  X: n x 80 floats, row-major. */
ct_status ct_mlp_forward(const float *params_dev, const float *X_dev, int n, float *out_dev,
                         int bf16, ct_stream_t stream);
/* Gradient of the mean squared error (1/n) sum_i (net(X_i) - Y_i)^2 with respect to every
 * parameter into grad_dev (CT_MLP_NPARAMS floats), and that error into *loss_dev (device, may
 * be NULL).  Deterministic (fixed summation order).  Allocates its scratch with
 * cudaMallocAsync/cudaFreeAsync on `stream`. */
ct_status ct_mlp_grad(const float *params_dev, const float *X_dev, const float *Y_dev, int n,
                      float *grad_dev, float *loss_dev, int bf16, ct_stream_t stream);
/* One Adam step (Kingma and Ba; beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected with
 * step number t >= 1) on the FP32 parameters, moments m_dev and v_dev updated in place. */
ct_status ct_mlp_adam(float *params_dev, const float *grad_dev, float *m_dev, float *v_dev,
                      float lr, int t, ct_stream_t stream);
/* Mini-batch training: `epochs` passes over the n samples in batches of `batch` rows (the last
 * partial batch of a pass included), one ct_mlp_grad and one ct_mlp_adam per batch, Adam's
 * step counter starting at *t + 1 (updated).  The caller shuffles X/Y between calls if it
 * wants a new order.  loss_hist_dev (device, may be NULL) receives each batch's loss in order
 * (ceil(n / batch) * epochs floats). */
ct_status ct_mlp_train(float *params_dev, float *m_dev, float *v_dev, const float *X_dev,
                       const float *Y_dev, int n, int batch, int epochs, float lr, int *t,
                       float *loss_hist_dev, int bf16, ct_stream_t stream);

/* Training samples from one hybrid AB-GMRES solve (Algorithm 1 with u0 = 0, o->max_iters = K
 * <= 64, FP32 basis, any rule but CT_LAMBDA_NONE) of b_dev, whose exact image x_true_dev
 * (n floats) is known.  For k = 1..K: feats_dev row k-1 (80 floats) gets the features of H_k
 * and labels_dev[k-1] = log10(lambda*_k / sigma_1(H_k)), where lambda*_k minimises the
 * reconstruction error ||x_k(lambda) - x_true|| with x_k(lambda) = B W_k y_k(lambda):
 * lambda is searched like GCV (256 log-spaced points on [1e-8 sigma_1, sigma_1], the best one
 * refined by 40 golden-section steps).  The error is a quadratic in y through
 * G = Z^T Z, g = Z^T x_true with Z = B W_K (K extra applications of B).  Labels are NaN
 * where H_k is zero.  x_dev (n floats) receives the solve's own iterate.  Allocates scratch
 * with cudaMallocAsync; synchronises `stream`. */
ct_status ct_lambda_samples(ct_geom *g, const float *b_dev, const float *x_true_dev,
                            const ct_hybrid_opts *o, float *x_dev, float *feats_dev,
                            float *labels_dev, ct_hybrid_info *info, ct_stream_t stream);

/* ------------------------------------------------------------------ instrumentation */

/* Device time per phase of the solvers and projectors, from CUDA events recorded on the
 * launching stream around every launch group while profiling is enabled (adds about one
 * microsecond per group).  Phases: */
enum {
    CT_PH_FORWARD = 0,   /* Joseph A kernel                                   */
    CT_PH_BACK = 1,      /* pixel-driven B kernel                             */
    CT_PH_LAYOUT = 2,    /* image pair layouts / padded sinogram copies        */
    CT_PH_ARNOLDI = 3,   /* the four Gram-Schmidt kernels of one Arnoldi step  */
    CT_PH_SMALL = 4,     /* the hybrid small solve (FP64; double-float bidiagonalisation) */
    CT_PH_OTHER = 5,     /* first normalisation, x = x0 + W y, residual updates */
    CT_PH_COUNT = 6
};
typedef struct { double ms; int64_t launches; int64_t groups; } ct_phase_time;

/* Enable (1) or disable (0) event timing; enabling clears the accumulated records. */
ct_status ct_profile_enable(int on);
/* Wait for the recorded events, add their durations into out[CT_PH_COUNT] (overwritten) and
 * clear the records.  Host-blocking. */
ct_status ct_profile_collect(ct_phase_time *out);
/* Number of kernels this library has launched since it was loaded (all phases). */
int64_t ct_launch_count(void);

/* Throughput probes for the rooflines of the gather-bound projectors: one wave of resident
 * blocks on every SM of the current device doing only the elementary work of a projector
 * sample, so that its duration (timed by the caller with events on `stream`) gives a measured
 * ceiling.  CT_PROBE_GATHER8: one 8-byte load from an L1-resident table (each warp reads 32
 * consecutive pairs, the best case of the projectors' near-contiguous tap-pair gathers) plus
 * one fused multiply-add that consumes it.  CT_PROBE_MUFU: one reciprocal and one square root
 * (the special-function pair of a fan-beam pixel-driven sample) plus one addition.  Every
 * thread does `reps` operations (rounded up to a multiple of 8) in 8 independent chains and
 * writes one float to out_dev (out_floats >= resident blocks x 256; 152 SMs x 8 x 256 always
 * suffices).  *ops (host) receives the operation count of the launch.  Asynchronous. */
typedef enum { CT_PROBE_GATHER8 = 0, CT_PROBE_MUFU = 1 } ct_probe_kind;
ct_status ct_probe(int kind, int64_t reps, float *out_dev, int64_t out_floats, int64_t *ops,
                   ct_stream_t stream);

/* Test hook of failure detection (off by default; not for production use).  enable != 0 arms
 * it on the current device: the next Gram-Schmidt tile pass launched there leaves the
 * asynchronous copies of its block 0's first tile unissued (nothing is in flight for them), so
 * that block's bounded waits run out after wait_cycles GPU clocks (2^16 .. 2^31); the pass
 * records CT_ETIMEOUT in the solver's state and returns, the rest of that solve is skipped and
 * the solver returns CT_ETIMEOUT (its iterate is not valid); later solves run normally.  The
 * hook disarms itself after that one use; enable = 0 disarms it and restores the default wait
 * limit (about 2^31 clocks).  Synchronous host call. */
ct_status ct_test_drop_tile_copy(int enable, int64_t wait_cycles);

/* Status name and the calling thread's last error message. */
const char *ct_status_string(ct_status s);
const char *ct_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CTABBA_H */
