/*
 * mvd.h -- C ABI of a GB300 (sm_103a) library for plane-wise multi-view
 * Richardson-Lucy (MV-RL) deconvolution.
 *
 * The method (Schmid & Huisken, "Real-time multi-view deconvolution"):
 *   - every registered view stack is resliced into planes orthogonal to the
 *     rotation axis (Abstract; Fig. 1a);
 *   - every plane is deconvolved independently with one 2D PSF per view
 *     (Results: the 3D transfer function is approximated by a 2D PSF);
 *   - one iteration is the multi-view RL update of Supp. Note 1:
 *         psi <- psi * prod_v [ (phi_v / (psi * P_v)) (*) P_v^* ]
 *     with P_v^* the flipped PSF (Supp. Note 2, sec. 1).
 *
 * Conventions used by every entry point
 *   - Pointers named *_dev are device pointers on the device that was current
 *     when the context was created; pointers named *_host are host pointers.
 *     All buffers passed in are owned by the caller; the library never frees
 *     or keeps them after the call returns.
 *   - Layouts are dense, row-major, the last index contiguous:
 *       stack   [V][Z][Y][X]   registered view stacks (z-slices of Y x X)
 *       planes  [V][P][H][W]   resliced data, P = Y planes of H = Z rows and
 *                              W = X columns
 *       estimate [P][H][W]     FP32
 *   - PSFs are K x K, K odd, centre (R, R) with R = (K-1)/2, row index along
 *     the plane's rows.  Convolution: b(y,x) = sum_ij P[i][j] psi(y-i+R, x-j+R).
 *   - Device work is asynchronous on the given stream (a cudaStream_t; NULL is
 *     the legacy default stream), like the paper's workflow (Supp. Note 2,
 *     sec. 3).  Argument errors are found before anything is enqueued.
 *   - Every function returns a status; nothing is thrown across the ABI.
 *     mvd_last_error() gives a human-readable detail for the calling thread.
 *   - A context may be used from one host thread at a time.
 */
#ifndef MVD_H
#define MVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mvd_ctx mvd_ctx;

typedef enum {
    MVD_OK = 0,
    MVD_ERR_ARG = 1,          /* an argument is invalid (see mvd_last_error) */
    MVD_ERR_CUDA = 2,         /* a CUDA call or kernel launch failed         */
    MVD_ERR_NOMEM = 3,        /* a device or host allocation failed           */
    MVD_ERR_TIMEOUT = 4,      /* a bounded device-side wait ran out           */
    MVD_ERR_STATE = 5,        /* the call is not valid in this state          */
    MVD_ERR_UNSUPPORTED = 6   /* the selected route cannot take these sizes   */
} mvd_status;

typedef enum {
    /* Outside the plane the estimate and the ratio are zero: the linear
     * convolution cropped to the plane, which is what padding each plane by
     * the PSF size for Fourier convolution implements (Supp. Table 1). */
    MVD_BOUNDARY_ZERO = 0,
    /* Plane indices are taken modulo H and W (needs K <= min(H, W)). */
    MVD_BOUNDARY_CIRCULAR = 1
} mvd_boundary;

typedef enum {
    MVD_U16 = 0,   /* camera data, uint16 (Supp. Note 1 memory table) */
    MVD_F32 = 1
} mvd_dtype;

typedef enum {
    /* Fused tiled path: per iteration one kernel blurs the estimate with
     * every view's PSF and forms the ratios, a second correlates, multiplies
     * the views' corrections and updates the estimate, for all planes in one
     * launch.  PSFs are used through an exact FP64 SVD factorisation
     * P = sum_q s_q u_q w_q^T truncated only below FP32 resolution. */
    MVD_ALGO_FUSED = 0,
    /* Plain per-plane path: one plane at a time, one kernel per step
     * (vertical pass, horizontal pass, ratio, ... , update), same factors.
     * Kept as the comparison baseline. */
    MVD_ALGO_PLAIN = 1,
    /* Plain per-plane path with K x K direct convolutions (no factorisation). */
    MVD_ALGO_DIRECT = 2,
    /* Fourier route (Supp. Note 2 sec. 4): both convolutions as products of
     * spectra, with the library's own batched mixed-radix FFT and the ratio,
     * product and update fused into the transforms.  The grid is padded to
     * the smallest 2^a 3^b 5^c sizes >= H + R and W + R (ZERO boundary) or is
     * the plane itself (CIRCULAR, whose sides must then be such sizes);
     * padded sides <= 2048.  Its cost does not grow with K or with the PSFs'
     * separable rank (oblique views). */
    MVD_ALGO_FFT = 3,
    /* Optional tensor-core route: the fused kernels with every separable 1D
     * pass run as a banded (Toeplitz) matrix product on the tcgen05 tensor
     * cores in BF16x3 (each FP32 operand split into BF16 hi + lo, three
     * products per multiply, FP32 accumulation: about 2^-16 relative error
     * per product instead of 2^-24); the ratio, the product over views and
     * the update stay FP32.  Odd K <= 47, any number of separable terms,
     * both boundaries.  Never chosen by default or by mvd_autotune. */
    MVD_ALGO_TENSOR = 4,
    /* Optional reduced-precision tensor-core route: the same banded matrix
     * products in TF32 (operands rounded to 10 explicit mantissa bits, round
     * to nearest; FP32 accumulation: about 2^-11 relative error per product),
     * one MMA per product.  The ratio, the product over views and the update
     * stay FP32.  Odd K <= 47, any number of separable terms, both
     * boundaries.  Its error against the exact result is larger than the
     * FP32 routes' and is reported, not bounded by their tolerance.  Never
     * chosen by default or by mvd_autotune. */
    MVD_ALGO_TF32 = 5,
    /* Plane-resident route: one thread-block cluster of up to 16 CTAs keeps
     * a plane's estimate, ratio and (simultaneous order) product of the
     * views' corrections in shared memory for all iterations; the vertical
     * passes read the rows next to a CTA's strip from its neighbours' shared
     * memory (distributed shared memory), cluster barriers separate the
     * phases of each iteration (Supp. Note 1 update).  Per iteration HBM is
     * read only for the data phi_v.  Same separable factors and FP32
     * arithmetic as MVD_ALGO_FUSED.  ZERO boundary, K <= 47, planes of up to
     * 512 columns whose three (simultaneous) or two (sequential) strip
     * buffers fit in shared memory: up to 512 x 512 (16 CTAs of 32 rows).
     * Never chosen by default or by mvd_autotune. */
    MVD_ALGO_RESIDENT = 6
} mvd_algo;

typedef enum {
    /* All views use the same estimate and their corrections are multiplied,
     * as the update equation of Supp. Note 1 is printed (default). */
    MVD_ORDER_SIMULTANEOUS = 0,
    /* The views update the estimate one after another, each with its own
     * factor of the same equation evaluated at the current estimate (the
     * sequential scheme of the multi-view RL work the paper builds on, Supp.
     * Note 2 sec. 1).  The simultaneous product over-corrects when several
     * views share a PSF (e.g. views 180 degrees apart) and can diverge;
     * each sequential sub-step is a single-view RL step. */
    MVD_ORDER_SEQUENTIAL = 1
} mvd_update_order;

/* Variants of multi-view RL (Supp. Note 2 sec. 1).  All keep the update
 * psi <- psi * prod_v [(phi_v / (psi * P_v)) * X_v] and differ in the kernel
 * X_v the ratio of view v is convolved with.  With P^* the flipped PSF, '.'
 * the entry-wise product over the K x K support, '*' a convolution of two
 * K x K kernels cropped to the K x K centre, and products over the other
 * views w != v, each X_v scaled to unit sum:
 *   INDEPENDENT          X_v = P_v^* (plain MV-RL; the PSF as given, unscaled)
 *   EFFICIENT_BAYESIAN   X_v = P_v^* . prod_w (P_v^* * P_w * P_w^*)
 *   OPTIMIZATION_1       X_v = P_v^* . prod_w (P_v^* * P_w)
 *   OPTIMIZATION_2       X_v = P_v^* . prod_w P_w^*
 * The printed formulas leave the support, the normalisation and, for
 * optimization I, an index open; these are the readings taken. */
typedef enum {
    MVD_VARIANT_INDEPENDENT = 0,
    MVD_VARIANT_EFFICIENT_BAYESIAN = 1,
    MVD_VARIANT_OPTIMIZATION_1 = 2,
    MVD_VARIANT_OPTIMIZATION_2 = 3
} mvd_variant;

/* Summary of what a context decided; filled by mvd_get_info. */
typedef struct {
    int views;
    int psf_size;
    int plane_h, plane_w;
    int iters;
    int boundary;
    int algo;                   /* mvd_algo in use                          */
    int order;                  /* mvd_update_order in use                  */
    int rank[16];               /* SVD terms kept per view (first 16 views) */
    int blur_groups;            /* number of distinct PSFs among the views  */
    int blur_terms;             /* SVD terms summed over distinct PSFs      */
    int tile_h, tile_w;         /* fused path output tile                   */
    size_t workspace_bytes;     /* device scratch currently held            */
    int variant;                /* mvd_variant in use                       */
    int corr_rank[16];          /* SVD terms of the correlation kernel per
                                   view (= rank for INDEPENDENT)            */
    int flops_blur;             /* fused kernels, FLOP per voxel and launch:
                                   2 per tap of every 1D pass run, blur of
                                   every distinct PSF (narrow factors run
                                   with their 17 central taps for K <= 31,
                                   21 above, when the rest is below the
                                   rank tolerance; full taps with weights
                                   set)                                     */
    int flops_corr;             /* the same for the correlation of all views */
} mvd_info;

/* Create a context for `views` views with K x K PSFs psfs_host[V][K][K]
 * (FP32, host memory, copied), planes of plane_h x plane_w pixels, `iters`
 * RL iterations, the given boundary and division guard eps
 * (ratio = phi / max(blur, eps)).  These are the quantities of the update
 * equation of Supp. Note 1 (one 2D PSF per view, Results: the plane-wise
 * approximation) and of the user's choice of the iteration count (Supp.
 * Note 2 sec. 2); the context keeps the PSFs' separable factors and the
 * device scratch the iterations need (the buffers of the memory table of
 * Supp. Note 1 that the library owns).
 *
 * Errors (MVD_ERR_ARG): views < 1 or > 64, K even or < 1, plane sizes < 1,
 * iters < 0, eps <= 0 or not finite, a PSF entry negative or not finite, a
 * PSF with sum <= 0, CIRCULAR with K > min(plane_h, plane_w).
 * The context binds to the current CUDA device. */
mvd_status mvd_create(mvd_ctx **out, int views, const float *psfs_host, int psf_size,
                      int plane_h, int plane_w, int iters, mvd_boundary boundary, float eps);

/* Release the context and every device buffer it owns (the library-owned
 * buffers of Supp. Note 1's memory table: ratio scratch, means, spectra);
 * caller-owned buffers are untouched.  NULL is accepted. */
mvd_status mvd_destroy(mvd_ctx *ctx);

/* Select the route (default MVD_ALGO_FUSED when the PSFs' separable terms
 * fit its parameter block, else the Fourier route, else plain).
 * MVD_ERR_UNSUPPORTED if the route cannot take this context:
 *   MVD_ALGO_FUSED        K <= 47 and the separable terms fit;
 *   MVD_ALGO_FFT          a padded grid of 2^a 3^b 5^c sides <= 2048 exists;
 *   MVD_ALGO_TENSOR/TF32  odd K <= 47;
 *   MVD_ALGO_RESIDENT     ZERO boundary, K <= 47, no weights or axial
 *                         profiles, a plane that fits on chip (see above);
 *   MVD_ALGO_PLAIN/DIRECT any K.
 * Weights, axial profiles, mvd_run_host and mvd_psf_grad add their own
 * restrictions (see there). */
mvd_status mvd_set_algo(mvd_ctx *ctx, mvd_algo algo);

/* Select how the views combine within one iteration (default simultaneous). */
mvd_status mvd_set_update_order(mvd_ctx *ctx, mvd_update_order order);

/* Select the RL variant (default INDEPENDENT).  The variant's kernels X_v are
 * built from the context's PSFs on the host in FP64 and factorised like the
 * PSFs; every route (fused, plain, direct, Fourier) then correlates with
 * them.  mvd_set_psfs rebuilds them.  MVD_ERR_ARG for an unknown variant. */
mvd_status mvd_set_variant(mvd_ctx *ctx, mvd_variant variant);

/* Pick the context's route by timing: every route that can take its PSFs
 * and plane (the fused separable kernels, the Fourier route) runs twice on
 * the first min(n_planes, 8) planes of data_dev [V][n_planes][H][W] and the
 * faster is kept.  Without tuning a context starts on the fused kernels when
 * the PSFs' separable terms fit them, else on the Fourier route.  With
 * MVD_TUNE_CACHE naming a file, choices are cached there by shape.  Uses
 * temporary device buffers; waits for `stream`. */
mvd_status mvd_autotune(mvd_ctx *ctx, const void *data_dev, mvd_dtype dt, int n_planes, void *stream);

/* Relative Frobenius tolerance below which trailing SVD terms of a PSF are
 * dropped (default 3e-7, below the FP32 rounding of the PSF's entries).
 * 0 keeps every non-zero term. */
mvd_status mvd_set_rank_tolerance(mvd_ctx *ctx, double tol);

mvd_status mvd_get_info(const mvd_ctx *ctx, mvd_info *info);

/* Reslicing (Abstract; Fig. 1a): stacks_dev [V][Z][Y][X] of dtype dt ->
 * planes_dev [V][Y][Z][X], i.e. plane y holds rows z and columns x.  The
 * rotation axis is the stacks' middle axis Y.  Buffers must not overlap.
 * Sizes are independent of the context's plane shape. */
mvd_status mvd_reslice(mvd_ctx *ctx, const void *stacks_dev, mvd_dtype dt, int views,
                       int nz, int ny, int nx, void *planes_dev, void *stream);

/* Run the context's `iters` MV-RL iterations (Supp. Note 1) on n_planes
 * independent planes.
 *   data_dev     [V][n_planes][H][W] of dtype dt (H, W = the context's plane)
 *   estimate_dev [n_planes][H][W] FP32.  If init_mean != 0 it is ignored on
 *                entry and every plane starts from the mean of that plane's
 *                pixels over all views (computed in FP64); else it holds the
 *                initial estimate.  On return (stream order) it holds the
 *                result.  It must not overlap data_dev.
 * The context keeps device scratch sized for the largest n_planes seen
 * (one estimate copy plus V ratio planes per plane). */
mvd_status mvd_deconvolve_planes(mvd_ctx *ctx, const void *data_dev, mvd_dtype dt,
                                 float *estimate_dev, int n_planes, int init_mean,
                                 void *stream);

/* End-to-end call on host buffers: stacks_host [V][Z][Y][X] (dt) ->
 * out_host [Y][Z][X] FP32 (Z = H, X = W of the context), i.e. copy to the
 * device, reslice, deconvolve from the per-plane mean and copy back.  Planes
 * move in chunks of `chunk_planes` (0 = automatic) so that copies in both
 * directions overlap the iterations of other chunks (the paper's interleaved
 * workflow, Supp. Note 2 sec. 3, with device memory instead of disk).  Host
 * buffers should be page-locked for full copy speed.  Returns when out_host
 * is complete. */
mvd_status mvd_run_host(mvd_ctx *ctx, const void *stacks_host, mvd_dtype dt,
                        int nz, int ny, int nx, float *out_host, int chunk_planes,
                        void *stream);

/* The chunks of planes mvd_run_host uses for ny planes of plane_bytes input
 * bytes each (all views).  With chunk_planes > 0 the chunks hold chunk_planes
 * planes (the last one the rest).  With chunk_planes = 0 they are chosen
 * automatically around base = 1 GiB of input per chunk (at most ny/4
 * planes): chunks of base/8, base/4 and base/2 planes first, then equal
 * chunks of at most base planes, and a last chunk of base/4.  The iterations
 * then start after a short first copy, the last copy back is short, every
 * other copy overlaps the iterations of a neighbouring chunk, and each
 * chunk's launches run long enough that their start-up and last partial
 * wave of tiles cost little.  Volumes under 256 MiB of input (or with base
 * below 8 planes) get four equal chunks instead.  Writes chunk i as planes
 * y0[i] .. y0[i] + n[i] - 1, in order and covering 0 .. ny - 1, for at most
 * `cap` chunks.  Returns the
 * number of chunks, or -1 if an argument is invalid (ny < 1,
 * plane_bytes < 1, chunk_planes < 0, NULL arrays) or cap is too small.
 * Host only: no device work. */
int mvd_host_chunks(int ny, long long plane_bytes, int chunk_planes, int *y0, int *n, int cap);

/* Device-side status of the context's kernels.  Waits for `stream`, then
 * reads and clears the context's device status word: MVD_ERR_TIMEOUT if a
 * kernel's bounded wait for a tile copy ran out (the kernel then left its
 * tile unfinished), MVD_OK otherwise.  Kernels never hang on a lost copy:
 * every wait spins for at most the context's wait budget. */
mvd_status mvd_device_status(mvd_ctx *ctx, void *stream);

/* Clock cycles a kernel may wait for one tile copy before it reports
 * MVD_ERR_TIMEOUT (default 2e9, about one second); 0 restores the default.
 * A negative value injects the fault: every tile wait reports a timeout once
 * its copy has landed, so the error path can be tested without a real one. */
mvd_status mvd_set_wait_budget(mvd_ctx *ctx, long long cycles);

/* ---- Batches of independent volumes -------------------------------------
 * Planes are independent (Results section), and so are volumes: a batch runs
 * many volumes of uneven plane size, plane count, view count, PSF size and
 * iteration count as one unit.  Its whole schedule (reslicing, means,
 * iterations of every volume) is captured once into a CUDA graph in which
 * every volume is its own branch, and replayed by each mvd_batch_run. */
typedef struct {
    int views;                /* V                                             */
    int psf_size;             /* K (odd)                                       */
    const float *psfs_host;   /* [V][K][K], copied at mvd_batch_create         */
    int plane_h, plane_w;     /* H (rows = z), W (columns = x)                 */
    int n_planes;             /* P (= the stacks' Y)                           */
    int iters;                /* RL iterations of this volume                  */
    const void *stacks_dev;   /* [V][H][P][W] view stacks to reslice, or NULL  */
    const void *planes_dev;   /* [V][P][H][W] planes, used if stacks_dev==NULL */
    float *estimate_dev;      /* [P][H][W] FP32 result (per-plane mean start)  */
    int variant;              /* mvd_variant of this volume                   */
} mvd_volume_desc;

typedef struct mvd_batch mvd_batch;

/* Create a batch (one internal context per volume, with all of its device
 * workspace, plus planes buffers for volumes given as stacks).  Descriptors
 * are copied; the device buffers they name must stay valid while the batch
 * is used.  dt, boundary, eps and order apply to every volume. */
mvd_status mvd_batch_create(mvd_batch **out, const mvd_volume_desc *vols, int n_volumes, mvd_dtype dt,
                            mvd_boundary boundary, float eps, mvd_update_order order);

/* Autotune the batch's launch shape: every candidate (all volumes as
 * concurrent graph branches or one after another; persistent grids of one
 * resident wave or half of one) is captured and timed on `stream`, the
 * fastest kept.  With the environment variable MVD_TUNE_CACHE naming a file,
 * choices are read from and appended to it, keyed by the batch's shapes.
 * Runs the batch's work while timing (results are recomputed by every run). */
mvd_status mvd_batch_tune(mvd_batch *b, void *stream);

/* Run the batch: capture its graph on first use, then launch it on
 * `stream` (asynchronous). */
mvd_status mvd_batch_run(mvd_batch *b, void *stream);

/* Launch shape in use: concurrent (1) or serial (0) branches, the
 * persistent-grid cap per launch (0 = one resident wave) and the number of
 * kernel nodes in the graph (0 before the first run). */
mvd_status mvd_batch_info(const mvd_batch *b, int *concurrent, int *max_ctas, int *graph_kernels);

/* Schedules of a batch.
 * MVD_BATCH_GRAPH: every volume is its own graph branch of per-iteration
 *   kernel launches (1 + 2 * iters per volume and view group).
 * MVD_BATCH_QUEUE: the volumes on the fused separable route (PSFs of rank
 *   low enough for it, K <= 47) run as ONE persistent launch per PSF-size
 *   class (K <= 17, <= 31, <= 47; factors padded with zero taps) over a
 *   device-side queue of (phase, volume, plane, tile) work items, where a
 *   phase is one half (blur/ratio or correlate/update) of an iteration's
 *   view group (Supp. Note 1 update).  Items are taken in phase order from
 *   an atomic counter; before reading, an item waits until every tile of its
 *   plane has finished the previous phase (a per-plane counter in device
 *   memory).  The waits are bounded by the batch's wait budget; an expired
 *   wait sets MVD_ERR_TIMEOUT in the batch's status word and every CTA of the
 *   launch leaves.  The other volumes (Fourier or other routes) stay graph
 *   branches.  Reslicing and the per-plane means run before the queue
 *   launches in the same graph.
 * mvd_batch_tune times both and keeps the faster; these calls override or
 * read the choice (the graph is recaptured on the next run). */
typedef enum { MVD_BATCH_GRAPH = 0, MVD_BATCH_QUEUE = 1 } mvd_batch_schedule;
mvd_status mvd_batch_set_schedule(mvd_batch *b, int schedule);
/* schedule in use, volumes on the queue and their work items in total. */
mvd_status mvd_batch_queue_info(const mvd_batch *b, int *schedule, int *queue_volumes, long long *queue_items);
/* Clock cycles one queue wait may spin before it reports a timeout (0: the
 * default, about one second).  A negative budget makes every wait report a
 * timeout once its counter is reached: a test hook for the error path. */
mvd_status mvd_batch_set_wait_budget(mvd_batch *b, long long cycles);
/* Synchronise the calling thread with the device, then read and clear the
 * batch's status word: MVD_ERR_TIMEOUT after an expired queue wait. */
mvd_status mvd_batch_device_status(mvd_batch *b);

mvd_status mvd_batch_destroy(mvd_batch *b);

/* PSF calibration: the Poisson data fit of the deconvolved estimate and its
 * gradient with respect to every PSF entry.  The forward map is the
 * context's `iters` simultaneous-order MV-RL iterations (Supp. Note 1) from
 * the per-plane mean on n_planes planes of data_dev [V][P][H][W]; the loss is
 *     L = sum_planes sum_v sum_x [ y_v(x) - phi_v(x) log max(y_v(x), eps) ],
 *     y_v = P_v * psi_T
 * (Poisson negative log-likelihood without constants).  The paper has no
 * calibration step; this differentiates its iteration.  The gradient is
 * taken with respect to the raw entries (non-negativity and normalisation
 * are the optimiser's projection) by a hand-written reverse sweep; psi is
 * kept every `checkpoint_every` iterations and each segment is recomputed
 * before it is swept.  Tile sums are FP32, their combination FP64.
 *   loss_host    receives L (may be NULL)
 *   grad_dev     [V][K][K] FP32, receives dL/dP; NULL computes the loss
 *                alone (forward iterations and data fit, no reverse sweep)
 *   estimate_dev [P][H][W] FP32 or NULL: receives psi_T
 * Uses the context's PSFs, boundary and eps with direct K x K stencils
 * (K <= 63).  MVD_ERR_UNSUPPORTED for the sequential update order and for a
 * variant other than INDEPENDENT (the gradient does not follow X_v).  Returns
 * after the result is on the host (waits for `stream`). */
mvd_status mvd_psf_grad(mvd_ctx *ctx, const void *data_dev, mvd_dtype dt, int n_planes,
                        int checkpoint_every, double *loss_host, float *grad_dev,
                        float *estimate_dev, void *stream);

/* 3D MV-RL for views turned about the rotation axis, against which the
 * plane-wise approximation (Results; Fig. 1a; compared with 3D deconvolution
 * in Supp. Figs. 3-4) can be measured: view v's PSF becomes
 * a_v(y) P_v(z, x), the in-plane PSF times a profile along the axis, and
 * the planes of one mvd_deconvolve_planes call are consecutive positions on
 * the axis (planes outside the call are zero, or wrapped for the circular
 * boundary).  axial_host [V][axial_size] FP32 (copied), odd length 1..127,
 * entries >= 0 with a positive sum; NULL or 0 clears (plane-wise, the
 * default; a centred delta profile gives the plane-wise result).  The
 * in-plane passes run in the fused kernels and the axial passes in their
 * own kernels; other routes, weights, mvd_run_host, mvd_psf_grad and a given
 * initial estimate return MVD_ERR_UNSUPPORTED. */
mvd_status mvd_set_axial_psfs(mvd_ctx *ctx, const float *axial_host, int axial_size);

/* Weighted MV-RL (the "weights" array of Supp. Note 1's memory table, 4 B
 * per pixel and view; the paper gives no formula for them).  weights_dev
 * [V][n_planes][H][W] FP32 (device memory, kept by pointer, not copied; it
 * must stay valid while deconvolutions use it) holds one weight per view and
 * pixel of the planes later passed to mvd_deconvolve_planes, which must then
 * have exactly n_planes planes; n_planes = 1 gives one weight plane per view
 * that serves every plane of any call.  Each view's factor of the update becomes
 *     c_v = ((w_v phi_v / max(psi * P_v, eps)) (*) P_v^*) / n_v,
 *     n_v = w_v (*) P_v^*  (recomputed at every call),
 * the EM update of a Poisson likelihood whose pixels count with weight w_v,
 * and c_v = 1 where n_v < 1e-6 (no weighted pixel in reach).  Unit weights,
 * normalised PSFs and the circular boundary give the unweighted update.
 * Zero weights mark pixels without data: with mvd_embed_padded this is the
 * estimate on the data + PSF padded domain (Supp. Table 1 caption).  Runs on
 * the fused, plain and direct routes (MVD_ERR_UNSUPPORTED on the Fourier and
 * tensor-core routes, mvd_run_host and mvd_psf_grad).  NULL clears. */
mvd_status mvd_set_weights(mvd_ctx *ctx, const float *weights_dev, int n_planes);

/* Padded domain: src [V][n_planes][H][W] (dt, device) -> dst
 * [V][n_planes][H+2pad][W+2pad] with the planes in the centre and zeros
 * around; weights (FP32 [V][weight_planes][H+2pad][W+2pad], weight_planes 1
 * or n_planes, may be NULL) 1 on the data, 0 in the padding.  pad >= R gives
 * the estimate room for the PSF; a padded width that is a multiple of 4 (16)
 * keeps the fused kernels on TMA (vector) loads.  Buffers must not overlap.
 * Asynchronous on `stream`. */
mvd_status mvd_embed_padded(const void *src_dev, mvd_dtype dt, int views, int n_planes, int plane_h,
                            int plane_w, int pad, void *dst_dev, float *weights_dev, int weight_planes,
                            void *stream);

/* src [n_planes][padded_h][padded_w] FP32 -> dst [n_planes][padded_h-2pad]
 * [padded_w-2pad], the centre of each plane.  Asynchronous on `stream`. */
mvd_status mvd_crop_planes(const float *src_dev, int n_planes, int padded_h, int padded_w, int pad,
                           float *dst_dev, void *stream);

/* Replace the context's PSFs (same views and size), e.g. after an optimiser
 * step of PSF calibration; same checks as mvd_create. */
mvd_status mvd_set_psfs(mvd_ctx *ctx, const float *psfs_host);

/* Fused deconvolution that allocates no GPU memory.  The paper has no
 * counterpart; this exists for callers that may not call cudaMalloc, such as
 * acquisition software deconvolving while a camera records (an allocation can
 * stall the device and has no latency bound) or a plug-in inside an
 * application that owns every byte of the GPU's memory.  It takes the
 * arguments of mvd_create and mvd_deconvolve_planes together, needs no
 * context, and runs the fused path (simultaneous order, default rank
 * tolerance) with all its scratch in one library-owned static device array
 * of 32 MiB (status word, per-plane means and the V ratio planes of every
 * plane; the factor taps travel in the kernels' parameter blocks).  Every
 * GPU that loads the library holds that array until the process exits.
 *   - Limits: views <= 8, K odd and <= 47, and
 *     256 + 4*n_planes + 4*V*n_planes*H*W bytes (the first two parts rounded
 *     up to 256) must fit in 32 MiB; larger calls fail with MVD_ERR_ARG and a
 *     message giving the bytes needed (split the planes over several calls).
 *   - The first call on a device looks up the array's device address with
 *     cudaGetSymbolAddress; make that first call before any stream capture.
 *   - Every call shares the one array and reuses what the last call left
 *     there; calls whose work overlaps on the GPU (other streams, other host
 *     threads) race.  Serialise them.
 *   - The call clears the status word at the start of the array; a tile
 *     wait that runs out sets it, and the call still returns MVD_OK (the
 *     result is then incomplete).  mvd_static_device_status reads it.
 * data_dev, estimate_dev, init_mean and stream mean what they mean for
 * mvd_deconvolve_planes; the other arguments what they mean for mvd_create
 * (MVD_ERR_ARG for a negative or non-finite PSF entry or a PSF with
 * sum <= 0). */
mvd_status mvd_deconvolve_planes_static(int views, const float *psfs_host, int psf_size,
                                        int plane_h, int plane_w, int iters,
                                        mvd_boundary boundary, float eps,
                                        const void *data_dev, mvd_dtype dt,
                                        float *estimate_dev, int n_planes, int init_mean,
                                        void *stream);

/* Device-side status of the last mvd_deconvolve_planes_static call on the
 * current device (no counterpart in the paper): waits for `stream`, then
 * reads and clears the status word in the static array.  MVD_ERR_TIMEOUT if
 * a tile wait of that call ran out (its estimate is incomplete), MVD_OK
 * otherwise.  Allocates nothing. */
mvd_status mvd_static_device_status(void *stream);

/* Clock cycles a tile wait of mvd_deconvolve_planes_static may spin before
 * it gives up and sets the status word (default 2e9, about one second;
 * 0 restores it).  A negative value injects the fault, as for
 * mvd_set_wait_budget.  Applies to every later static call in the process. */
mvd_status mvd_static_set_wait_budget(long long cycles);

/* Per-kernel device time of this context's launches, taken with CUDA events
 * recorded on the launching stream around every kernel.  Enabling (on != 0)
 * or disabling clears what was collected.  mvd_profile_read waits for the
 * recorded events, then fills up to `capacity` entries (one per kernel
 * name) and sets *count to the number of names. */
typedef struct {
    char name[32];
    double total_ms;
    uint64_t launches;
} mvd_kernel_stat;

mvd_status mvd_profile_enable(mvd_ctx *ctx, int on);
mvd_status mvd_profile_read(mvd_ctx *ctx, mvd_kernel_stat *out, int capacity, int *count);

/* Host-only: the separable factorisation the library uses for the PSFs of
 * psfs_host [V][K][K] (FP64 one-sided Jacobi SVD, terms dropped below
 * rank_tol relative Frobenius norm).  rank_out[V] receives the terms kept
 * per view; taps_out (capacity `taps_capacity` floats, V*K*4*K suffices)
 * receives, per kept term in view order, four K-vectors: the vertical factor
 * (singular value folded in) reversed, the horizontal factor reversed, the
 * vertical factor and the horizontal factor, so that
 *     P[i][j] = sum_q u_q[i] * w_q[j]   with u_q = block 2, w_q = block 3.
 * Views with bitwise-identical PSFs share the first such view's terms, which
 * are stored once.  Needs no GPU. */
mvd_status mvd_psf_factors(const float *psfs_host, int views, int psf_size, double rank_tol,
                           int *rank_out, float *taps_out, int taps_capacity);

/* Host-only: the kernels X_v of `variant` (see mvd_variant) for the PSFs
 * psfs_host [V][K][K], written to x_out [V][K][K] (FP64 arithmetic, rounded
 * to FP32; each unit sum, INDEPENDENT included).  MVD_ERR_ARG on an invalid
 * size, variant or PSF.  Needs no GPU. */
mvd_status mvd_variant_kernels(const float *psfs_host, int views, int psf_size, mvd_variant variant,
                               float *x_out);

/* Fixed English text of a status code (a static string; never NULL).  The
 * paper's C workflow is called from a Java plugin through JNI (Supp. Note 2
 * sec. 4); this library is such a C interface, and every entry point of it
 * reports failures as an mvd_status that this turns into text. */
const char *mvd_status_string(mvd_status s);

/* Detail of the last error raised on the calling thread ("" if none). */
const char *mvd_last_error(void);

/* Number of kernels this library has launched in this process (all
 * contexts, all threads); used to count launches inside a timed region. */
uint64_t mvd_launch_count(void);

/* Test hook for the out-of-memory paths (no counterpart in the paper): the
 * next n device allocations the library makes, in any context, fail as if
 * cudaMalloc had returned cudaErrorMemoryAllocation, so the calls that
 * needed them return MVD_ERR_NOMEM.  A buffer that was to grow is released
 * first, as on a real failure; the context stays usable and allocates again
 * on a later call.  0 clears.  MVD_ERR_ARG for n < 0.  Needs no GPU. */
mvd_status mvd_debug_fail_allocations(int n);

#ifdef __cplusplus
}
#endif

#endif /* MVD_H */
