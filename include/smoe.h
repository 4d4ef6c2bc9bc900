/*
 * smoe.h -- C ABI of libsmoe.so: rasterised Steered Mixture of Experts (SMoE)
 * image regression on one NVIDIA GB300 GPU (sm_103a).
 *
 * Method (arXiv 2510.05814, "Rasterized Steered Mixture of Experts for
 * Efficient 2D Image Regression"):
 *   steered kernel   K_k(x) = exp(-1/2 (x-mu_k)^T L_k L_k^T (x-mu_k))   Eq. 2
 *   softmax gate     w_k(x) = K_k(x) / sum_i K_i(x)   (pi_k = 1)          Eq. 4
 *   regression       y(x)   = sum_{k in K_n} m_k(x) w_k(x)                Eqs. 3, 5
 * where K_n is the list of kernels whose bounding box touches the tile n that
 * holds x (Sec. IV-B "geometry shader", Sec. IV-C subset selection), and each
 * kernel's support is truncated to q = ||L_k^T (x-mu_k)||^2 <= q_max (Sec. IV).
 * The parameters are fitted by Adam on the MSE through the rasteriser
 * (Sec. III-D, Sec. VI-B).  Resampling the fitted model on a finer raster is
 * the native super-resolution of Sec. II-B / VII-C.
 *
 * Conventions shared by every entry point
 *   - Pixel (i, j) is column i, row j; its centre is (i + 0.5, j + 0.5).
 *   - Images are FP32, channel-planar C x H x W, contiguous.
 *   - Parameters are FP32 structure-of-arrays (smoe_params): mu[K][2] in
 *     normalised [0,1] image units (centre in pixels = mu * (W, H)),
 *     chol[K][3] = (a, b, c) of L = [[a, 0], [b, c]] in pixel units of the
 *     fitted raster, ea[K][C] expert offsets, eW[K][C][2] expert slopes
 *     (linear experts m(x) = ea + eW (x - mu)); eW is NULL for constant
 *     experts.  The sign of a and c is free (L L^T does not see it).
 *   - Truncation predicate, evaluated in FP32 with one rounding per step:
 *       dx = x0 - mx, dy = y0 - my, t = b*dy, z0 = fma(a, dx, t),
 *       z1 = c*dy, q32 = fma(z0, z0, z1*z1);  included <=> q32 <= q_max.
 *     A pixel with no included kernel renders 0 and has 1/D = 0.
 *   - Bounding box: a square centred on mu with half side
 *     r = sqrt(q_max * lambda_max(Sigma)) * (1 + 2^-10), clamped to the image
 *     in tiles (Sec. IV-B, Fig. 3b); a kernel whose box is degenerate
 *     (det = 0 or non-finite) is listed in every tile; a kernel with a
 *     non-finite parameter is listed in none.
 *   - Tile lists are CSR: tile_off[n_tiles + 1] (int32) and pair_k[] (int32),
 *     tiles in row-major order, kernel ids ascending inside every tile.  The
 *     lists are unique, so they are bit-exact across runs.
 *
 * Ownership and errors
 *   - Every pointer argument marked (device) is GPU memory that the caller
 *     owns; the library never allocates or frees device memory and never
 *     synchronises except in smoe_get_status.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).
 *   - Argument errors and launch failures are returned synchronously.
 *     Data-dependent failures (a pair count above pair_cap) are written to
 *     the device status word (int32, 0 = OK) and every later kernel that sees
 *     a non-zero status returns without work, so a captured CUDA graph stops
 *     cleanly; read it with smoe_get_status.
 */
#ifndef SMOE_H
#define SMOE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SMOE_API __attribute__((visibility("default")))
#else
#define SMOE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SMOE_OK = 0,
    SMOE_ERR_ARG = 1,        /* bad argument (sizes, NULL, alignment) */
    SMOE_ERR_CAPACITY = 2,   /* pair count above pair_cap (device status) */
    SMOE_ERR_CUDA = 3,       /* a CUDA call or launch failed */
    SMOE_ERR_TIMEOUT = 4,    /* reserved: no kernel of this library waits on another
                                (the persistent launch takes tiles from an atomic
                                counter), so none returns it */
    SMOE_ERR_WORKSPACE = 5   /* workspace too small or misaligned */
} smoe_status;

/* One raster. */
typedef struct {
    int32_t W, H;     /* raster size in pixels (the output raster for a render) */
    int32_t C;        /* channels: 1 or 3 */
    int32_t tile;     /* tile side in pixels: 8, 16 or 32 (Sec. IV-C uses 16) */
    int32_t expert;   /* 0 = constant experts, 1 = linear experts */
    float qmax;       /* truncation radius q_max (Mahalanobis, squared); 9 = 3 sigma;
                         at most 174, so that exp(-q/2) of every included pair is a
                         normal FP32 number (larger values: SMOE_ERR_ARG) */
    float scale;      /* resampling scale s >= 0: L' = L / s, eW' = eW / s; 1 for a fit */
    int32_t gate;     /* 0 = SMoE softmax gates (Eq. 4): y = N / D;
                         1 = RBF / Gaussian-splatting regression (Eq. 1): y = N, D = 1 */
} smoe_desc;

/* Parameters (or gradients, or Adam moments) of K kernels, all device SoA. */
typedef struct {
    int64_t K;
    float *mu;        /* K x 2 */
    float *chol;      /* K x 3 */
    float *ea;        /* K x C */
    float *eW;        /* K x C x 2, NULL for constant experts */
    float *logpi;     /* K gate weights log pi_k (Eq. 4: pi_k = exp(logpi_k)), or NULL
                         for pi = 1.  Gradients and moments carry it when p does. */
} smoe_params;

/* Library version, (major << 16) | minor. */
SMOE_API int32_t smoe_version(void);

/* Bytes of device workspace that smoe_bin / smoe_render /
 * smoe_render_backward need for this raster, K kernels and pair_cap pairs.
 * The workspace must be 256-byte aligned. */
SMOE_API smoe_status smoe_workspace_size(const smoe_desc *d, int64_t K, int64_t pair_cap,
                                size_t *bytes);

/* Geometry shader + subset kernel selection (Sec. IV-B, IV-C; Eq. 5).
 * For every kernel: transform to output-pixel units, bounding box, tile
 * rectangle; then a counting sort of (tile, kernel) pairs by tile: per-tile
 * counts, an exclusive prefix sum (tile_off), an atomic scatter and a per-tile
 * sort that restores ascending kernel order.  Also leaves the kernels'
 * prepared records in `ws` for smoe_render / smoe_render_backward.
 *   p          parameters (device SoA, K = p->K)
 *   ws         workspace (device, smoe_workspace_size bytes)
 *   tile_off   out: n_tiles + 1 int32 (device)
 *   pair_k     out: pair_cap int32 (device)
 *   n_pairs    out: one int64, the total pair count P (device)
 *   status     in/out: one int32 (device); set to SMOE_ERR_CAPACITY if
 *              P > pair_cap (the lists are then not written) */
SMOE_API smoe_status smoe_bin(const smoe_desc *d, const smoe_params *p, void *ws, size_t ws_bytes,
                     int32_t *tile_off, int32_t *pair_k, int64_t pair_cap,
                     int64_t *n_pairs, int32_t *status, void *stream);

/* Forward render per tile (Eqs. 2-5): y_c = N_c / D with N_c = sum e m_c,
 * D = sum e over the tile's list, e = pi exp(-q/2) [q32 <= q_max] (d->gate = 1:
 * y_c = N_c, Eq. 1).  FP32 accumulation.  Reads the prepared records that smoe_bin left in `ws` (same
 * desc and parameters).
 *   y      out: C x H x W (device)
 *   inv_d  out: H x W, 1/D (0 where D = 0), or NULL (device)
 *   status in: skipped when non-zero (device) */
SMOE_API smoe_status smoe_render(const smoe_desc *d, int64_t K, const void *ws, size_t ws_bytes,
                        const int32_t *tile_off, const int32_t *pair_k,
                        float *y, float *inv_d, const int32_t *status, void *stream);

/* Backward of smoe_render (the gradient-descent fit through the rasteriser,
 * Sec. III-D): gradients of a loss L w.r.t. mu, chol, ea, eW and, when
 * grad->logpi is set, the gate weights logpi (Eq. 4; at pi = 1 when p->logpi
 * is NULL), ADDED into `grad` (caller zeroes it).  Upstream: gy = dL/dy
 * (C x H x W) or, if gy is NULL, the MSE sum((y - target)^2) / (C H W)
 * against `target`.  Gates are recomputed from the lists; y and inv_d are the
 * outputs of smoe_render with the same desc (d->gate = 1: the RBF sum of
 * Eq. 1, whose gradient has no -y term).  Per-kernel partial sums are
 * accumulated with atomics in `ws`, so the result is deterministic only up to
 * FP32 summation order. */
SMOE_API smoe_status smoe_render_backward(const smoe_desc *d, const smoe_params *p, void *ws,
                                 size_t ws_bytes, const int32_t *tile_off,
                                 const int32_t *pair_k, const float *y, const float *inv_d,
                                 const float *gy, const float *target,
                                 const smoe_params *grad, const int32_t *status,
                                 void *stream);

/* Adam (Sec. VI-B), torch semantics, FP32 state, one fused launch over the
 * parameter groups; zeroes g.  1 - b1, 1 - b2 and the bias corrections
 * are formed in FP64 and rounded once.  lr = {mu, chol, ea, eW, logpi}; step >= 1
 * is the 1-based step used for the bias corrections.  C is the channel count
 * (sizes of ea / eW).  eW pointers must all be NULL or all non-NULL, and so must
 * the logpi pointers. */
SMOE_API smoe_status smoe_adam_step(const smoe_params *p, const smoe_params *g, const smoe_params *m,
                           const smoe_params *v, int32_t C, const float lr[5], double b1,
                           double b2, double eps, int32_t step, void *stream);

/* Sum of squared differences over n floats, FP64 accumulation, ADDED to
 * *out (device); with clamp != 0, y is clamped to [0, 1] first (the PSNR
 * convention). */
SMOE_API smoe_status smoe_sq_error(const float *y, const float *target, int64_t n, int32_t clamp,
                          double *out, void *stream);

/* ------------------------------------------------------------------------ */
/* Fit: a batch of B images (B = 1 for a single image), one iteration =      */
/* bin -> fused forward/backward per tile (MSE) -> finalize + Adam.          */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t W, H;           /* image size */
    const float *target;    /* C x H x W (device) */
    smoe_params p;          /* this image's parameters (device SoA, K = p.K), updated in place */
    smoe_params m, v;       /* its Adam moments (device SoA, same K) */
    int32_t iters;          /* length of this image's run (lr schedule, loss history) */
    float lr_mu0, lr_mu1;   /* centre rate, decayed exponentially lr_mu0 -> lr_mu1 */
    float lr_chol, lr_ea, lr_eW;
    float lr_pi;            /* rate of the gate weights (used when p.logpi is set) */
} smoe_fit_image;

typedef struct {
    int32_t B;              /* images */
    int32_t C, tile, expert;
    float qmax;
    double b1, b2, eps;     /* Adam (1 - b and the bias corrections are formed in FP64) */
    int32_t *step;          /* device, B: iterations done per image (caller-owned) */
    double *loss;           /* device, B x hist: MSE per image and iteration, or NULL */
    int32_t hist;           /* columns of `loss` */
    int32_t persistent;     /* 1: the fused tile kernel runs as one persistent grid that
                               takes tiles from a work queue; 0: one CTA per tile */
    int32_t deterministic;  /* 1: every (tile, kernel) pair writes its partial gradient
                               sums to its own slot and the Adam step adds a kernel's
                               slots in row-major tile order (through an index of them
                               the binning builds), so a fit is bit-reproducible and
                               independent of the other images in the batch (costs 68 B
                               per pair and 8 B per kernel of workspace; at most
                               16.7 M kernels in the batch); 0: float atomics (faster,
                               order-dependent) */
    int32_t gate;           /* as smoe_desc.gate: 0 softmax gates, 1 RBF sum */
} smoe_fit_batch;

/* Workspace bytes for a fit of this batch with pair_cap pairs in total. */
SMOE_API smoe_status smoe_fit_workspace_size(const smoe_fit_batch *batch, const smoe_fit_image *imgs,
                                    int64_t pair_cap, size_t *bytes);

/* Images keep their own parameter tensors, so a batch can be re-formed (an
 * image added or retired) without moving any parameters: build the new
 * batch and call smoe_fit_init with reset = 0 to continue the others' runs.
 *
 * Prepare a fit: writes the batch table into `ws` (one host-to-device copy
 * on `stream`, after which the stream is synchronised once) and zeroes the
 * workspace's gradient sums.  With reset != 0 it also zeroes the Adam moments
 * m and v, the step counters, the loss history and the status word, i.e.
 * starts every image's run from iteration 0; with reset == 0 a run continues
 * (e.g. after re-initialising with a larger pair_cap).  Call outside stream
 * capture. */
SMOE_API smoe_status smoe_fit_init(const smoe_fit_batch *batch, const smoe_fit_image *imgs,
                          int64_t pair_cap, void *ws, size_t ws_bytes, int32_t reset,
                          int32_t *status, void *stream);

/* Run n_iters fit iterations of the batch prepared in `ws` by smoe_fit_init
 * with the same batch, imgs and pair_cap.  One iteration = binning of all
 * images' kernels, one fused forward/MSE/backward launch over all tiles of all
 * images (a ragged tile table), and one fused finalize + Adam launch.  No host
 * synchronisation, so iterations can be captured in a CUDA graph and
 * replayed.  Image b stops updating after imgs[b].iters iterations; the MSE
 * of its iteration i (before that iteration's update) is written to
 * loss[b * hist + i] when i < hist. */
SMOE_API smoe_status smoe_fit(const smoe_fit_batch *batch, const smoe_fit_image *imgs, int64_t pair_cap,
                     void *ws, size_t ws_bytes, int32_t n_iters, int32_t *status,
                     void *stream);

/* One phase of one fit iteration (the iteration of smoe_fit is phases 0, 1,
 * 2 in this order): 0 = binning of all images' kernels, 1 = the fused
 * forward / MSE / backward launch over the ragged tile table, 2 = finalize +
 * Adam (advances the step counters).  Lets a caller place or time the phases
 * separately; the three in order are exactly one smoe_fit iteration. */
SMOE_API smoe_status smoe_fit_phase(const smoe_fit_batch *batch, const smoe_fit_image *imgs,
                                    int64_t pair_cap, void *ws, size_t ws_bytes, int32_t phase,
                                    int32_t *status, void *stream);

/* The gradients of one fit iteration (Sec. III-D: gradient descent through
 * the rasteriser), read out instead of applied: bins the batch's current
 * parameters (phase 0), runs the fused forward / MSE / backward launch over
 * the ragged tile table (phase 1, with the batch's persistent and
 * deterministic settings), and turns every kernel's sums into dL/dtheta of
 * that image's MSE, sum((y - target)^2) / (C H W), by the same device code
 * the Adam launch of phase 2 uses, writing them to `grad` instead of
 * updating the parameters.  Parameters, Adam moments, step counters and the
 * loss history are left as they are, and the workspace's gradient sums are
 * zero again afterwards, so the fit can continue with smoe_fit.
 *   batch, imgs, pair_cap, ws, ws_bytes: as smoe_fit_phase, after
 *              smoe_fit_init on this workspace
 *   grad       out: one parameter set of K_total = sum_b imgs[b].p.K rows
 *              (device SoA), image b's kernels at rows sum_{b' < b} K_b' ..,
 *              in the order of the batch's parameter arrays; mu in the
 *              normalised units of smoe_params; eW set iff the experts are
 *              linear; logpi optional (when set: dL/dlogpi, at pi = 1 for
 *              images without gate weights).  Kernels of an image whose run
 *              has ended (step >= iters) get 0.
 *   status     device status word: a pair count above pair_cap sets
 *              SMOE_ERR_CAPACITY and grad is then not written
 * Returns SMOE_ERR_ARG for a grad whose K or groups do not match. */
SMOE_API smoe_status smoe_fit_gradients(const smoe_fit_batch *batch, const smoe_fit_image *imgs,
                                        int64_t pair_cap, void *ws, size_t ws_bytes,
                                        const smoe_params *grad, int32_t *status, void *stream);

/* Multi-model fusion for denoising (Sec. V-C, Eq. 11): y_m = (1/H) sum_h y_h,
 * the per-pixel mean of the renders of the H = batch->B models of a fit
 * batch whose images all have one size W x H (the H models of MM-RSMoE are
 * fits of one noisy image from differently shifted initial kernel lattices).
 * The call bins the models' current parameters (as phase 0 does, into the
 * batch's lists) and renders the mean in one launch, one CTA per output tile
 * visiting the H models in index order: y_h is exactly what smoe_render
 * gives for model h (0 where no kernel of model h is included), and H = 1
 * returns that render bit for bit.
 *   batch, imgs, pair_cap, ws, ws_bytes: as smoe_fit_phase, after
 *                smoe_fit_init on this workspace
 *   y            out: C x H x W FP32 (device)
 *   status       device status word: a pair count above pair_cap sets
 *                SMOE_ERR_CAPACITY and y is then not written
 * Returns SMOE_ERR_ARG if the images differ in size. */
SMOE_API smoe_status smoe_fit_render_mean(const smoe_fit_batch *batch, const smoe_fit_image *imgs,
                                          int64_t pair_cap, void *ws, size_t ws_bytes, float *y,
                                          int32_t *status, void *stream);

/* Spatial reordering of a fit batch's kernels (an aid to the tile binning
 * of Sec. IV-C, not part of the method).  The fit moves kernel centres, so
 * after some iterations kernels with consecutive indices are no longer
 * neighbours and the binning's per-warp aggregation and run merge stop
 * applying.  This call permutes each image's kernels into tile-major order
 * of their current centres (centres outside the raster clamp to the nearest
 * edge tile, non-finite ones go last), ascending current index within a
 * tile: the parameters and both Adam moments of every group move together,
 * kernels stay in their image, and the order is a function of the centres
 * alone.  The model is the same set of kernels; later renders and gradients
 * differ from those of the unpermuted model only in the order of the FP32
 * sums over kernels.
 *   batch, imgs, pair_cap, ws, ws_bytes: as smoe_fit_phase, after
 *                smoe_fit_init on this workspace; call between iterations
 *                (the next iteration rebins)
 *   order        in/out, optional: K_total int32 (device), slot -> the
 *                kernel's index in the caller's original order, permuted
 *                with the kernels (initialise to 0 .. K_total-1; slots of
 *                image b keep values in its own range)
 *   status       device status word: when it is already set the call
 *                changes nothing */
SMOE_API smoe_status smoe_fit_reorder(const smoe_fit_batch *batch, const smoe_fit_image *imgs,
                                      int64_t pair_cap, void *ws, size_t ws_bytes,
                                      int32_t *order, int32_t *status, void *stream);

/* Row scatter of a parameter set: dst row (index[i] - base) <- src row i for
 * i < src->K, in every group (mu 2, chol 3, ea C, eW 2C, logpi 1 values per
 * row) present in both sets.  Returns a reordered batch's parameters in the
 * caller's order: src = an image's slots, index = that image's range of the
 * batch's order array, base = the image's first kernel index.
 *   index: src->K int32 (device), a permutation of base .. base + K - 1
 *   dst: K rows (device, not overlapping src)
 * Returns SMOE_ERR_ARG for a negative K, C not 1 or 3, or missing arrays. */
SMOE_API smoe_status smoe_scatter_params(const smoe_params *src, const int32_t *index,
                                         int64_t base, int32_t C, const smoe_params *dst,
                                         void *stream);

/* Multi-model fusion (Sec. V-C, Eq. 11) of H separate models on any raster:
 * y = (1/H) sum_h y_h, each y_h the render of models[h] on d's W x H raster
 * at d->scale (so a denoised MM-RSMoE result can be resampled at 1-4x), in
 * one binning pass over the H models and one averaging launch; y_h is what
 * smoe_render gives for model h, and H = 1 returns that render bit for bit.
 *   models: H parameter sets (device SoA; logpi all set or all NULL)
 *   ws: smoe_render_mean_workspace_size(d, models, H, pair_cap) bytes
 *       (256-byte aligned); pair_cap bounds the (tile, kernel) pairs of all
 *       H models together
 *   y: out, C x H x W (d's raster); status: device word, zeroed by the
 *      caller; a pair count above pair_cap sets SMOE_ERR_CAPACITY and y is
 *      then not written
 * With H > 1 the call uploads the H models' table into ws and synchronises
 * the stream first (not capturable in a graph). */
SMOE_API smoe_status smoe_render_mean_workspace_size(const smoe_desc *d,
                                                     const smoe_params *models, int32_t H,
                                                     int64_t pair_cap, size_t *bytes);
SMOE_API smoe_status smoe_render_mean(const smoe_desc *d, const smoe_params *models, int32_t H,
                                      void *ws, size_t ws_bytes, int64_t pair_cap, float *y,
                                      int32_t *status, void *stream);

/* Native sharpening by kernel editing (Sec. II-B, Sec. VII-C): the kernel
 * bandwidths divided by a sharpening factor f, i.e. L' = f L (P' = f^2 P):
 * chol_out[i] = f * chol_in[i] for the 3K entries, each rounded to float
 * once, and the cutoff to render the edited model with,
 * *qmax_out = qmax * (f * f) (two FP32 products), so that each kernel keeps
 * the support of the fitted model and only the gates steepen (f > 1 sharpens
 * edges; flat regions keep their value).
 *   chol_in, chol_out: K x 3 FP32 (device); they may be the same buffer
 *   factor: finite, > 0;  qmax: the fitted model's cutoff, > 0
 *   qmax_out: out, one float (host)
 * Returns SMOE_ERR_ARG for a bad K, factor or qmax, or when q_max' exceeds
 * 174 (f <= 4.39 for q_max = 9), where the gate of a far included pair would
 * leave the FP32 range; nothing is written then. */
SMOE_API smoe_status smoe_sharpen(const float *chol_in, float *chol_out, int64_t K,
                                  float factor, float qmax, float *qmax_out, void *stream);

/* Bytes of the scratch that smoe_render_points needs for n_points points on
 * the raster of d. */
SMOE_API smoe_status smoe_points_workspace_size(const smoe_desc *d, int64_t n_points,
                                                size_t *bytes);

/* Resample the continuous regression function y(x) (Eqs. 3-5) at arbitrary
 * sample points: super-resolution to any size on a regular or an irregular
 * raster (Sec. II-B).  The model is the one smoe_bin(d, ...) prepared in ws
 * with its lists tile_off / pair_k (any d->scale; the points are in the
 * pixel units of d's W x H raster, pixel (i, j) having centre
 * (i + 0.5, j + 0.5)).  Each point is evaluated with the same truncated model
 * as smoe_render (FP32 predicate at the point's FP32 coordinates, kernels in
 * ascending order); a point outside [0, W) x [0, H) or with a non-finite
 * coordinate gets y = 0 and inv_d = 0.
 *   K, ws, ws_bytes, tile_off, pair_k: as smoe_render
 *   xy:   n_points x 2 FP32 (device, 8-byte aligned), (x, y) per point
 *   pws:  scratch of smoe_points_workspace_size bytes (256-byte aligned)
 *   y:    out, C x n_points FP32 (channel-planar); inv_d: out, n_points or NULL
 *   status: the binning's status word; nothing is written if it is nonzero
 * Returns SMOE_ERR_ARG / SMOE_ERR_WORKSPACE synchronously. */
SMOE_API smoe_status smoe_render_points(const smoe_desc *d, int64_t K, const void *ws,
                                        size_t ws_bytes, const int32_t *tile_off,
                                        const int32_t *pair_k, int64_t n_points, const float *xy,
                                        void *pws, size_t pws_bytes, float *y, float *inv_d,
                                        const int32_t *status, void *stream);

/* Diagnostic: adds to *out (device, uint64) the number of (pixel, kernel)
 * pairs of the lists whose kernel includes the pixel (q32 <= q_max, the
 * truncation of Sec. IV), i.e. the pairs that contribute to the render, as
 * against the listed pairs (sum over tiles of pixels x list length).  Same
 * arguments as smoe_render; not part of the fit. */
SMOE_API smoe_status smoe_count_inrange(const smoe_desc *d, int64_t K, const void *ws,
                                        size_t ws_bytes, const int32_t *tile_off,
                                        const int32_t *pair_k, uint64_t *out,
                                        const int32_t *status, void *stream);

/* Bin and render one model without allocating anything: for callers that
 * cannot call cudaMalloc (a plugin inside an application that owns every
 * device allocation, code that must not touch the allocator).  The paper has
 * no counterpart; it is smoe_bin followed by smoe_render with every
 * intermediate buffer in one fixed 8 MiB device array inside the library,
 * which every GPU that loads the library holds until the process exits.
 *   The raster checks are smoe_render's (SMOE_ERR_ARG, q_max <= 174 included).
 *   Limits: K <= 32768 kernels, at most 16384 tiles on the output raster
 *   (e.g. 2048x2048 at tile 16), at most 524288 (tile, kernel) pairs.
 *   Larger K or rasters are refused with SMOE_ERR_WORKSPACE before any work;
 *   a pair count above the limit sets *status = SMOE_ERR_CAPACITY on the
 *   device and y / inv_d are then not written.
 *   p      parameters (device SoA); y: C x H x W out; inv_d: H x W out or NULL
 *   status out: one int32 (device), zeroed by the call, then as smoe_bin.
 * Outside stream capture every call looks up the array's device address
 * (cudaGetSymbolAddress) on the current device, so a device reset leaves no
 * stale address; a call under capture uses the address of the last call on
 * that device outside capture, so make the first call on a device before any
 * stream capture.  All calls share the one array and it keeps the
 * last call's contents, so calls whose work overlaps on the GPU (different
 * streams, or different host threads on one device) race: serialise them.
 * The call itself allocates nothing and does not synchronise. */
SMOE_API smoe_status smoe_render_static(const smoe_desc *d, const smoe_params *p, float *y,
                                        float *inv_d, int32_t *status, void *stream);

/* Synchronise `stream` and return the device status word (SMOE_OK, or the
 * first data-dependent error), or SMOE_ERR_CUDA if the stream failed. */
SMOE_API smoe_status smoe_get_status(const int32_t *status, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SMOE_H */
