/*
 * sixdgs.h -- C ABI of the GB300 (sm_103a) differentiable 6D Gaussian render.
 *
 * The library implements the render path of 6DGS (arXiv 2410.04974):
 *   condition_project : slice each 6D Gaussian at the view direction into a
 *                       conditional 3D Gaussian (section 3.2, Eq. mu, Eq.
 *                       sigma, Eq. pdf/alpha refined by Eq. pdfv2; Algorithm 1
 *                       steps 1-3), evaluate its sigmoid-SH colour (section
 *                       4.2) and EWA-project it to a 2D conic (the 3DGS step
 *                       that section 4.4 keeps unchanged);
 *   bin_sort          : duplicate every visible Gaussian into the screen tiles
 *                       of its tile rectangle (settings.alpha_footprint: the
 *                       3-sigma square, by default intersected with the box
 *                       of its alpha >= 1/255 ellipse) and radix-sort the
 *                       (tile, depth) keys (section 4.4, inherited 3DGS step);
 *   raster_fwd        : blend every tile front to back (section 4.4), with an
 *                       optional fused L1 loss (the 3DGS loss section 4.4
 *                       keeps);
 *   raster_bwd        : the hand-written reverse of all of the above, down to
 *                       the raw 6D parameters (section 4.4: training uses the
 *                       differentiable rasteriser; gradients reach mu_p, mu_d,
 *                       the Cholesky parameters, opacity and SH).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Ownership: the caller allocates and frees every buffer, including the
 *   workspace; the library never allocates device or host memory.
 * Pointers: every pointer marked _dev is a device pointer; structs
 *   (sixdgs_plan, sixdgs_scene, sixdgs_camera arrays) live in host memory and
 *   are read during the call only.
 * Streams: every call enqueues work on `stream` and returns without
 *   synchronising.  The return value reports host-detectable errors only
 *   (bad sizes, null pointers, launch failure).  All calls are legal inside
 *   CUDA stream capture.
 * Device status: `status_dev` points to one int32 in device memory that the
 *   caller zeroes before a frame.  Kernels OR (1 << code) into it for every
 *   condition they detect (SIXDGS_ERR_CAPACITY, SIXDGS_ERR_TIMEOUT,
 *   SIXDGS_ERR_NONFINITE); read it after synchronising.
 * Order: the stages of one frame run condition_project -> bin_sort ->
 *   raster_fwd -> raster_bwd on the same plan and workspace, in stream order.
 * Layouts: per-Gaussian inputs and gradients are structure-of-arrays
 *   float32 planes of length n (plane p of array X is X[p*n .. p*n+n-1]).
 *   Images are planar float32 (3, H, W) per camera, cameras packed one after
 *   another in camera order.
 */
#ifndef SIXDGS_H
#define SIXDGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* sixdgs_stream_t; /* same object as cudaStream_t */

typedef enum sixdgs_status {
  SIXDGS_OK = 0,
  SIXDGS_ERR_INVALID_ARG = 1, /* bad size, null pointer, unsupported setting  */
  SIXDGS_ERR_CUDA = 2,        /* a CUDA launch or copy failed                 */
  SIXDGS_ERR_CAPACITY = 3,    /* more (Gaussian, tile) duplicates than the
                                 plan's dup_capacity: SIXDGS_WS_COUNTS[1]
                                 holds the required number; grow, re-run      */
  SIXDGS_ERR_TIMEOUT = 4,     /* a device-side wait ran out of its budget     */
  SIXDGS_ERR_NONFINITE = 5,   /* a Gaussian produced a non-finite value; it
                                 was culled                                   */
  SIXDGS_ERR_WORKSPACE = 6    /* workspace smaller than sixdgs_workspace_size */
} sixdgs_status;

/* Pinhole camera.  Camera axes: x right, y down, z forward.  A world point X
 * maps to t = R X + t_w with world_to_cam = [R | t_w] (row-major 3x4), and
 * to pixel coordinates (fx t_x / t_z + cx, fy t_y / t_z + cy); pixel (i, j)
 * covers [i, i+1) x [j, j+1) and is sampled at its centre (i+0.5, j+0.5).   */
typedef struct sixdgs_camera {
  int32_t width, height;
  float fx, fy, cx, cy;
  float world_to_cam[12];
  float campos[3];   /* camera centre in world space                         */
  float znear;       /* conditional means with t_z <= znear are culled       */
} sixdgs_camera;

/* A 6D Gaussian scene (section 3.1): all pointers are device SoA planes.
 *  mu_p           3 planes  position mean
 *  mu_d           3 planes  direction mean (used as given, not normalised)
 *  l_raw         21 planes  Cholesky factor L of the 6x6 covariance
 *                           Sigma = L L^T: planes 0-5 the diagonal,
 *                           L_ii = exp(raw); planes 6-20 the strictly lower
 *                           entries in row-major order (1,0) (2,0) (2,1)
 *                           (3,0) ... (5,4), L_ij = 2*sigmoid(raw) - 1
 *  opacity_logit  1 plane   alpha = sigmoid(raw)
 *  sh   (deg+1)^2*3 planes  SH coefficient beta_{k,c} in plane k*3+c, real
 *                           orthonormal basis index k = l*l + l + m, no
 *                           Condon-Shortley phase; colour = sigmoid(sum_k
 *                           beta_k Y_k(d)) (section 4.2)
 *  lambda_raw     1 plane   optional (NULL: settings.lambda_opa for all):
 *                           per-Gaussian learnable lambda_opa = sigmoid(raw),
 *                           in (0, 1) (section 4.2, Eq. pdfv2)
 *  cond_cache    25 planes  optional (NULL: computed from l_raw and
 *                           opacity_logit): the view-independent state written
 *                           by sixdgs_condition_cache for these l_raw and
 *                           opacity_logit; the projection then reads it and
 *                           ignores l_raw and opacity_logit.  The result is
 *                           bit-identical to the uncached projection.  For a
 *                           fixed scene (inference; the caption of Algorithm 1)
 *                           the state is computed once instead of every frame.
 *                           The backward never reads it.                    */
typedef struct sixdgs_scene {
  int64_t n;
  int32_t sh_degree;   /* 0..3 */
  int32_t _pad;
  const float* mu_p;
  const float* mu_d;
  const float* l_raw;
  const float* opacity_logit;
  const float* sh;
  const float* lambda_raw;
  const float* cond_cache;
} sixdgs_scene;

/* Render settings. */
typedef struct sixdgs_settings {
  int32_t tile_w;      /* screen tile width  in {8, 16, 32}                   */
  int32_t tile_h;      /* screen tile height in {8, 16}                       */
  int32_t batch;       /* list entries staged per shared-memory batch, a
                          multiple of 32 in [32, 1024] (48 bytes each)        */
  float lambda_opa;    /* Eq. pdfv2: f_cond = exp(-lambda_opa * D), [0, 1]    */
  float bg[3];         /* background colour                                   */
  int32_t store_aux;   /* 1: raster_fwd stores the per-pixel walk length and
                          raster_bwd reuses it; 0: raster_bwd recomputes it
                          (no per-pixel auxiliary buffer)                     */
  int64_t spin_budget; /* clock cycles a device-side wait may spin before it
                          reports SIXDGS_ERR_TIMEOUT; <= 0 selects the default
                          (2^31 cycles, about one second)                     */
  float loss_norm;     /* number of values the fused L1 mean divides by; <= 0
                          selects 3 * total_pixels of the plan (use the whole
                          batch's count when one batch is rendered one camera
                          per plan)                                           */
  int32_t count_pairs; /* 1: raster_fwd also counts evaluated and compositing
                          (pixel, list entry) pairs into SIXDGS_WS_COUNTS     */
  int32_t persistent;  /* 1: the blend kernels run as one resident grid whose
                          CTAs take the tiles of all cameras from a device
                          queue; 0: one CTA per tile                          */
  int32_t inference;   /* 1: forward-only plan: no gradient-record section in
                          the workspace, the projection writes no gradient
                          records, store_aux must be 0 and the backward entry
                          points return SIXDGS_ERR_INVALID_ARG                */
  int32_t alpha_footprint; /* tile rectangle of a Gaussian: 0: the 3-sigma
                          square of the 3DGS rasteriser that section 4.4 keeps;
                          1: that square intersected with the bounding box of
                          the Gaussian's alpha >= 1/255 ellipse (half-extents
                          sqrt(2 ln(255 alpha_cond) Sigma2D_ii), widened by
                          1e-4 relative + 0.01 px).  Tiles outside that box
                          hold no pixel that composites the Gaussian, so images
                          and gradients are the same with 1, and the tile lists
                          shorter (about 40% fewer duplicates at 300k / 800^2) */
  int32_t _pad;
} sixdgs_settings;

/* Sizes and workspace layout of one frame, filled by sixdgs_plan_init. */
typedef struct sixdgs_plan {
  int64_t n;              /* Gaussians                                        */
  int32_t sh_degree;
  int32_t n_cams;
  sixdgs_settings settings;
  int64_t n_pairs;        /* n_cams * n (view, Gaussian) pairs                */
  int64_t total_tiles;    /* screen tiles over all cameras                    */
  int64_t total_pixels;   /* pixels over all cameras                          */
  int64_t dup_capacity;   /* room for (Gaussian, tile) duplicates             */
  int32_t depth_passes;   /* radix passes over the depth key                  */
  int32_t tile_passes;    /* radix passes over the tile key                   */
  int64_t ws_bytes;       /* required workspace size                          */
  int64_t off[32];        /* byte offsets of the workspace sections           */
} sixdgs_plan;

/* Workspace sections (indices into sixdgs_plan.off) that callers may read
 * after synchronising, for inspection and testing. */
enum {
  SIXDGS_WS_CAMS = 0,      /* per-camera records                              */
  SIXDGS_WS_REC = 1,       /* n_pairs x 12 float: u, v, qa, qb, qc, lo, r, g,
                              b, hx, hy, depth of each (view, Gaussian):
                              log2 alpha = qa dx^2 + qb dx dy + qc dy^2 + lo,
                              (hx, hy) the alpha >= 1/255 bounding box       */
  SIXDGS_WS_NTILES = 2,    /* n_pairs x uint32 tiles touched (0 = culled)      */
  SIXDGS_WS_RECT = 3,      /* n_pairs x 4 uint16 tile rect x0, x1, y0, y1      */
  SIXDGS_WS_DEPTHKEY = 4,  /* n_pairs x uint32                                 */
  SIXDGS_WS_COUNTS = 5,    /* uint32 visible pairs, uint32 duplicates (K),
                              8 bytes unused, then (count_pairs) uint64
                              evaluated and compositing (pixel, entry) pairs
                              and uint64 (warp, entry) pairs walked          */
  SIXDGS_WS_SORTED = 6,    /* dup_capacity x uint32 pair index, sorted by
                              (global tile, depth, Gaussian id)               */
  SIXDGS_WS_RANGES = 7,    /* total_tiles x uint32[2] [start, end) in SORTED  */
  SIXDGS_WS_NWALK = 8,     /* total_pixels x uint32 list entries walked       */
  SIXDGS_WS_GRADREC = 9,   /* n_pairs x 12 float: sums over pixels of g, g dx,
                              g dy, g dx^2, g dx dy, g dy^2 (g = dL/dq / ln 2)
                              and dL/d(r, g, b) of each (view, Gaussian)     */
  SIXDGS_WS_SORTEDKEY = 10 /* dup_capacity x uint32 global tile of SORTED     */
};

/* Library version, "major.minor.patch". */
const char* sixdgs_version(void);

/* Human-readable name of a status code. */
const char* sixdgs_status_string(int32_t status);

/* Fill `plan` for a frame of n Gaussians seen by n_cams cameras.
 * cams: host array of n_cams cameras (only sizes are read here).
 * dup_capacity: room for (Gaussian, tile) duplicates; <= 0 picks
 *   4 * n_pairs + 4096.  Limits: 1 <= n_cams <= 256, n_cams * n < 2^31,
 *   dup_capacity < 2^30, at most 65535 tiles per image side.
 * Errors: SIXDGS_ERR_INVALID_ARG. */
sixdgs_status sixdgs_plan_init(int64_t n, int32_t sh_degree,
                               const sixdgs_camera* cams, int32_t n_cams,
                               const sixdgs_settings* settings,
                               int64_t dup_capacity, sixdgs_plan* plan);

/* Bytes of device workspace a frame with this plan needs (16-byte aligned
 * base required). */
size_t sixdgs_workspace_size(const sixdgs_plan* plan);

/* Stage 1 -- slice, colour and project (section 3.2 Eqs. mu/sigma/alpha with
 * Eq. pdfv2, section 4.2, section 4.4).  For every Gaussian: L from l_raw,
 * Sigma = L L^T, Sigma_d^-1 (3x3 Cholesky), A = Sigma_pd Sigma_d^-1 and the
 * Schur complement Sigma_cond = Sigma_p - A Sigma_pd^T, computed once; then
 * for every camera: d = normalize(mu_p - campos), mu_cond = mu_p +
 * A (d - mu_d), D = (d-mu_d)^T Sigma_d^-1 (d-mu_d), alpha_cond =
 * sigmoid(logit) exp(-lambda_opa D), colour, EWA conic and the tile rect
 * (the 3-sigma square, intersected with the alpha >= 1/255 box when
 * settings.alpha_footprint = 1).
 * cams: host array of plan->n_cams cameras; their values are copied into the
 * workspace through kernel parameters (and so into a captured graph).
 * Errors: INVALID_ARG, WORKSPACE, CUDA; device: NONFINITE. */
sixdgs_status sixdgs_condition_project(const sixdgs_plan* plan, const sixdgs_scene* scene,
                                       const sixdgs_camera* cams, void* ws_dev,
                                       size_t ws_bytes, int32_t* status_dev,
                                       sixdgs_stream_t stream);

/* Stage 2 -- binning and sort (section 4.4).  Visible (view, Gaussian) pairs
 * are radix-sorted by depth (stable, so equal depths keep Gaussian-id
 * order), duplicated once per touched tile in that order, and stably
 * radix-sorted by global tile id: an LSD sort of the composite
 * (tile, depth, id) key whose depth digits run before duplication.  Both
 * sorts are single-pass-per-digit "onesweep" sorts with decoupled look-back.
 * Writes SORTED, RANGES and COUNTS.  Device: CAPACITY, TIMEOUT. */
sixdgs_status sixdgs_bin_sort(const sixdgs_plan* plan, void* ws_dev, size_t ws_bytes,
                              int32_t* status_dev, sixdgs_stream_t stream);

/* Stage 3 -- front-to-back blend of every tile (section 4.4): per pixel,
 * alpha_i = min(0.99, alpha_cond_i exp(-1/2 Delta^T conic_i Delta)); entries
 * with alpha_i < 1/255 are skipped; the walk stops, excluding the current
 * entry, once T (1 - alpha_i) < 1e-4; C = sum_i c_i alpha_i T_i + T bg.
 * images_dev: output, total_pixels * 3 floats (planar per camera).
 * targets_dev, grad_images_dev, loss_dev: optional (all NULL or all set):
 *   fused L1 loss L = mean |C - target| over all values; grad_images receives
 *   dL/dC = sign(C - target) / (3 * total_pixels); *loss_dev (a double that
 *   the caller zeroes) accumulates L.
 * Errors: INVALID_ARG, WORKSPACE, CUDA. */
sixdgs_status sixdgs_raster_fwd(const sixdgs_plan* plan, void* ws_dev, size_t ws_bytes,
                                float* images_dev, const float* targets_dev,
                                float* grad_images_dev, double* loss_dev,
                                int32_t* status_dev, sixdgs_stream_t stream);

/* Stages 3 + 4a fused for the L1 loss (section 4.4 keeps the 3DGS losses;
 * L1 is the term used here): raster_fwd with targets, then blend_bwd of that
 * loss, in one kernel.  Each pixel's dL/dC = sign(C - target) / M (M as in
 * raster_fwd) is known when its forward walk ends, so its backward replay
 * follows in the same CTA with C, dL/dC and the walk length in registers.
 * Results equal raster_fwd (with targets) followed by sixdgs_blend_bwd, up to
 * the order of the atomic additions into the record gradients.
 * images_dev: written; targets_dev: required; grad_images_dev: optional
 * (NULL: dL/dC is not stored); loss_dev: required, accumulated as in
 * raster_fwd.  Follow with sixdgs_project_bwd for the parameter gradients.
 * The per-pair gradient records it accumulates are zeroed by
 * condition_project, so call it (or blend_bwd) once per condition_project.
 * Errors: INVALID_ARG (also for an inference plan), WORKSPACE, CUDA. */
sixdgs_status sixdgs_raster_fwd_bwd(const sixdgs_plan* plan, void* ws_dev, size_t ws_bytes,
                                    float* images_dev, const float* targets_dev,
                                    float* grad_images_dev, double* loss_dev,
                                    int32_t* status_dev, sixdgs_stream_t stream);

/* Stage 4 -- gradients of sum <grad_images, images> with respect to every
 * raw scene parameter, through the blend (replayed in sorted order, front
 * to back, with the suffix colour taken from the forward image), the
 * projection, the SH colour, the slice and the Cholesky activation.
 * Equivalent to sixdgs_blend_bwd followed by sixdgs_project_bwd.
 * images_dev: the forward output; grad_images_dev: dL/dC, same layout.
 * grad_*: outputs with the layout of the scene planes; overwritten with the
 * sum over all cameras of the plan, or added to when accumulate != 0.
 * grad_lambda_raw is used only when the scene has a lambda_raw plane (may be
 * NULL otherwise, or to skip that gradient).
 * The per-pair gradient records that this call accumulates are zeroed by
 * condition_project, so call it at most once per condition_project.
 * Errors: INVALID_ARG, WORKSPACE, CUDA. */
sixdgs_status sixdgs_raster_bwd(const sixdgs_plan* plan, const sixdgs_scene* scene,
                                void* ws_dev, size_t ws_bytes,
                                const float* images_dev, const float* grad_images_dev,
                                float* grad_mu_p, float* grad_mu_d, float* grad_l_raw,
                                float* grad_opacity_logit, float* grad_sh, float* grad_lambda_raw,
                                int32_t accumulate, int32_t* status_dev, sixdgs_stream_t stream);

/* Stage 4a -- blend backward only (section 4.4, the differentiable 3DGS
 * rasteriser): for every (view, Gaussian) pair, the gradient of
 * sum <grad_images, images> with respect to the pair's screen record
 * (2D mean, conic, alpha_cond, colour) is accumulated into the workspace
 * section SIXDGS_WS_GRADREC.  Errors: INVALID_ARG, WORKSPACE, CUDA. */
sixdgs_status sixdgs_blend_bwd(const sixdgs_plan* plan, void* ws_dev, size_t ws_bytes,
                               const float* images_dev, const float* grad_images_dev,
                               int32_t* status_dev, sixdgs_stream_t stream);

/* Stage 4b -- per-Gaussian backward of the projection, SH colour (section
 * 4.2), slice (Eq. mu, Eq. pdfv2, Eq. alpha), Schur complement (Eq. sigma)
 * and Cholesky activation (section 3.1), summed over the plan's cameras, from
 * the records that sixdgs_blend_bwd left.  grad_* as in sixdgs_raster_bwd.
 * Errors: INVALID_ARG, WORKSPACE, CUDA. */
sixdgs_status sixdgs_project_bwd(const sixdgs_plan* plan, const sixdgs_scene* scene,
                                 void* ws_dev, size_t ws_bytes, float* grad_mu_p,
                                 float* grad_mu_d, float* grad_l_raw, float* grad_opacity_logit,
                                 float* grad_sh, float* grad_lambda_raw, int32_t accumulate,
                                 int32_t* status_dev, sixdgs_stream_t stream);

/* A whole frame in one call, for every camera of the plan: the batched
 * driver over the stages above (condition_project, bin_sort, raster_fwd and,
 * with targets, raster_bwd), all enqueued on `stream` so that the call can
 * be captured as one CUDA graph.
 * targets_dev == NULL: forward only (images_dev written; grad_images_dev,
 *   loss_dev and every grad_* are ignored and may be NULL; the plan may be an
 *   inference plan).
 * targets_dev != NULL: forward with the fused L1 loss, then the backward of
 *   that loss (sixdgs_raster_fwd_bwd, then sixdgs_project_bwd): *loss_dev (a
 *   double) is overwritten with the loss, grad_images_dev (optional) receives
 *   dL/dC, grad_* are overwritten as in sixdgs_raster_bwd (grad_lambda_raw as
 *   there).
 * Errors: those of the stages; a capacity overflow is reported through
 * *status_dev by bin_sort as usual. */
sixdgs_status sixdgs_render_batched(const sixdgs_plan* plan, const sixdgs_scene* scene,
                                    const sixdgs_camera* cams_host, void* ws_dev, size_t ws_bytes,
                                    float* images_dev, const float* targets_dev, float* grad_images_dev,
                                    double* loss_dev, float* grad_mu_p, float* grad_mu_d,
                                    float* grad_l_raw, float* grad_opacity_logit, float* grad_sh,
                                    float* grad_lambda_raw, int32_t* status_dev, sixdgs_stream_t stream);

/* Measurement helper, no counterpart in the paper: `blocks` CTAs of 256
 * threads each run `iters` iterations of 8 independent dependency chains of
 * FP32 fused multiply-adds (kind 0: 2 flops each) or of MUFU ex2 plus one add
 * (kind 1), and write one float per thread to out_dev (blocks * 256 floats,
 * caller-owned device memory).  Timing the call gives the FP32-pipe and MUFU
 * rates at the GPU's current clocks.  Errors: INVALID_ARG, CUDA. */
sixdgs_status sixdgs_peak_probe(int32_t kind, int64_t iters, float* out_dev, int32_t blocks,
                                sixdgs_stream_t stream);

/* View-independent part of the slice (section 3.2, Eq. sigma; Algorithm 1
 * steps 1-3) for every Gaussian, stored for the cond_cache field of
 * sixdgs_scene: A = Sigma_pd Sigma_d^-1 (planes 0-8, row-major), the upper
 * triangle of Sigma_d^-1 (planes 9-14: 00 01 02 11 12 22), Sigma_cond
 * (planes 15-23, row-major) and alpha = sigmoid(opacity_logit) (plane 24;
 * NaN for a Gaussian whose Sigma_d is not numerically positive definite,
 * which the projection then reports as SIXDGS_ERR_NONFINITE).
 * l_raw_dev: 21 planes, opacity_logit_dev: 1 plane, cache_dev:
 * SIXDGS_COND_CACHE_PLANES planes, all of n floats, device memory owned by
 * the caller.  No workspace.  Errors: INVALID_ARG, CUDA. */
#define SIXDGS_COND_CACHE_PLANES 25
sixdgs_status sixdgs_condition_cache(int64_t n, const float* l_raw_dev, const float* opacity_logit_dev,
                                     float* cache_dev, sixdgs_stream_t stream);

/* Scale and rotation of every conditional 3D Gaussian (section 4.3;
 * Algorithm 1 steps 4-5), the input of adaptive density control:
 * Sigma_cond = U D U^T, R = U with its third column multiplied by
 * sign(det R), S = sqrt(diag D), eigenvalues in decreasing order.
 * l_raw_dev: the scene's 21 raw Cholesky planes (n each).
 * rotation_dev: output, 9 planes (R row-major: plane i*3+j holds R_ij);
 * scale_dev: output, 3 planes.  No workspace.  A Gaussian whose covariance is
 * not finite gets zeros and SIXDGS_ERR_NONFINITE in *status_dev.
 * Errors: INVALID_ARG, CUDA. */
sixdgs_status sixdgs_scale_rotation(int64_t n, const float* l_raw_dev, float* rotation_dev,
                                    float* scale_dev, int32_t* status_dev, sixdgs_stream_t stream);

/* Forward render without any caller-provided workspace.  The paper has no
 * counterpart: this is a convenience of this library.
 *
 * For callers that cannot allocate device memory: code embedded in a host
 * application whose own allocator owns the device memory (plugins, engines
 * with a fixed budget), or loops that must never call cudaMalloc.  It runs
 * the same work as sixdgs_condition_project + sixdgs_bin_sort +
 * sixdgs_raster_fwd (no loss) and writes the same images, but keeps the
 * frame's workspace in one array of SIXDGS_STATIC_WS_BYTES (32 MiB) that
 * lives in the library's device memory.  Every GPU that loads the library
 * holds that array until the process exits.  The call allocates nothing
 * (no cudaMalloc, cudaFree or allocating library routine).
 *
 * Limits: the frame is planned forward-only whatever the caller's settings
 * say (as with settings.inference = 1 and store_aux = 0: no gradient
 * records, no per-pixel walk lengths) with the default duplicate capacity,
 * and that plan must need at most SIXDGS_STATIC_WS_BYTES of workspace, about
 * 225,000 (camera, Gaussian) pairs (e.g. 225,925 Gaussians seen by one
 * 800x800 camera, or 56,504 Gaussians by four 256x256 cameras); larger
 * frames are refused with SIXDGS_ERR_WORKSPACE before anything is launched.  The array is
 * shared by all calls on a device and keeps the last call's contents (each
 * call clears what it needs); calls that overlap on the GPU (different
 * streams or threads, same device) race on it, so serialise them.  The
 * first call on each device looks up the array's device address (with that
 * device current); make that first call before any stream capture.
 * Arguments are those of the staged calls; scene and images as there.
 * Errors: INVALID_ARG, WORKSPACE, CUDA; device status as the staged calls. */
#define SIXDGS_STATIC_WS_BYTES (32u << 20)
sixdgs_status sixdgs_render_fwd_static(int64_t n, int32_t sh_degree, const sixdgs_scene* scene,
                                       const sixdgs_camera* cams, int32_t n_cams,
                                       const sixdgs_settings* settings, float* images_dev,
                                       int32_t* status_dev, sixdgs_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SIXDGS_H */
