/*
 * gsreg.h -- C ABI of the GB300 (sm_103a) 3D-Gaussian submap registration
 * library libgsreg.so.
 *
 * The method is LoopSplat's registration of Gaussian-splat submaps
 * (arXiv 2408.10154, Sec. 3.2): one submap is moved by a rigid transform,
 * rendered (RGB + depth) at keyframes of the other submap, and the L1 colour
 * + L1 depth loss is descended on the transform, in both directions; the
 * per-keyframe estimates are fused by residual-weighted rotation averaging
 * (Eq. 7).  The renderer is the 3D Gaussian splatting forward model the
 * paper builds on (EWA projection, 16x16 screen tiles sorted by depth,
 * front-to-back alpha compositing) and its adjoint.
 *
 * Conventions (all entry points):
 *   - Every array argument is a DEVICE pointer owned by the caller unless its
 *     comment says "host".  Arrays are C-contiguous float32 unless stated.
 *   - Calls are stream-ordered on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream) and return once the work is enqueued, except where a
 *     comment says the call synchronises.  Device pointers must stay valid
 *     until that work completes.
 *   - Every function returns a gs_status_t.  GS_ERR_* leaves outputs
 *     undefined; gs_last_error() then describes the failure.  No C++
 *     exception crosses this boundary.  Device code never traps: faults of the
 *     data (non-finite inputs, list capacity) are reported through a device
 *     status word read back by the synchronising calls.
 *   - Matrices are row-major 3x4 [R | t].  A "pose" maps the moving submap's
 *     object frame to the world frame (mu' = R mu + t, Sigma' = R Sigma R^T,
 *     Eq. 8/9).  Cameras are OpenCV-style (x right, y down, z forward) with a
 *     world -> camera transform; pixel (px, py) samples the image at
 *     (px + 0.5, py + 0.5).
 *   - The library owns scratch memory only inside a gs_ctx_t, allocated with
 *     cudaMalloc on first use and grown up to the context's byte budget.
 */
#ifndef GSREG_H
#define GSREG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GSREG_VERSION 1
/* screen tile side in pixels (fixed: the kernels run one 16x16 CTA per tile) */
#define GS_TILE 16
/* floats per projected record (gs_project) and per auxiliary record */
#define GS_RECORD_FLOATS 12
#define GS_AUX_FLOATS 8

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1, /* bad pointer, size, camera or option */
    GS_ERR_OOM = 2,         /* workspace would exceed the context budget or cudaMalloc failed */
    GS_ERR_CUDA = 3,        /* a CUDA runtime call failed (message in gs_last_error) */
    GS_ERR_NONFINITE = 4,   /* an input Gaussian parameter or pose is NaN / Inf */
    GS_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
    GS_ERR_DIVERGED = 6,    /* a registration ended with a non-finite residual */
    GS_ERR_CAPACITY = 7     /* the tile lists outgrew their capacity (gs_register* after its redos,
                               gs_bin's caller capacity), or the work exceeds the fixed scratch of
                               gs_render_noalloc */
} gs_status_t;

typedef struct gs_ctx gs_ctx_t;
typedef void *gs_stream_t; /* cudaStream_t */

/* A submap of n Gaussians {mu, Sigma, o, C} (Eq. 1), SoA, float4-padded:
 * Sigma = R(q) diag(e^{2 s}) R(q)^T from per-axis log-scales s and a
 * quaternion q (normalised on use); opacity o = sigmoid(logit); colour C in
 * [0,1]^3, no spherical harmonics (Sec. 3.3, last paragraph). */
typedef struct {
    const float *means;          /* [n][4]: x, y, z, unused */
    const float *log_scales;     /* [n][4]: sx, sy, sz, unused */
    const float *quats;          /* [n][4]: w, x, y, z */
    const float *opacity_logits; /* [n] */
    const float *rgb;            /* [n][4]: r, g, b, unused */
    int64_t n;                   /* 0 <= n < 2^31 */
} gs_gaussians_t;

/* Pinhole keyframe camera: intrinsics, image size and world -> camera. */
typedef struct {
    float fx, fy, cx, cy;
    int32_t width, height; /* 1..32768 each */
    float world_to_cam[12];
} gs_camera_t;

/* A keyframe viewpoint v = (I, D, T) (Eq. 6): its colour and depth images
 * (device, planar) and its camera. */
typedef struct {
    const float *rgb;   /* [3][H][W] */
    const float *depth; /* [H][W] */
    gs_camera_t cam;
} gs_view_t;

/* Renderer and optimiser options; gs_default_options() fills them. */
typedef struct {
    int32_t tile;      /* must be GS_TILE */
    float z_near;      /* cull Gaussians with camera depth <= z_near (0.2 m) */
    float dilation;    /* 2D low-pass added to the projected covariance (0.3 px^2) */
    float alpha_min;   /* skip contributions with alpha < alpha_min (1/255) */
    float alpha_max;   /* clamp alpha to alpha_max (0.99) */
    float t_min;       /* stop before transmittance would drop below t_min (1e-4) */
    float bg[3];       /* background colour (0) */
    int32_t smooth;    /* 1: no radius cull (every tile), for derivative checks */
    /* registration (Sec. 3.2; learning rates from Supp. B) */
    float lr_rot;      /* 0.015 rad */
    float lr_trans;    /* 0.005 m */
    float beta1;       /* 0.8 */
    float beta2;       /* 0.99 */
    float adam_eps;    /* 1e-8 */
    float lr_final;    /* cosine decay of both rates to this fraction (0.001) */
    int32_t profile;   /* 1: gs_register times each phase with CUDA events (gs_ctx_stats);
                          2: also counts the pairs that pass the alpha test (a slower forward
                          variant: use a separate call for the count, 1 for timing) */
    /* loss of the registration calls: 0 = the registration loss of Sec. 3.2
     * (L1 colour + L1 depth means); 1 = the frame-to-model tracking loss of
     * Eq. 2 with the masks of Supp. A (see gs_track_loss) */
    int32_t tracking_loss;
    float lambda_c;    /* colour weight of the tracking loss (0.6: TUM-RGBD / ScanNet, Supp. A) */
    /* exposure compensation of the registration loss (Supp. B): each keyframe
     * problem fits a gain e^a and an offset b of the rendered colour
     * (e^a I^ + b, shared by the channels; a = b = 0 at the start) with its
     * pose; not combinable with tracking_loss */
    int32_t exposure;
    float lr_exposure; /* 0.1 (Supp. B) */
    /* CTA schedule of the compositing kernels in gs_register* and the
     * server (results are identical either way): 0 = picked by the
     * autotuner (the first registration of a plan shape on a context times
     * the four below on trial iterations from the initial poses, keeps the
     * fastest per shape and starts over); one CTA per tile in 1 = natural
     * tile order, 2 = longest tile lists first; persistent CTAs (as many as
     * fit on the GPU) pulling tiles of every keyframe problem from one work
     * queue in 3 = natural order, 4 = longest lists first */
    int32_t tile_schedule;
    /* tile rectangles of every call that projects or bins (gs_project and
     * so gs_bin, gs_render, gs_render_backward, gs_render_noalloc,
     * gs_register*, the server): 1 = each Gaussian listed only on the tiles
     * of its 3-sigma rectangle whose pixel centres can reach alpha_min (the
     * box of its alpha-threshold ellipse, with margins, by a fixed FP32
     * operation sequence; about a third fewer duplicates on room-sized
     * scenes), 0 = the 3-sigma rectangles.  Colour, depth, alpha and final
     * transmittance are identical either way (the dropped pairs fail the
     * alpha test); list positions (`last`) differ, so gs_render and
     * gs_render_backward must use the same value.  Needs alpha_min >=
     * FLT_MIN and smooth = 0, else the 3-sigma rectangles are used. */
    int32_t tight_lists;
    /* capacity of the tile lists of gs_register* as a multiple of the
     * duplicates at the initial poses (1.5; 64 Ki entries more when >= 1):
     * the lists move with the poses, and when an iteration outgrows them
     * the edge is redone from its initial poses with max(2 x, 1.5) (the
     * results are those of a run that did not outgrow them).  Finite and
     * in (0, 64]; below 1 the first attempt always outgrows its lists. */
    float list_headroom;
    /* compositing of the registration iterations of gs_register* and the
     * server: 1 = the forward and the adjoint of a tile in one CTA (one
     * launch; the pixel state stays in registers), for problems whose
     * keyframes all use the registration loss (the tracking loss needs every
     * tile's forward before any adjoint and always runs them as two
     * kernels); 0 = two kernels.  Results are bit-identical either way; with
     * 1, the profile's forward phase holds the fused kernel and its backward
     * phase is empty.  Default 1. */
    int32_t fuse_compositing;
} gs_options_t;

/* Statistics of the last gs_register / gs_render call on a context. */
typedef struct {
    int64_t kernel_launches; /* kernels of this library launched by the call */
    int64_t n_dups;          /* tile duplicates at the last binning */
    int64_t n_pixels;        /* pixels of one render pass over all keyframes */
    int64_t pairs;           /* sum over iterations and pixels of the list prefix the adjoint re-walks */
    int32_t iterations;      /* optimisation iterations run */
    int32_t schedule;        /* CTA schedule the registration ran (1..4, see tile_schedule) */
    /* profile != 0: summed CUDA-event time (ms) of each phase over the
     * iterations: project, bin (tile counts and ranges, placement, per-tile
     * sort), forward+loss, backward, pose update */
    double phase_ms[5];
    int64_t contributing;    /* profile = 2 only (else 0): sum over iterations of the (pixel,
                                Gaussian) pairs that pass the alpha test before the early stop */
} gs_stats_t;

/* ---------------------------------------------------------------- context */

/* Fills *o with the defaults listed in gs_options_t. */
void gs_default_options(gs_options_t *o);

/* Creates a context on CUDA device `device` whose scratch memory never
 * exceeds `hbm_budget_bytes` (0 = 16 GiB).  Allocates nothing yet. */
gs_status_t gs_ctx_create(int device, size_t hbm_budget_bytes, gs_ctx_t **out);

/* Frees the context's scratch (synchronises the device first). */
gs_status_t gs_ctx_destroy(gs_ctx_t *ctx);

/* Message of the last failure on this context (static storage; "" if none). */
const char *gs_last_error(const gs_ctx_t *ctx);

/* Bytes of scratch the context holds now. */
size_t gs_ctx_bytes(const gs_ctx_t *ctx);

/* Copies the statistics of the last gs_register / gs_render call. */
gs_status_t gs_ctx_stats(const gs_ctx_t *ctx, gs_stats_t *out);

/* sizeof of the ABI structs, for binding checks (no device needed):
 * out[0..6] = gs_gaussians_t, gs_camera_t, gs_view_t, gs_options_t,
 * gs_stats_t, gs_gaussian_grads_t, gs_problem_t; returns the number
 * written (<= n). */
int gs_abi_sizes(size_t *out, int n);

/* -------------------------------------------------------------- rendering */

/* Projection of a submap moved by one pose per camera (Eq. 8/9, then the EWA
 * projection of the 3DGS renderer: mean to pixel, covariance to the screen,
 * 3-sigma radius, tile rectangle).
 *   g         submap (n Gaussians)
 *   poses     [n_cams][12] device: pose of the submap for camera c
 *   cams      [n_cams] host
 *   records   [n_cams * n][GS_RECORD_FLOATS] out: record of (camera c,
 *             Gaussian i) at index c*n + i:
 *             {u, v, ca, cb, cc, o, z, rect_x, r, g, b, rect_y}; the exponent
 *             at pixel offset (dx, dy) = (u - x, v - y) is
 *             ca dx^2 + cb dx dy + cc dy^2; rect_x / rect_y hold the tile
 *             range bits (lo | hi << 16) as uint32.  Undefined when culled.
 *   aux       [n_cams * n][GS_AUX_FLOATS] out or NULL: camera-space mean
 *             x, y and covariance {S00, S01, S02, S11, S12, S22}.
 *   counts    [n_cams * n] int32 out: tiles touched, 0 if culled.
 * Every integer outcome (cull, rect, count) and every FP32 bit of the
 * record follows a fixed single-precision operation sequence. */
gs_status_t gs_project(gs_ctx_t *ctx, const gs_gaussians_t *g, const float *poses,
                       const gs_camera_t *cams, int n_cams, const gs_options_t *opt,
                       float *records, float *aux, int32_t *counts, gs_stream_t stream);

/* Tile binning of the records of gs_project: duplicates every visible record
 * into each tile of its rectangle (the tight or the 3-sigma one, as
 * gs_project's options chose) with key (global tile << 32) | float bits of z,
 * value = record index, sorted stably by key (ties keep record order), and
 * per-tile [start, end) ranges (0,0 when empty).  Camera c's tiles follow
 * those of cameras 0..c-1 (row-major within a camera).
 *   keys      [capacity] uint64 out, vals [capacity] uint32 out
 *   ranges    [total tiles][2] uint32 out
 *   n_dups    host out: number of duplicates (may exceed capacity: then
 *             nothing is written and GS_ERR_CAPACITY is returned).
 * Synchronises `stream`. */
gs_status_t gs_bin(gs_ctx_t *ctx, const float *records, const int32_t *counts, const gs_camera_t *cams,
                   int n_cams, int64_t n, uint64_t *keys, uint32_t *vals, int64_t capacity,
                   uint32_t *ranges, int64_t *n_dups, gs_stream_t stream);

/* Renders a submap moved by poses[c] at cams[c] (Sec. 3.2 "render RGB and
 * depth").  Outputs are concatenated per camera: camera c's planes start
 * after those of cameras 0..c-1 (rgb: 3*W*H floats per camera, planar).
 *   rgb [sum 3HW], depth [sum HW], alpha [sum HW] (= 1 - final
 *   transmittance), t_final [sum HW], last [sum HW] int32 (one past the
 *   tile-list position of the last contributor).  Any output may be NULL
 *   except t_final and last when gs_render_backward will follow.
 * Synchronises `stream` once (to size the tile lists). */
gs_status_t gs_render(gs_ctx_t *ctx, const gs_gaussians_t *g, const float *poses, const gs_camera_t *cams,
                      int n_cams, const gs_options_t *opt, float *rgb, float *depth, float *alpha,
                      float *t_final, int32_t *last, gs_stream_t stream);

/* Per-Gaussian parameter gradients (all device, any may be NULL); they are
 * OVERWRITTEN: means [n][4], log_scales [n][4], quats [n][4],
 * opacity_logits [n], rgb [n][4] (the 4th component is written as 0). */
typedef struct {
    float *means, *log_scales, *quats, *opacity_logits, *rgb;
} gs_gaussian_grads_t;

/* Adjoint of gs_render for the cotangents d_rgb, d_depth, d_alpha (any may
 * be NULL = 0), given the forward's t_final and last.
 *   pivots     [n_cams][3] device or NULL (= origin): the pose gradient is
 *              that of a left perturbation about pivot c,
 *              x -> exp([w]x)(x - c) + c + v, in the world frame.
 *   pose_grad  [n_cams][6] float out or NULL: dL/d(w, v) per camera.
 *   grads      per-Gaussian gradients or NULL (summed over cameras).
 * Synchronises `stream` (to size the lists, and at the end to read the
 * device status word). */
gs_status_t gs_render_backward(gs_ctx_t *ctx, const gs_gaussians_t *g, const float *poses,
                               const gs_camera_t *cams, int n_cams, const gs_options_t *opt,
                               const float *t_final, const int32_t *last, const float *d_rgb,
                               const float *d_depth, const float *d_alpha, const float *pivots,
                               float *pose_grad, const gs_gaussian_grads_t *grads, gs_stream_t stream);

/* A forward pass kept for its adjoint (the saved state of the 3DGS
 * rasteriser the paper renders with, Sec. 3.2): gs_render_saved renders like
 * gs_render and keeps the projected records, their camera-frame means and
 * covariances, the sorted tile lists and the per-pixel final transmittance
 * and last contributor; gs_render_backward_saved then runs the adjoint from
 * them -- no second projection or binning, and no host synchronisation.
 * The saved state lives in two device blocks allocated stream-ordered
 * (cudaMallocAsync on `stream`, outside the context's scratch budget) and
 * freed by gs_saved_destroy (cudaFreeAsync on its stream).  The submap's
 * arrays and the options are read again by the adjoint: keep the arrays
 * unchanged until then.  gs_render_saved synchronises `stream` like
 * gs_render; rgb, depth, alpha may be NULL. */
typedef struct gs_saved gs_saved_t;

gs_status_t gs_render_saved(gs_ctx_t *ctx, const gs_gaussians_t *g, const float *poses, const gs_camera_t *cams,
                            int n_cams, const gs_options_t *opt, float *rgb, float *depth, float *alpha,
                            gs_saved_t **saved, gs_stream_t stream);

/* Device pointers of the saved per-pixel state ([sum HW] each, owned by
 * the saved forward): final transmittance and last contributor. */
gs_status_t gs_saved_outputs(const gs_saved_t *saved, float **t_final, int32_t **last);

/* gs_render_backward from a saved forward (same cotangents, pivots and
 * outputs); stream-ordered, returns once the work is enqueued. */
gs_status_t gs_render_backward_saved(gs_ctx_t *ctx, const gs_saved_t *saved, const float *d_rgb,
                                     const float *d_depth, const float *d_alpha, const float *pivots,
                                     float *pose_grad, const gs_gaussian_grads_t *grads, gs_stream_t stream);

/* Frees a saved forward (stream-ordered after the work already on `stream`). */
gs_status_t gs_saved_destroy(gs_saved_t *saved, gs_stream_t stream);

/* L1 colour + L1 depth loss per view (Sec. 3.2: L = L_col + L_depth):
 * L_v = mean over 3HW of |I^ - I| + mean over HW of |D^ - D|, and its
 * gradients sign(.)/(3HW), sign(.)/(HW) (sign(0) = 0).  Images are
 * concatenated per camera as in gs_render.
 *   loss [n_cams] double out; d_rgb, d_depth out or NULL. */
gs_status_t gs_loss(gs_ctx_t *ctx, const gs_camera_t *cams, int n_cams, const float *rgb, const float *depth,
                    const float *t_rgb, const float *t_depth, double *loss, float *d_rgb, float *d_depth,
                    gs_stream_t stream);

/* Frame-to-model tracking loss per view (Eq. 2 with the masks of Supp. A):
 *   L_v = sum over pixels of M_in * M_a * (lambda_c |I^ - I|_1 + (1 - lambda_c) |D^ - D|),
 * |.|_1 over the colour channels, M_a = alpha^3 (alpha = 1 - t_final; a
 * weight, not differentiated), M_in = 1 where the input depth D > 0 and the
 * depth error e = |D^ - D| (FP32) is at most 50 times the view's median
 * error (the lower median over pixels with D > 0; FP32 product 50 * median).
 * Gradients (mask held fixed): dL/dI^ = M lambda_c sign(I^ - I),
 * dL/dD^ = M (1 - lambda_c) sign(D^ - D), sign(0) = 0.  Images concatenated
 * per camera as in gs_render (depth must be gs_render's FP32 depth for the
 * inlier decisions to be reproducible).
 *   loss [n_cams] double device out; d_rgb, d_depth, inlier (uint8 [pixels])
 *   and median [n_cams] float device out or NULL. */
gs_status_t gs_track_loss(gs_ctx_t *ctx, const gs_camera_t *cams, int n_cams, const float *rgb, const float *depth,
                          const float *t_final, const float *t_rgb, const float *t_depth, float lambda_c,
                          double *loss, float *d_rgb, float *d_depth, uint8_t *inlier, float *median,
                          gs_stream_t stream);

/* ---------------------------------------------------------- registration */

/* One Adam step on the pose twist and the pose update about the pivot, for
 * n independent poses (the on-device update of the registration loop):
 *   pose   [n][12] double in/out (object -> world)
 *   state  [n][13] double in/out: Adam m[6], v[6], step count
 *   grad   [n][6] double: dL/d(w, v) about pivot
 *   pivot  [n][3] double: rotation centre (world frame)
 * Learning rate = lr * (f + (1-f)(1 + cos(pi k / iters))/2), f = lr_final;
 * new pose: R <- exp([-w_step]x) R, t <- exp(.)(t - c) + c - v_step. */
gs_status_t gs_pose_step(gs_ctx_t *ctx, int n, double *pose, double *state, const double *grad,
                         const double *pivot, int k, int iters, const gs_options_t *opt, gs_stream_t stream);

/* Multi-view pose refinement (Eq. 7): fuses k estimates of T_{P->Q}.
 *   est      [k][12] double: estimates; reverse[i] != 0 marks an estimate of
 *            T_{Q->P}, inverted first (int32 [k])
 *   eps      [k] double: residuals; weights 1/max(eps, 1e-12)
 *   T_out    [12] double out: rotation = weighted chordal L2 mean,
 *            translation = weighted mean; conf [1] double out: mean weight. */
gs_status_t gs_fuse(gs_ctx_t *ctx, int k, const double *est, const int32_t *reverse, const double *eps,
                    double *T_out, double *conf, gs_stream_t stream);

/* 3DGS registration of submap P (src) and Q (tgt) (Sec. 3.2), both
 * directions in parallel:
 *   - each keyframe of V^P (src_views) localised in Q: Q moved by X so that
 *     its render at the keyframe matches the keyframe; estimate X^-1;
 *   - each keyframe of V^Q (tgt_views) localised in P: estimate Y;
 *   each from the identity, `iters` Adam steps on the twist about the
 *   moving submap's centroid; residual eps = loss at the final pose;
 *   fused by Eq. 7.  n_src_views or n_tgt_views may be 0 (one direction).
 *   T_out [12] host out: T_{P->Q} (float64)
 *   confidence host out: mean inverse residual
 *   eps_out [n_src_views + n_tgt_views] host out or NULL
 *   est_out [n_src_views + n_tgt_views][12] host out or NULL: per-keyframe
 *   estimates of T_{P->Q} (V^P first).
 * Synchronises `stream`. */
gs_status_t gs_register(gs_ctx_t *ctx, const gs_gaussians_t *src, const gs_gaussians_t *tgt,
                        const gs_view_t *src_views, int n_src_views, const gs_view_t *tgt_views,
                        int n_tgt_views, const gs_options_t *opt, int iters, double *T_out,
                        double *confidence, double *eps_out, double *est_out, gs_stream_t stream);

/* -------------------------------------------------- no-allocation render */

/* Bytes of the fixed device scratch behind gs_render_noalloc. */
#define GS_NOALLOC_SCRATCH_BYTES (32u << 20)

/* gs_render for callers that cannot allocate device memory.  The paper has
 * no counterpart; this is a deployment convenience.
 *
 * Some callers are not allowed to call cudaMalloc / cudaFree at all: code
 * running inside a host program whose allocator owns every byte of device
 * memory (an engine plugin, a robotics or game runtime with a fixed memory
 * plan), and latency-bound loops where an allocation or a free would
 * synchronise the whole device.  This entry point takes no context and
 * allocates nothing: its scratch is one fixed array of
 * GS_NOALLOC_SCRATCH_BYTES in device memory that every GPU which loads the
 * library holds until the process exits.  It runs on the caller's current
 * CUDA device.
 *
 * Arguments and outputs are those of gs_render (all outputs may be NULL).
 * The work must fit the fixed scratch: about 52 B per (camera, Gaussian)
 * record, 25 B per tile duplicate, 12 B per tile, 200 B per camera; larger
 * requests are rejected with GS_ERR_CAPACITY before any output is written
 * (the record part is checked before any GPU work, the duplicate part after
 * counting them).  The call synchronises `stream` (to count duplicates) and
 * returns GS_ERR_NONFINITE for non-finite Gaussian parameters.
 *
 * The scratch's device address belongs to the CUDA context the call runs
 * in (a device's primary context, a context made current with the driver
 * API, or a primary context re-created after cudaDeviceReset each have
 * their own copy of the array): the first call in each context looks it up
 * with that context current and caches it under the context's id; make
 * that first call before any stream capture.  Every call in a context
 * reuses the same scratch and leaves its contents behind; the call clears
 * what must start at zero.  Two calls that overlap on the GPU (different
 * streams or threads at the same time) race on the scratch and produce
 * undefined results: serialise them. */
gs_status_t gs_render_noalloc(const gs_gaussians_t *g, const float *poses, const gs_camera_t *cams, int n_cams,
                              const gs_options_t *opt, float *rgb, float *depth, float *alpha, float *t_final,
                              int32_t *last, gs_stream_t stream);

/* One registration problem of a batch: submaps P (src) and Q (tgt) and
 * their keyframes V^P, V^Q (Eq. 6); either keyframe list may be empty. */
typedef struct {
    gs_gaussians_t src, tgt;
    const gs_view_t *src_views; /* host array of n_src_views */
    int32_t n_src_views;
    const gs_view_t *tgt_views; /* host array of n_tgt_views */
    int32_t n_tgt_views;
    /* this problem's learning rates and loss (lr_rot, lr_trans,
     * tracking_loss, lambda_c; the other fields are the call's), or NULL =
     * the call's options */
    const gs_options_t *opt;
} gs_problem_t;

/* Batched 3DGS registration (Sec. 3.2 for each problem): all keyframe
 * problems of all n problems -- uneven submap sizes, keyframe counts and
 * image sizes -- advance together, each iteration one projection pass per
 * moving submap, one sort and one compositing launch over every tile of
 * every keyframe, replayed from one CUDA graph; Eq. 7 fuses each problem.
 *   T_out [n][12] host out; conf_out [n] host out;
 *   eps_out [sum of keyframes] host out or NULL (problem-major, V^P first).
 * Results equal n separate gs_register calls up to the order of floating
 * point reductions (every reduction is per keyframe, so in practice bit-equal).
 * Synchronises `stream`. */
gs_status_t gs_register_batch(gs_ctx_t *ctx, const gs_problem_t *problems, int n, const gs_options_t *opt, int iters,
                              double *T_out, double *conf_out, double *eps_out, gs_stream_t stream);

/* The registration loss of Sec. 3.2 and its pose gradient at the starting
 * poses: the keyframe problems gs_register would set up (the same submaps,
 * keyframes and options; every keyframe starts from the identity), run for
 * one iteration's forward and adjoint with nothing updated -- the kernels
 * of the registration hot path (fused or not, per fuse_compositing).
 *   loss_out [keyframes] double, host, or NULL: each keyframe's loss (the
 *     residual a 0-iteration gs_register returns), V^P first;
 *   grad_out [keyframes][6] double, host: each keyframe's gradient of its
 *     loss with respect to the pose of the submap that moves for it (Q for
 *     the keyframes of P, P for those of Q), as a world-frame twist
 *     (rotation w, then translation v) about that submap's centroid.
 * Synchronises `stream`; errors as gs_register. */
gs_status_t gs_register_gradient(gs_ctx_t *ctx, const gs_gaussians_t *src, const gs_gaussians_t *tgt,
                                 const gs_view_t *src_views, int n_src_views, const gs_view_t *tgt_views,
                                 int n_tgt_views, const gs_options_t *opt, double *loss_out, double *grad_out,
                                 gs_stream_t stream);

/* Stream-ordered forms of gs_register and gs_register_batch (Sec. 3.2, the
 * same problem statement: P, Q, their keyframes -> T_{P->Q} and the
 * residuals eps): every output is a DEVICE buffer written on `stream`, and
 * the call returns once the work is enqueued, so a caller can chain edges
 * (or feed T to its own kernels) without a host round trip.  Results equal
 * the synchronous calls' bit for bit.
 *   T_dev [problems][12] double, conf_dev [problems] double,
 *   eps_dev [keyframes] double or NULL (V^P first, problem-major),
 *   est_dev [keyframes][12] double or NULL (gs_register_async only),
 *   status_dev [1] int32: written on the stream when the work completes --
 *     GS_OK, GS_ERR_NONFINITE, GS_ERR_TIMEOUT, GS_ERR_DIVERGED, or
 *     GS_ERR_CAPACITY when the tile lists outgrew their capacity (the
 *     outputs are then invalid: redo with gs_register, which grows them).
 * The lists are sized from the largest duplicate count an earlier call on
 * this context saw for the same plan shape (tiles, keyframe problems,
 * records) times list_headroom; for a shape it has not seen, the call
 * counts them first, which synchronises `stream` once.  Growing the
 * context's scratch (a larger plan than before) frees and allocates device
 * memory, which synchronises the device.  The CTA schedule is the one the
 * autotuner chose earlier for the shape, else natural order (no trial
 * runs); profile is ignored.  Calls on one context must use one stream. */
gs_status_t gs_register_async(gs_ctx_t *ctx, const gs_gaussians_t *src, const gs_gaussians_t *tgt,
                              const gs_view_t *src_views, int n_src_views, const gs_view_t *tgt_views,
                              int n_tgt_views, const gs_options_t *opt, int iters, double *T_dev, double *conf_dev,
                              double *eps_dev, double *est_dev, int32_t *status_dev, gs_stream_t stream);
gs_status_t gs_register_batch_async(gs_ctx_t *ctx, const gs_problem_t *problems, int n, const gs_options_t *opt,
                                    int iters, double *T_dev, double *conf_dev, double *eps_dev, int32_t *status_dev,
                                    gs_stream_t stream);

/* ----------------------------------------------------------- loop filter */

/* Overlap ratio of submaps P and Q under T = T_{P->Q} (the loop filter of
 * the supplement, after Predator): P's means are moved by T (FP32, fused
 * multiply-adds translation first), each moved mean and each mean of Q find
 * their exact nearest neighbour on the other side (FP32 squared distance
 * fma(dz, dz, fma(dy, dy, dx * dx)), dx = b - a; ties to the smaller index),
 * the reciprocal pairs form K, and
 *   OR = |{(p, q) in K : |T p - q|^2 < tau^2 (FP32)}| / |K|  (0 if K is empty).
 *   T_host [12] host (row-major [R|t]); tau in metres (0.2 on TUM-RGBD /
 *   ScanNet / ScanNet++, 0.1 on Replica);
 *   ratio, n_corr (= |K|) host out; nn_pq [P.n], nn_qp [Q.n] device out or
 *   NULL (nearest neighbour indices, -1 when the other side is empty).
 * Synchronises `stream`. */
gs_status_t gs_overlap_ratio(gs_ctx_t *ctx, const gs_gaussians_t *p, const gs_gaussians_t *q, const double *T_host,
                             float tau, double *ratio, int64_t *n_corr, int32_t *nn_pq, int32_t *nn_qp,
                             gs_stream_t stream);

/* --------------------------------------------------------------- utility */

/* Stable sort of n (key, value) pairs by the low `bits` bits of the keys
 * (device arrays, sorted in place): a one-sweep LSD radix sort (8-bit
 * digits; one histogram pass, one look-back scatter per digit).  GS_ERR_TIMEOUT if a pass's bounded wait gave up (the device
 * keeps answering; the arrays' contents are then unspecified).
 * Synchronises `stream`. */
gs_status_t gs_sort_u32(gs_ctx_t *ctx, uint32_t *keys, uint32_t *vals, int64_t n, int bits, gs_stream_t stream);

/* FP32 peak probe (no counterpart in the paper; the denominator of the
 * compositing kernels' roofline): 8 independent FMA chains per thread,
 * 8 CTAs of 256 threads per SM, 4096 rounds, timed with CUDA events on
 * `stream`, once with scalar FMAs and once with packed ones (fma.rn.f32x2,
 * the compositing kernels' form); *tflops = the best of the ten timed
 * launches (five per form, 2 flops per FMA), *sm_count (may be NULL) = the
 * device's multiprocessor count.  Synchronises `stream`. */
gs_status_t gs_probe_fp32(gs_ctx_t *ctx, double *tflops, int *sm_count, gs_stream_t stream);

/* Self-test of the bounded device waits (no counterpart in the paper): one
 * sort pass over (keys, vals) whose first tile of 2048 keys is withheld, so
 * that every later tile's look-back runs out of its spin limit (well under
 * a second), sets the status word and returns.  Returns GS_ERR_TIMEOUT when
 * the waits behave; the context stays usable. */
gs_status_t gs_selftest_bounded_wait(gs_ctx_t *ctx, uint32_t *keys, uint32_t *vals, int64_t n, gs_stream_t stream);

/* ---------------------------------------------------------------- serving */

/* Continuous-batching registration server.  A request is one registration
 * problem (Sec. 3.2, as in gs_register; a frame-to-model tracking request is
 * a problem with one target keyframe -- the frame, its camera at the initial
 * guess -- and no source keyframes, whose estimate T maps the submap so that
 * it renders the frame, i.e. the tracked camera is world_to_cam o T) with its
 * own iteration count.  The submaps and keyframe images stay resident in
 * caller-owned device memory until the request is done.
 *
 * gs_server_step runs one round on `stream`:
 *   1. admits waiting requests in submission order while the in-flight
 *      keyframe problems stay <= max_keyframes and the scratch footprint of
 *      the in-flight requests stays <= hbm_budget_bytes (the first waiting
 *      request is always admitted into an empty server).  A request's
 *      footprint comes from its tile lists counted at submission (its
 *      Gaussians projected and binned at its starting poses on a separate
 *      measuring context and stream; see gs_server_footprint);
 *   2. when the in-flight set changed, re-plans it: one projection pass per
 *      moving submap, one sort and one compositing launch over every tile of
 *      every in-flight keyframe per iteration, captured into a CUDA graph,
 *      each request's pose and optimiser state carried over;
 *   3. replays the graph for min(max_round_iters, the fewest iterations any
 *      in-flight request has left) iterations;
 *   4. retires the requests whose iterations are done (plus one iteration at
 *      the frozen final pose that measures the residual of Eq. 7) and fuses
 *      their estimates by Eq. 7.
 * Every iteration of a request depends only on its own problem, so its
 * result equals gs_register's for the same problem and iteration count,
 * whatever else is in flight.  Synchronises `stream` once per round. */
typedef struct gs_server gs_server_t;

gs_status_t gs_server_create(int device, size_t hbm_budget_bytes, int max_keyframes, int max_round_iters,
                             const gs_options_t *opt, gs_server_t **out);
gs_status_t gs_server_destroy(gs_server_t *srv);
const char *gs_server_last_error(const gs_server_t *srv);

/* Queues a request; the problem's arrays must stay valid until it is done.
 * iters >= 0.  *id_out = the request id (ids start at 0 and increase).
 * Counts the request's tile lists first (synchronises the measuring
 * context's own stream, not the serving stream).  GS_ERR_OOM if the
 * request's footprint alone exceeds the budget (hbm_budget_bytes, 0 =
 * 16 GiB; the scratch arena may exceed it by a quarter, at least 256 MiB,
 * for the lists' growth as the poses move). */
gs_status_t gs_server_submit(gs_server_t *srv, const gs_problem_t *problem, int iters, int64_t *id_out);

/* One round (see above).  done_ids [max_done] host out (may be NULL): ids of
 * the requests retired in this round; *n_done = their number. */
gs_status_t gs_server_step(gs_server_t *srv, gs_stream_t stream, int64_t *done_ids, int max_done, int *n_done);

/* Result of request `id`: *state = 0 waiting, 1 in flight, 2 done.  When
 * done: T_out [12] host (row-major [R|t] of T_{P->Q}), *confidence,
 * eps_out [its keyframes] host or NULL (residuals, V^P first).  *t_submit,
 * *t_done: seconds on the server's clock (steady, from creation); any
 * output pointer may be NULL. */
gs_status_t gs_server_poll(gs_server_t *srv, int64_t id, int *state, double *T_out, double *confidence,
                           double *eps_out, double *t_submit, double *t_done);

/* Counts: requests waiting, in flight, done; rounds and re-plans run. */
gs_status_t gs_server_counts(const gs_server_t *srv, int64_t out[5]);

/* Admission by measured footprint: out[0] = requests whose tile lists were
 * counted at submission, out[1] = requests the memory budget kept waiting
 * at least once, out[2] = scratch bytes of the requests in flight now. */
gs_status_t gs_server_admission(const gs_server_t *srv, int64_t out[3]);

/* The footprint admission used for request `id`: *dups = its tile
 * duplicates at its starting poses, *bytes = its scratch in a plan (per
 * record 100 B, per list entry 12.5 B at the server's list headroom, per
 * pixel 9 B (+12 B for tracking), per tile 92 B, per keyframe problem its
 * optimiser state).  Either pointer may be NULL. */
gs_status_t gs_server_footprint(const gs_server_t *srv, int64_t id, int64_t *dups, int64_t *bytes);

/* Rigid transform of a submap by T (Eq. 8/9): mu <- R mu + t,
 * q <- q_R (x) q (so Sigma <- R Sigma R^T); scales, opacities, colours
 * unchanged.  out_means, out_quats [n][4] device (may alias the inputs). */
gs_status_t gs_transform(gs_ctx_t *ctx, const gs_gaussians_t *g, const double *T_host, float *out_means,
                         float *out_quats, gs_stream_t stream);

/* Map adjustment after pose-graph optimisation (Eq. 8/9 on every submap):
 * gs_transform of n_maps submaps, each by its own T, in one launch.
 *   T_host [n_maps][12] host; out_means, out_quats: host arrays of n_maps
 *   device pointers ([n][4] each, may alias the inputs).  Results equal
 *   gs_transform's bit for bit.  Keyframe poses of a corrected submap follow
 *   on the host: world_to_cam <- world_to_cam o T^-1 (a 3x4 product each). */
gs_status_t gs_transform_batch(gs_ctx_t *ctx, const gs_gaussians_t *maps, int n_maps, const double *T_host,
                               float *const *out_means, float *const *out_quats, gs_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* GSREG_H */
