/*
 * clod.h -- C ABI of libclod, the GB300 (sm_103a) CLoD-GS rasterizer.
 *
 * CLoD-GS (continuous level of detail for 3D Gaussian splatting) attenuates
 * each Gaussian's opacity with a learnable, distance-dependent decay
 * (Sec. 3.2, Eq. 2), culls primitives whose attenuated opacity falls under a
 * threshold that grows with the virtual distance scale (Sec. 3.2, mask M_i),
 * and renders the rest with a tile-based, depth-sorted, front-to-back
 * alpha-blending rasterizer (Sec. 3.1, Eq. 1).
 *
 * Conventions for every entry point:
 *   - Returns a clod_status; never throws, never aborts.  The message of the
 *     last failure on the calling thread is returned by clod_last_error().
 *   - Every array pointer is DEVICE memory owned by the caller, unless the
 *     parameter says "host".  The library never frees caller memory.
 *   - Work is enqueued on the given CUDA stream (a cudaStream_t passed as
 *     void*; NULL means the legacy default stream) and is asynchronous: the
 *     outputs are valid once the stream reaches them.  Calls that read a
 *     device value back say so and synchronise the stream.
 *   - Scene parameters come in ACTIVATED: opacity in (0, 1), scales > 0,
 *     quaternions (w, x, y, z) of any non-zero norm (normalised inside),
 *     decay sigma_d raw (the ReLU of Eq. 2 is applied inside).
 *   - Arithmetic is FP32.  Every quantity that decides an integer outcome
 *     (the mask, the tile rectangle, the depth key, the per-pixel skip and
 *     stop of the blend) is computed by a fixed sequence of IEEE operations
 *     with a fixed, monotone exponential, so the decisions are reproducible
 *     bit for bit by any implementation of the same sequence.
 */
#ifndef CLOD_H
#define CLOD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t clod_status;
#define CLOD_OK              0
#define CLOD_ERR_ARG         1  /* invalid argument (null pointer, bad size, ...)      */
#define CLOD_ERR_CAPACITY    2  /* a caller buffer is too small; required size reported */
#define CLOD_ERR_CUDA        3  /* a CUDA runtime call failed                          */
#define CLOD_ERR_TIMEOUT     4  /* a bounded device or host wait gave up               */
#define CLOD_ERR_QUEUE_FULL  5  /* serving queue full                                  */
#define CLOD_ERR_NOT_READY   6  /* serving request not finished                        */
#define CLOD_ERR_NAN         7  /* non-finite input detected (checked calls only)      */

/* view flags */
#define CLOD_LOD_OFF       1u  /* plain 3DGS: alpha'' = alpha, no level-of-detail cull */
#define CLOD_NO_NORMALIZE  2u  /* use d_i itself instead of d_i / max d (Sec. 3.2)    */
/* The blends (forward and backward) evaluate each (pixel, Gaussian) opacity
 * alpha'' exp(power) of Eq. 1 with the GPU's base-2 exponential unit instead of
 * the reproducible software exponential.  Opacities then carry a relative
 * error of a few 1e-7, the images stay within the FP32 rounding of the
 * real-arithmetic blend, and integer stages (mask, rectangles, keys, ranges)
 * are unchanged; but a skip or stop decision within that error of its
 * threshold may fall differently, so the images and contributor counts are no
 * longer bit-reproducible by another implementation of the FP32 sequence.
 * All views of one frame must agree on this flag. */
#define CLOD_FAST_EXP      4u

typedef void* clod_stream;     /* cudaStream_t */

/* A resident Gaussian scene (Sec. 3.1 primitives plus the per-Gaussian decay
 * sigma_d of Sec. 3.2).  All arrays are device memory, float32, row-major. */
typedef struct clod_scene {
    int64_t n;              /* number of Gaussians, 0 <= n < 2^31               */
    int32_t sh_degree;      /* 0..3                                             */
    int32_t reserved;
    const float* means;     /* n x 3                                            */
    const float* scales;    /* n x 3, activated (> 0)                           */
    const float* quats;     /* n x 4, (w, x, y, z)                              */
    const float* opacity;   /* n, activated, in (0, 1)                          */
    const float* sh;        /* n x (sh_degree+1)^2 x 3                          */
    const float* decay;     /* n, raw sigma_d                                   */
} clod_scene;

/* A pinhole camera and its level-of-detail setting.  Host memory. */
typedef struct clod_view {
    int32_t width, height;  /* pixels, 1..16384                                 */
    float viewmat[12];      /* world -> camera [R | t], row-major 3x4; camera
                               x right, y down, z forward                      */
    float fx, fy, cx, cy;   /* focal lengths and principal point, pixels; pixel
                               (x, y) has its centre at (x + 0.5, y + 0.5)      */
    float near_z;           /* near plane on the camera z axis                  */
    float campos[3];        /* camera centre c in world coordinates (Sec. 3.2)  */
    float s_v;              /* virtual distance scale s_v (Sec. 3.2)            */
    float tau;              /* base opacity threshold tau: M_i = alpha'' > tau s_v */
    float eps;              /* epsilon of Eq. 2                                 */
    float bg[3];            /* background colour                                */
    uint32_t flags;         /* CLOD_LOD_OFF | CLOD_NO_NORMALIZE | CLOD_FAST_EXP  */
    /* Region of a larger frame (regional level of detail, Sec. 4.4: one image
     * whose vertical bands are rendered at different s_v).  With
     * full_width > 0 the view is the width x height window at pixel
     * (region_x, region_y) of a full_width x full_height frame: viewmat,
     * fx, fy, cx, cy describe the FULL frame; the frustum of Sec. 3.2
     * (d_max) and the projection are the full frame's, and every output
     * pixel equals, bit for bit, the same pixel of the full-frame render at
     * this view's s_v.  region_x and region_y must be multiples of 16 (tile
     * aligned) and the window must lie inside the frame.  full_width = 0:
     * the view is a whole frame (region_x, region_y, full_height ignored). */
    int32_t region_x, region_y;
    int32_t full_width, full_height;
    /* Primitive budget (Sec. 4.2: models compared at equal Gaussian counts by
     * applying the attenuation of Eq. 2 and keeping the primitives of highest
     * attenuated opacity).  budget > 0 replaces the threshold test: M_i = 1
     * for the min(budget, n) Gaussians of highest alpha'' (equal alpha'' in
     * increasing index order), 0 for the rest.  0: M_i = alpha'' > tau s_v. */
    uint32_t budget;
} clod_view;

/* Byte offsets of the arrays inside a frame workspace (for inspection). */
typedef struct clod_frame_layout {
    uint64_t total_bytes;
    uint64_t views;         /* n_views device view records                      */
    uint64_t dmax_key;      /* u64 [n_views]: (bits(d_max) << 32) | ~argmax     */
    uint64_t n_survivors;   /* u32 [2 * n_views]: sum M_i, rendered (per view)  */
    uint64_t rec0;          /* float4 [n_views * n]: u, v, -A/2, -B             */
    uint64_t rec1;          /* float4 [n_views * n]: -C/2, alpha'', r, g        */
    uint64_t rec2;          /* float4 [n_views * n]: b, reach half-extents x, y (pixels; -inf: reaches no pixel), 0 */
    uint64_t depth;         /* float  [n_views * n]: camera-space z             */
    uint64_t rect;          /* uint2  [n_views * n]: (x0 | y0 << 16, x1 | y1 << 16), tiles [x0,x1)x[y0,y1) */
    uint64_t tile_count;    /* u32 [total_tiles]                                */
    uint64_t tile_offset;   /* u32 [total_tiles + 1]: exclusive scan of tile_count */
    uint32_t total_tiles;   /* sum over views of ceil(W/16) * ceil(H/16)        */
    uint32_t n_views;
} clod_frame_layout;

/* Last error message of the calling thread ("" if none). */
const char* clod_last_error(void);

/* Library version string and the compute capability it was built for. */
const char* clod_version(void);

/* ------------------------------------------------------------------------ */
/* Forward pipeline: clod_preprocess -> clod_bin_sort -> clod_render_fwd      */
/* ------------------------------------------------------------------------ */

/* Size and layout of the frame workspace for n Gaussians and the given views
 * (host array of n_views >= 1 records).  *layout may be NULL. */
clod_status clod_frame_workspace_size(int64_t n, const clod_view* views, int32_t n_views,
                                      size_t* bytes, clod_frame_layout* layout);

/* Per-Gaussian preprocessing of every view (Sec. 3.2 and Sec. 3.1):
 *   d_i = |mu_i - c|; d_max = max of d over the view frustum (t_z > near and
 *   projected centre in [0,W]x[0,H]); alpha'' of Eq. 2 with d' = d / d_max;
 *   mask M_i = alpha'' > tau s_v (or the top-budget selection, see
 *   clod_view.budget: a radix select of the keys (bits(alpha'') << 32 | ~i)
 *   over all n Gaussians, six 11/10-bit digit passes); for survivors (M_i, t_z > near, det > 0,
 *   non-empty tile rectangle) the EWA projection (2D covariance + 0.3 I,
 *   its inverse, 3-sigma radius, 16x16-pixel tile rectangle), depth and the
 *   SH colour; per-tile pair counts and their exclusive scan.
 * ws:             frame workspace of ws_bytes >= clod_frame_workspace_size().
 * mask_out:       u8 [n_views * n] (view-major), the mask M_i of Sec. 3.2;
 *                 may be NULL.
 * alpha_eff_out:  f32 [n_views * n] alpha''; may be NULL.
 * counts_out:     u32 [2 * n_views]: [2v] = sum_i M_i of view v (the count
 *                 of Eq. 4's eta_actual), [2v + 1] = Gaussians rendered in
 *                 view v (M_i and the survivor conditions); may be NULL.
 * n_pairs_out:    u64 [1] total (view, tile, Gaussian) pairs K; may be NULL.
 * views is read on the host during the call.  Errors: CLOD_ERR_ARG for null
 * scene arrays (n > 0), n_views < 1, bad sizes or sh_degree; CLOD_ERR_CUDA. */
clod_status clod_preprocess(const clod_scene* scene, const clod_view* views, int32_t n_views,
                            void* ws, size_t ws_bytes,
                            uint8_t* mask_out, float* alpha_eff_out,
                            uint32_t* counts_out, uint64_t* n_pairs_out,
                            clod_stream stream);

/* Emits every (view, tile, Gaussian) pair of the preprocessed frame in the
 * order of the key ((tile_base(view) + ty * TX + tx) << 32) | bits(depth),
 * equal keys in Gaussian-index order -- "sorted by depth" per tile
 * (Sec. 3.1) -- and the tile ranges.  Built from a stable radix sort of the
 * survivors' depths (depth ranks) and an order-preserving walk of the tile
 * rectangles in rank order; no pair is sorted or written twice.
 * keys_out:   u64 [pair_capacity] sorted keys; may be NULL.
 * vals_out:   u32 [pair_capacity] Gaussian index of each sorted pair.
 * ranges_out: u32 [total_tiles * 2] [first, last) of each tile in vals_out;
 *             tiles without pairs get [0, 0).
 * If K > pair_capacity nothing is written to keys_out/vals_out and the frame
 * is marked overflowed: clod_render_fwd then writes nothing and
 * clod_frame_check() returns CLOD_ERR_CAPACITY with the required K.
 * The sort consumes the depth keys and digit counts clod_preprocess left in
 * ws: call it once per clod_preprocess (to retry with a larger capacity, run
 * clod_preprocess again). */
clod_status clod_bin_sort(void* ws, uint64_t pair_capacity,
                          uint64_t* keys_out, uint32_t* vals_out, uint32_t* ranges_out,
                          clod_stream stream);

/* Front-to-back alpha blending of every tile of every view (Eq. 1):
 * per pixel, in list order: power = -(A dx^2 + C dy^2)/2 - B dx dy; skip if
 * power > 0; a = min(0.99, alpha'' exp(power)); skip if a < 1/255; stop
 * (excluding this Gaussian) once T (1 - a) < 1e-4; colour += rgb a T.
 * Output colour + T bg.  Packed outputs: view v's pixels start at
 * P_v = sum_{u<v} W_u H_u; image f32 [3 * sum W H] with view v's planes at
 * 3 P_v (CHW); T_final f32 [sum W H]; n_contrib u32 [sum W H] (1 + list
 * position of the last contributor, 0 if none).  T_final and n_contrib may
 * be NULL.  vals/ranges are clod_bin_sort's outputs for the same frame. */
clod_status clod_render_fwd(const void* ws, const uint32_t* vals, const uint32_t* ranges,
                            float* image, float* T_final, uint32_t* n_contrib, clod_stream stream);

/* Synchronises the stream and reads the frame's status: K into *n_pairs
 * (may be NULL) and CLOD_ERR_CAPACITY if a clod_bin_sort overflowed. */
clod_status clod_frame_check(const void* ws, uint64_t pair_capacity, uint64_t* n_pairs, clod_stream stream);

/* Same as clod_render_fwd (without the blend's per-warp skipping, which
 * changes no output), also accumulating into evaluated[0..2] (device u64):
 * the (pixel, Gaussian) pairs visited before the pixel stopped, those whose
 * power fell in [-5.6, 0] (the exponential is evaluated), and those that
 * contributed. */
clod_status clod_render_fwd_count(const void* ws, const uint32_t* vals, const uint32_t* ranges,
                                  float* image, float* T_final, uint32_t* n_contrib,
                                  unsigned long long* evaluated, clod_stream stream);

/* ------------------------------------------------------------------------ */
/* Backward pass                                                              */
/* ------------------------------------------------------------------------ */

/* Scratch bytes of clod_render_bwd for n Gaussians and n_views views. */
clod_status clod_backward_workspace_size(int64_t n, int32_t n_views, size_t* bytes);

/* Gradients of a scalar loss L with respect to the six activated parameter
 * groups, given dL/d(image) of the frame rendered from ws/vals/ranges (the
 * forward's outputs, unchanged since) and, optionally, an external
 * dL/d(alpha'') for every (view, Gaussian) -- the training step's
 * straight-through gradient of the point-count regulariser (Eq. 4).
 * Differentiates Eq. 1 (blending, with the forward's skip/stop decisions and
 * the 0.99 opacity clamp), the EWA projection, Sigma = R S S^T R^T, the SH
 * colour (clamped at 0) and Eq. 2 (alpha, sigma_d with its ReLU, and mu
 * through d_i and through d_max = d_{j*}, j* the lowest-index farthest
 * Gaussian in the view frustum).
 * T_final, n_contrib: the forward's packed outputs.  dL_dimage: packed like
 * the image.  dL_dalpha_eff: f32 [n_views * n] or NULL.  dL_dalpha_view:
 * f32 [n_views] or NULL, one external dL/d(alpha'') shared by every Gaussian
 * of a view (the straight-through gradient is such a constant; added to
 * dL_dalpha_eff when both are given).
 * Outputs are ACCUMULATED (+=): dmeans n x 3, dscales n x 3, dquats n x 4,
 * dopacity n, dsh n x (deg+1)^2 x 3, ddecay n. */
clod_status clod_render_bwd(const clod_scene* scene, const void* ws, const uint32_t* vals,
                            const uint32_t* ranges, const float* T_final, const uint32_t* n_contrib,
                            const float* dL_dimage, const float* dL_dalpha_eff, const float* dL_dalpha_view,
                            void* bwd_ws, size_t bwd_ws_bytes,
                            float* dmeans, float* dscales, float* dquats, float* dopacity,
                            float* dsh, float* ddecay, clod_stream stream);

/* As clod_render_bwd, but the six gradient arrays are OVERWRITTEN: every
 * element is written (zero for a Gaussian that survives in no view), so the
 * caller need not zero them first.  Same arguments, layouts and errors.  A
 * training step that runs one backward per update (followed by
 * clod_adam_step with keep_grads = 1) then reads and writes each gradient
 * once instead of zeroing, reading and adding to it. */
clod_status clod_render_bwd_set(const clod_scene* scene, const void* ws, const uint32_t* vals,
                                const uint32_t* ranges, const float* T_final, const uint32_t* n_contrib,
                                const float* dL_dimage, const float* dL_dalpha_eff, const float* dL_dalpha_view,
                                void* bwd_ws, size_t bwd_ws_bytes,
                                float* dmeans, float* dscales, float* dquats, float* dopacity,
                                float* dsh, float* ddecay, clod_stream stream);

/* L1 term of the rendering loss (Sec. 3.3): *loss += scale * mean |image -
 * target| over count elements (device f32 scalar, may be NULL) and
 * dL_dimage = scale * sign(image - target) / count (may be NULL). */
clod_status clod_l1_loss(const float* image, const float* target, int64_t count, float scale,
                         float* loss, float* dL_dimage, clod_stream stream);

/* Scratch bytes of clod_render_loss for a channels x height x width image. */
clod_status clod_render_loss_workspace_size(int32_t channels, int32_t height, int32_t width, size_t* bytes);

/* Rendering loss of Sec. 3.3, L_render = (1 - w) L1 + w (1 - SSIM), with
 * w = dssim_weight in [0, 1] (0.2 in the 3DGS training the paper builds on).
 * SSIM: 11x11 Gaussian window (sigma 1.5, zero outside the image),
 * C1 = 0.01^2, C2 = 0.03^2, mean over pixels and channels.  image, target:
 * device f32 channels x height x width.  *loss (device f32, may be NULL) +=
 * L_render; dL_dimage (may be NULL) = grad_scale * dL_render/dimage (the
 * factor of this term in the caller's total), which for w > 0 needs ws
 * (device, size from clod_render_loss_workspace_size; w = 0 needs none). */
clod_status clod_render_loss(const float* image, const float* target, int32_t channels, int32_t height,
                             int32_t width, float dssim_weight, float grad_scale, void* ws, size_t ws_bytes,
                             float* loss, float* dL_dimage, clod_stream stream);

/* Per-view weights of one training step (Sec. 3.3, Eq. 5, averaged over the
 * step's views): weight[v] = w_s(s_v[v]) / n_views with
 * w_s(s) = (1 - 0.5 s / s_max)^2, s_max the largest scale the step's sampler
 * draws.  Host arrays s_v (> 0) and weight, n_views in [1, 64]; s_max > 0.
 * The weights scale the rendering loss (clod_render_loss grad_scale) and
 * the objective of clod_lreg_grad. */
clod_status clod_step_weights(const float* s_v, int32_t n_views, float s_max, float* weight);

/* Point-count regulariser and total objective of the training step
 * (Sec. 3.3, Eq. 3-5), on the device, for n_views views of one step:
 *   eta_actual_v = counts[2v] / n (the mask counts of clod_preprocess),
 *   L_reg_v = (s_v - 1)^2 ReLU(eta_actual_v - s_v^-1.5)^2,
 *   *total = sum_v weight_v (lrender_v + lambda_reg L_reg_v)   (written),
 *   dL_dalpha_view[v] = weight_v lambda_reg 2 (s_v - 1)^2 ReLU(.) / n,
 * the straight-through gradient (dM_i/dalpha''_i := 1) for clod_render_bwd.
 * weight_v = w_s(s_v) / n_views for Eq. 5 averaged over the step's views.
 * counts: device u32 [2 n_views].  s_v, weight: host f32 [n_views].
 * lrender: device f32 [n_views] or NULL (0).  dL_dalpha_view, total,
 * lreg_out (device f32 [n_views]): each may be NULL. */
clod_status clod_lreg_grad(const uint32_t* counts, int64_t n, int32_t n_views, const float* s_v,
                           const float* weight, float lambda_reg, const float* lrender,
                           float* dL_dalpha_view, float* total, float* lreg_out, clod_stream stream);

/* Adam (beta1, beta2, eps; bias-corrected, no weight decay) over the six
 * parameter groups, learning rate per group: means, log-scales, quaternions,
 * opacity logits, SH, sigma_d (Sec. 4.1 gives sigma_d 1e-2). */
typedef struct clod_adam_cfg {
    float lr[6];
    float beta1, beta2, eps;
    int32_t step;           /* t >= 1 */
    int32_t keep_grads;     /* 0: zero the six gradient arrays after the update;
                               1: leave them (a backward with overwritten outputs,
                               clod_render_bwd_set, refills them every step) */
} clod_adam_cfg;

/* One Adam step fused with the activations.  raw: host array of 6 device
 * pointers, the raw parameters (means n x 3, log-scales n x 3, quats n x 4,
 * opacity logits n, sh n x (deg+1)^2 x 3, sigma_d n), updated in place.
 * grads: host array of 6 device pointers, the gradients with respect to the
 * ACTIVATED parameters (clod_render_bwd's outputs); the log-scale and logit
 * gradients are formed inside (times scale, times a (1 - a)); all six are
 * zeroed afterwards unless cfg->keep_grads.  scales, opacity: the activated copies the rasterizer
 * reads (exp(log-scale), sigmoid(logit)), read for the chain rule and
 * rewritten from the updated raw values.  m, v: device f32 moments of
 * clod_adam_state_size() elements each (zero before the first step), the six
 * groups in the order above, each starting at a multiple of 4 elements.
 * Every array must be 16-byte aligned (CLOD_ERR_ARG otherwise). */
clod_status clod_adam_state_size(int64_t n, int32_t sh_degree, int64_t* elements);
clod_status clod_adam_step(const clod_adam_cfg* cfg, int64_t n, int32_t sh_degree, float* const* raw,
                           float* const* grads, float* scales, float* opacity, float* m, float* v,
                           clod_stream stream);

/* Measurement aid (no counterpart in the paper): launches one full wave of
 * threads that each run 8 independent chains of `iters` FP32 fused
 * multiply-adds, so that timing the launch gives this GPU's FP32 peak (the
 * roofline of the FP32-bound blend).  sink: device f32 [1] (never written in
 * practice); *flops (host) = the launch's floating-point operations. */
clod_status clod_probe_fma(int32_t iters, float* sink, uint64_t* flops, clod_stream stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching over a resident scene                         */
/* ------------------------------------------------------------------------ */

typedef struct clod_server clod_server;

typedef struct clod_server_cfg {
    int32_t max_views_per_batch;   /* views per launch, 1..64                        */
    int32_t n_slots;               /* batches in flight at once, 1..16               */
    int32_t queue_capacity;        /* pending requests before CLOD_ERR_QUEUE_FULL    */
    int32_t use_graphs;            /* 1: every slot replays one captured CUDA graph  */
    uint64_t max_pixels_per_batch; /* admission: sum of W*H in one batch; the slots'
                                      workspaces are sized for it                   */
    uint64_t pair_capacity;        /* (view, tile, Gaussian) pairs per slot          */
    int32_t batch_window_us;       /* wait up to this long for a fuller batch (0: no) */
    int32_t max_width, max_height; /* largest view accepted                          */
    int32_t fast_exp;              /* 1: every batch blends with CLOD_FAST_EXP's
                                      exponential (the requests' own flag is ignored) */
} clod_server_cfg;

typedef struct clod_req_stats {
    int32_t status;                /* CLOD_OK, or the request's error                */
    int32_t batch_size;            /* views in the launch that rendered it           */
    double submit_us, launch_us, done_us;  /* steady host clock, microseconds        */
    uint32_t n_rendered;           /* Gaussians rendered in this view                */
    uint32_t reserved;
    uint64_t n_pairs;              /* pairs of its launch                            */
} clod_req_stats;

/* Creates a server over a scene that stays resident (the scene arrays must
 * outlive the server).  Allocates n_slots workspaces sized for the largest
 * batch and starts a worker thread.  Requests are admitted in arrival order
 * into batches of at most max_views_per_batch views and max_pixels_per_batch
 * pixels as slots free up; batches on different slots run concurrently on
 * their own streams.  A batch renders every view with one launch sequence
 * (the scene is read once per batch).  A batch whose pairs exceed
 * pair_capacity is re-run one request at a time with buffers sized from its
 * pair count. */
clod_status clod_server_create(const clod_scene* scene, const clod_server_cfg* cfg, clod_server** out);

/* Queues one render of *view into image_out (device, 3 x H x W, caller-owned,
 * must stay valid until the request is done).  Returns a ticket.
 * CLOD_ERR_QUEUE_FULL when queue_capacity requests are pending; CLOD_ERR_ARG
 * for views larger than the server's maximum. */
clod_status clod_serve_submit(clod_server* server, const clod_view* view, float* image_out, uint64_t* ticket);

/* Non-blocking: *done = 1 and stats filled when the request has finished
 * (its image is then complete in device memory), after which the ticket is
 * released; otherwise *done = 0 and CLOD_ERR_NOT_READY. */
clod_status clod_serve_poll(clod_server* server, uint64_t ticket, int32_t* done, clod_req_stats* stats);

/* Blocks up to timeout_us for the request; CLOD_ERR_TIMEOUT if it has not
 * finished by then (the ticket stays valid). */
clod_status clod_serve_wait(clod_server* server, uint64_t ticket, int64_t timeout_us, clod_req_stats* stats);

/* Stops the worker after the batches in flight, frees the server. */
clod_status clod_server_destroy(clod_server* server);

/* ------------------------------------------------------------------------ */
/* Allocation-free forward render                                             */
/* ------------------------------------------------------------------------ */

/* One view rendered like clod_preprocess + clod_bin_sort + clod_render_fwd,
 * without any device allocation, for callers that cannot call cudaMalloc
 * (device memory owned by another framework's allocator, loops that must not
 * allocate after start-up, plug-ins given only raw pointers).  The paper has
 * no counterpart; it is an interface convenience.
 * All scratch lives in one file-scope __device__ array of about 16 MB that
 * every GPU loading the library holds until the process exits.  Limits:
 * scene->n <= 65536, width and height <= 1024, at most 2^21 pairs; larger
 * scenes or views are rejected with CLOD_ERR_ARG before any work, a frame
 * with more pairs returns CLOD_ERR_CAPACITY (with the count) and writes no
 * image.  image (3 x H x W), T_final (H x W, may be NULL), n_contrib (H x W,
 * may be NULL) are caller device buffers.  The call is synchronous: it
 * waits for the frame on its stream and reads the frame header back to the
 * host before returning, so it must not be called while its stream (or any
 * stream it depends on) is being captured into a CUDA graph.  Calls share the
 * array: calls whose work overlaps on the GPU race and must be serialised by
 * the caller.  The first call on a device also looks up the array's device
 * address, with that device current. */
clod_status clod_render_noalloc(const clod_scene* scene, const clod_view* view,
                                float* image, float* T_final, uint32_t* n_contrib,
                                clod_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* CLOD_H */
