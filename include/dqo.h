/* dqo.h -- C ABI of the GB300 (sm_103a) implementation of DQO-MAP's GPU optimisation
 * hot path (arXiv 2503.02223):
 *
 *   - the differentiable 3D Gaussian Splatting tile rasterizer the paper optimises its
 *     object Gaussians with (implemented, like its backward pass, as CUDA kernels per
 *     Sec. IV, implementation details): EWA projection, tile binning + depth radix
 *     sort, front-to-back blending of colour, depth, alpha, the instance channel
 *     ins (Eq. 15) and the object-id argmax map; the colour, depth and instance
 *     losses (Eq. 7-10) fused into the blend epilogue; and the full backward;
 *   - the dual-quadric pose step: Q* from (centre, semi-axes, rotation) (Eq. 1-3),
 *     C* = P Q* P^T (Eq. 4), BBox(C*) and the bbox loss of Eq. 12 with its gradient.
 *
 * Conventions shared by every call
 *   - Every array argument is a DEVICE pointer owned by the caller unless stated;
 *     the library never frees or retains it past the call's stream work.
 *   - Calls are asynchronous on the given stream (NULL = legacy default stream);
 *     results are valid after the stream synchronises.  dqo_render_forward
 *     synchronises the stream once, after binning, to size the pair buffers.
 *   - Argument errors return DQO_EINVAL before anything is launched.  CUDA errors
 *     return DQO_ECUDA; dqo_last_cuda_error() gives the cudaError_t code.
 *   - A context owns a grow-only device workspace (projected Gaussians, sort
 *     buffers, tile lists, per-pixel T_final / n_contrib, pixel loss gradients).  The
 *     state of the last dqo_render_forward stays valid for the matching
 *     dqo_render_backward on the same context; the next forward replaces it.  A
 *     context is not thread-safe; use one per host thread / stream.
 *   - Layouts are C-contiguous row-major; images are [H, W] (+ channel last).
 */
#ifndef DQO_H
#define DQO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define DQO_API __attribute__((visibility("default")))
#else
#define DQO_API
#endif

/* Same type as cudaStream_t (a CUstream handle); no CUDA header needed. */
typedef struct CUstream_st* dqo_stream;

typedef struct dqo_ctx dqo_ctx;

typedef enum {
  DQO_OK = 0,
  DQO_EINVAL = 1,   /* invalid argument (NULL pointer, size, setting out of range) */
  DQO_ENOMEM = 2,   /* device workspace allocation failed */
  DQO_ECUDA = 3,    /* a CUDA runtime call or launch failed */
  DQO_ETIMEOUT = 4, /* a bounded device wait ran out */
  DQO_ENOTIMPL = 5, /* not implemented */
  DQO_ESTATE = 6    /* backward without a matching forward on this context */
} dqo_status;

/* Rasterizer settings.  The paper inherits these from 3D Gaussian Splatting without
 * stating them; dqo_settings_default() gives the values below. */
typedef struct {
  int32_t tile_w, tile_h; /* tile shape in pixels; tile_w * tile_h == 256, tile_w in {8,16,32} (16x16) */
  float alpha_clamp;      /* alpha = min(alpha_clamp, opacity * G)                  (0.99)  */
  float alpha_min;        /* a Gaussian with alpha < alpha_min is skipped            (1/255) */
  float t_stop;           /* stop before the Gaussian that makes T (1-alpha) < t_stop (1e-4)  */
  float znear;            /* cull Gaussians with camera z < znear (m)                (0.2)   */
  float lowpass;          /* added to the 2D covariance diagonal (px^2)              (0.3)   */
  float radius_sigma;     /* screen radius = ceil(radius_sigma * sqrt(lambda_max))   (3)     */
  float lambda_ins;       /* lambda of Eq. 10                                        (1)     */
  float bg[3];            /* background colour                                       (0,0,0) */
  int32_t og_filter;      /* 1: only opaque (OG) Gaussians count toward ins, Eq. 15  (1)     */
  int32_t batch;          /* reserved: checked (32..256, multiple of 32) but unused -- every warp of the
                             blend kernels stages its own 32-Gaussian chunks                   (256) */
  float theta_alpha;      /* Eq. 11 instance threshold of Mask_geo (not given in the paper)    (0.5)   */
  float theta_d;          /* Eq. 11 depth threshold of Mask_geo (m)                            (0.1)   */
  float theta_c;          /* Eq. 11 colour threshold of Mask_rgb                               (0.1)   */
  int32_t grads_zero;     /* 0: Gaussian gradients are added (+=) to the caller's buffers; 1: the
                             call overwrites them with its own gradients (zero for culled Gaussians),
                             so the caller need not clear them first                      (0)     */
} dqo_settings;

typedef struct {
  float fx, fy, cx, cy;   /* pinhole intrinsics; pixel (u, v) centre is at integer (u, v) */
  int32_t width, height;  /* image size in pixels, each 1..32768 */
  float viewmat[12];      /* row-major [R | t], world -> camera, OpenCV axes (x right, y down, z forward) */
} dqo_camera;

/* Gaussians as structure-of-arrays (device pointers).  n may be 0. */
typedef struct {
  int64_t n;                  /* number of Gaussians, 0 .. 2^26 */
  int32_t num_objects;        /* object ids live in [0, num_objects), 1 .. 4096 */
  const float* means;         /* [n,3] world-space centres */
  const float* log_scales;    /* [n,3] log standard deviations along the local axes */
  const float* quats;         /* [n,4] rotation quaternion (w,x,y,z), normalised inside */
  const float* opacity_logit; /* [n]   opacity = sigmoid(logit) */
  const float* rgb;           /* [n,3] colour (SH degree 0, used as is) */
  const int32_t* obj_id;      /* [n]   object id; outside [0, num_objects) = no object */
  const uint8_t* flags;       /* [n]   bit0 = opaque Gaussian (OG), else transparent (TG) */
} dqo_gaussians;

/* Keyframe targets (device pointers, [H,W] images).  May be NULL as a whole: then no
 * loss is computed and dqo_render_backward needs explicit pixel gradients. */
typedef struct {
  const float* rgb;      /* [H,W,3] observed colour */
  const float* depth;    /* [H,W]   observed depth, <= 0 = no depth; may be NULL */
  const int32_t* gt_id;  /* [H,W]   observed instance id, -1 = unlabelled; must not be NULL */
} dqo_targets;

/* Forward outputs (device pointers; each may be NULL to skip it). */
typedef struct {
  float* rgb;       /* [H,W,3] C = sum_i w_i c_i + T_final bg,  w_i = alpha_i T_i */
  float* depth;     /* [H,W]   D = sum_i w_i z_i (camera z of the Gaussian centre) */
  float* alpha;     /* [H,W]   A = 1 - T_final */
  float* ins;       /* [H,W]   sum of w_i over the opaque Gaussians whose id equals the pixel's
                               gt_id (Eq. 15 reading); 0 without targets */
  int32_t* id_map;  /* [H,W]   argmax_k sum_{i: id_i = k} w_i, ties to the smaller id; -1 if empty */
  float* loss;      /* [4]     (L_rgb, L_depth, L_ins, L_total) of Eq. 7-10 (needs targets) */
  uint8_t* update_mask; /* [H,W] incremental-update masks of Eq. 11 (needs targets; 0 on unlabelled
                               pixels): bit0 Mask_geo = ins < theta_alpha or |D - D^| > theta_d (where
                               D^ > 0); bit1 Mask_rgb = max_c |C_c - C^_c| > theta_c.  Mask^{O_k} of
                               Eq. 13 = the pixels whose gt_id is k. */
} dqo_render_out;

/* Upstream gradients of the forward outputs (device pointers; each may be NULL = zero). */
typedef struct {
  const float* rgb;    /* [H,W,3] */
  const float* depth;  /* [H,W] */
  const float* alpha;  /* [H,W] */
  const float* ins;    /* [H,W] */
} dqo_pixel_grads;

/* Parameter gradients, ACCUMULATED (+=) into caller buffers, or overwritten when
 * dqo_settings.grads_zero is 1 (each may be NULL). */
typedef struct {
  float* means;          /* [n,3] */
  float* log_scales;     /* [n,3] */
  float* quats;          /* [n,4] */
  float* opacity_logit;  /* [n] */
  float* rgb;            /* [n,3] */
} dqo_gaussian_grads;

/* Intermediate buffers of the last forward, for inspection and parity tests. */
typedef enum {
  DQO_BUF_PROJ = 0,        /* float4 [3][n]: (x, y, a', b') (c', opacity, z, id|OG<<31) (r, g, b, lvl);
                              a', b', c' = conic (a, 2b, c) scaled by -log2(e)/2; lvl = log2(opacity /
                              alpha_min) (slightly widened; < 0 if alpha never reaches alpha_min) */
  DQO_BUF_RECT = 1,        /* uint16 [n][4]: tile rect (tx0, ty0, tx1, ty1), tx1/ty1 exclusive:
                              tiles holding a pixel centre in the 3-sigma square narrowed
                              (alpha_min > 0) to the bounding box of the ellipse where alpha
                              can reach alpha_min (K1 in csrc/k_preprocess.cu)             */
  DQO_BUF_DEPTH_ORDER = 2, /* uint32 [n]: Gaussian indices sorted by (z bits, index), visible first */
  DQO_BUF_TILE_RANGES = 3, /* uint32 [T][2]: [start, end) of each tile in the tile list */
  DQO_BUF_TILE_LIST = 4,   /* uint32 [M]: Gaussian indices ordered by (tile, z bits, index) */
  DQO_BUF_T_FINAL = 5,     /* float  [H,W] transmittance after the last blended Gaussian */
  DQO_BUF_N_CONTRIB = 6,   /* uint32 [H,W] 1 + position in the tile list of the last blended Gaussian */
  DQO_BUF_GRAD2D = 7       /* float  [n][12] backward moments (see dqo_render_backward) */
} dqo_buffer;

/* ------------------------------------------------------------------ context */

/* Fills *s with the defaults listed in dqo_settings. */
DQO_API void dqo_settings_default(dqo_settings* s);

/* Creates a context on CUDA device `device` (makes it current for the call).
 * Returns DQO_EINVAL for a NULL out pointer, DQO_ECUDA if the device is unusable. */
DQO_API dqo_status dqo_create(dqo_ctx** out, int device);

/* Frees the context's workspace.  NULL is allowed.  Waits for nothing: the caller must
 * ensure no work using the context is still running. */
DQO_API void dqo_destroy(dqo_ctx* ctx);

/* Static English name of a status code. */
DQO_API const char* dqo_status_str(dqo_status s);

/* cudaError_t of the last DQO_ECUDA returned on this context (0 if none). */
DQO_API int dqo_last_cuda_error(const dqo_ctx* ctx);

/* Library version as major*10000 + minor*100 + patch. */
DQO_API int dqo_version(void);

/* ------------------------------------------------------------------ rasterizer */

/* Forward render of one keyframe (3DGS rasterizer as used by DQO-MAP, Sec. III-D and
 * Sec. IV impl.; ins per Eq. 15 reading; losses per Eq. 7-10 reading):
 *   L_rgb   = 1/(HW) sum_{p: gt(p) >= 0} sum_c |C_c(p) - C^_c(p)|
 *   L_depth = 1/(HW) sum_{p: gt(p) >= 0, D^(p) > 0} |D(p) - D^(p)|
 *   L_ins   = 1/(HW) sum_{p: gt(p) >= 0} |ins(p) - 1|
 *   L_total = L_rgb + L_depth + lambda_ins L_ins
 * Stages: projection, depth radix sort, scan of tiles per Gaussian in depth order, pair
 * emission in depth order + a radix sort on the tile bits, tile ranges, tile schedule
 * (heaviest tiles first), blend + fused loss.  With targets, dL/d(pixel) is kept in the context for the
 * backward.  out->loss requires targets (DQO_EINVAL otherwise).
 * Errors: DQO_EINVAL (NULL ctx/settings/gaussians/camera/out, settings out of range,
 * n > 0 with a NULL input array, targets without gt_id or rgb), DQO_ENOMEM, DQO_ECUDA. */
DQO_API dqo_status dqo_render_forward(dqo_ctx* ctx, const dqo_settings* settings, const dqo_gaussians* g,
                              const dqo_camera* cam, const dqo_targets* targets,
                              dqo_render_out* out, dqo_stream stream);

/* Backward of the last forward on this context (same settings, Gaussians, camera and
 * targets).  Upstream pixel gradients: `pixel_grads` if non-NULL, else the gradient of
 * L_total saved by the forward (which then must have had targets).  Per pixel it walks
 * the blended Gaussians back to front from the saved T_final / n_contrib, sums
 * per-Gaussian partials over each warp (or per lane when few lanes contribute), then adds
 * them to a per-Gaussian
 * moment record (DQO_BUF_GRAD2D: sum over pixels of g dx, g dy, g dx^2, g dx dy, g dy^2
 * with g = dL/d(exponent), then dL/dopacity, dL/drgb (3), dL/dz), and chains the record
 * through the projection to the parameters, ACCUMULATING into `grads`.
 * Errors: DQO_EINVAL, DQO_ESTATE (no forward on this context, or different n / image
 * size / tile shape, or neither pixel_grads nor saved loss gradients), DQO_ECUDA. */
DQO_API dqo_status dqo_render_backward(dqo_ctx* ctx, const dqo_settings* settings, const dqo_gaussians* g,
                               const dqo_camera* cam, const dqo_targets* targets,
                               const dqo_pixel_grads* pixel_grads, dqo_gaussian_grads* grads,
                               dqo_stream stream);

/* Copies an intermediate buffer of the last forward into dst (device or host memory,
 * asynchronously on `stream`).  *bytes receives the buffer's size; if dst is NULL only
 * the size is returned.  DQO_EINVAL if capacity < size; DQO_ESTATE without a forward. */
DQO_API dqo_status dqo_get_buffer(dqo_ctx* ctx, dqo_buffer which, void* dst, size_t capacity,
                          size_t* bytes, dqo_stream stream);

/* Phases timed by dqo_set_timing / dqo_get_timings. */
typedef enum {
  DQO_PHASE_PROJECT = 0,     /* K1 projection */
  DQO_PHASE_DEPTH_SORT = 1,  /* depth radix sort, scan of tiles per Gaussian in depth order */
  DQO_PHASE_BINNING = 2,     /* pair emission, pair radix sort, tile ranges (after the host sync) */
  DQO_PHASE_BLEND_FWD = 3,   /* tile schedule, K6 blend + fused losses (+ loss reduction) */
  DQO_PHASE_BLEND_BWD = 4,   /* tile schedule, K7 blend backward */
  DQO_PHASE_PROJECT_BWD = 5, /* K8 projection backward */
  DQO_PHASE_QUADRIC = 6,     /* dual-quadric projection or bbox loss */
  DQO_PHASE_BLEND_STEP = 7,  /* dqo_batch_step: tile schedules, forward + backward blend, loss sums */
  DQO_PHASE_COUNT = 8
} dqo_phase;

/* Enables (1) or disables (0) CUDA-event timing of the phases above on the calls'
 * streams.  Off by default; when on, every call records a start / end event per phase. */
DQO_API dqo_status dqo_set_timing(dqo_ctx* ctx, int enable);

/* Device milliseconds of each phase in its most recent timed call (ms[DQO_PHASE_COUNT];
 * -1 for a phase not run since timing was enabled).  Waits for those events.  A call
 * captured in a CUDA graph records its events as graph nodes: each query then reads the
 * times of the latest replay.
 * n = capacity of ms.  DQO_EINVAL if ctx or ms is NULL or n < 1. */
DQO_API dqo_status dqo_get_timings(dqo_ctx* ctx, float* ms, int32_t n);

/* Number of kernels this context has launched since it was created. */
DQO_API int64_t dqo_launch_count(const dqo_ctx* ctx);

/* Sizes of the last forward: tile-Gaussian pairs M, visible Gaussians, tiles. */
DQO_API dqo_status dqo_get_counts(const dqo_ctx* ctx, int64_t* n_pairs, int64_t* n_visible, int32_t* n_tiles);

/* ------------------------------------------------------------------ allocation-free depth order */

/* Stable ascending sort of Gaussian indices by 32-bit depth keys, allocating nothing.
 * The paper has no counterpart: this is a library service for callers that cannot call
 * cudaMalloc while they run -- a real-time loop that must not take the implicit device
 * synchronisation of an allocation, a plugin whose host framework owns all device
 * memory, or a deployment with a fixed memory budget.  It runs the depth radix sort of
 * dqo_render_forward (DQO_BUF_DEPTH_ORDER) on keys the caller supplies.
 *   depth_keys [n] (device, read only): the float bit pattern of each Gaussian's positive
 *     camera depth, or 0xFFFFFFFF for a culled Gaussian (any uint32 keys sort correctly);
 *   order [n] (device, written): indices 0..n-1 ordered by (key, index);
 *   status (device, optional, written): 0 when `order` is valid, 1 when one of the sort's
 *     bounded look-back waits gave up after about a second (then `order` is not valid).
 *     Read it after the stream has synchronised.
 * Scratch memory is a fixed array of about 16 MiB inside the library, held by every GPU
 * that loads the library until the process exits.  n may be 0 .. 1048576 (2^20);
 * larger n returns DQO_EINVAL, as do NULL arrays with n > 0.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) for that device; with
 * CUDA's lazy module loading that lookup may also load the library's device code onto
 * that GPU, which allocates the array and synchronises the device.  Make one warm-up
 * call on each device before a real-time loop or any stream capture.  No call allocates
 * device or host memory itself.  All calls share the one scratch array, which keeps the
 * previous call's contents (each call clears the parts it needs, including its error
 * word): calls that overlap on the GPU race and must be serialised by the caller (for
 * example by issuing them on one stream).  Asynchronous on `stream`; DQO_ECUDA on a CUDA
 * failure. */
DQO_API dqo_status dqo_depth_order_noalloc(const uint32_t* depth_keys, int64_t n, uint32_t* order,
                                           uint32_t* status, dqo_stream stream);

/* ------------------------------------------------------------------ dual quadrics */

/* Projects dual quadrics into views (Eq. 1-4; reading C* = P Q* P^T).
 * params [nq,9]: centre (3), log semi-axes (3), rotation vector (3); Q* = Z diag(a^2,
 *   b^2, c^2, -1) Z^T with Z = [R t; 0 1].
 * P [nv,12]: row-major 3x4 camera matrices K [R|t].
 * Pairs in CSR: the pairs of quadric q are k = q_ptr[q] .. q_ptr[q+1]-1 (q_ptr[0] = 0,
 *   non-decreasing, q_ptr[nq] = npairs) and pair k uses view pair_v[k] in [0, nv).
 * Outputs per pair (each may be NULL): conic [npairs,6] = (c11 c12 c13 c22 c23 c33) of
 *   C*, bbox [npairs,4] = (u_min, v_min, u_max, v_max), valid [npairs].  A pair is valid
 *   iff c33 < 0 (ellipsoid clear of the principal plane), the centre is in front, and
 *   both tangent discriminants are positive; invalid pairs get a zero box.
 * Index arrays are device arrays; out-of-range view indices give valid = 0.
 * Errors: DQO_EINVAL (nq < 0, npairs < 0, NULL required arrays), DQO_ECUDA. */
DQO_API dqo_status dqo_quadric_project(dqo_ctx* ctx, int32_t nq, const float* params, int32_t nv,
                               const float* P, const int32_t* q_ptr, const int32_t* pair_v,
                               int32_t npairs, float* conic, float* bbox, uint8_t* valid,
                               dqo_stream stream);

/* Bbox loss of Eq. 12 (reading: J_k = sum over the valid views of quadric k of
 * (1 - IoU(BBox(C*_k), obs))) and its gradient.  Same pair layout as
 * dqo_quadric_project; obs_bbox [npairs,4] = (u_min, v_min, u_max, v_max).
 * loss [nq] and dparams [nq,9] are OVERWRITTEN (either may be NULL).  The gradient of
 * max/min in the intersection follows the predicted box only when it is strictly the
 * selected one; zero overlap gives a zero IoU gradient.
 * Errors: as dqo_quadric_project. */
DQO_API dqo_status dqo_quadric_bbox_loss(dqo_ctx* ctx, int32_t nq, const float* params, int32_t nv,
                                 const float* P, const int32_t* q_ptr, const int32_t* pair_v,
                                 int32_t npairs, const float* obs_bbox, float* loss,
                                 float* dparams, dqo_stream stream);

/* Plain multi-view fit of each quadric (Eq. 1 initialisation + Eq. 12 refinement), all
 * quadrics in one launch, one warp per quadric.
 *   Initialisation (Eq. 1, pi^T Q* pi = 0 for every plane pi = P^T l through a box edge
 *   line l): the 4V planes of a quadric's V >= 3 views, taken in a frame centred on the
 *   views' camera centres and scaled to unit mean distance and scaled to unit norm, give
 *   a 4V x 10 linear system in Q*'s entries; its least-squares null vector (smallest
 *   eigenvector of A^T A, fp64) is scaled to Q*44 = -1 and decomposed into centre
 *   t = -Q*[0:3,3] and R diag(a^2, b^2, c^2) R^T = Q*[0:3,0:3] + t t^T (axes descending,
 *   a^2 >= 1e-6 m^2, det R = +1).
 *   Refinement: `iters` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, step `lr`) on the
 *   bbox loss of dqo_quadric_bbox_loss (fp32).
 * start [nq,9] (device, may be NULL): if given, the refinement starts from these
 * parameters instead of the initialisation (any quadric with at least one view is ok; init
 * then holds the start).
 * Pairs in CSR as in dqo_quadric_project.  Outputs (device, each may be NULL): init [nq,9]
 * and params [nq,9] in the dqo_quadric_project parameterisation, loss [nq] at the final
 * parameters, ok [nq] (0 if fewer than 3 views or a degenerate system: zeros written).
 * Errors: DQO_EINVAL (nq < 0, iters < 0, NULL required arrays), DQO_ECUDA. */
DQO_API dqo_status dqo_quadric_fit(dqo_ctx* ctx, int32_t nq, int32_t nv, const float* P, const int32_t* q_ptr,
                                   const int32_t* pair_v, int32_t npairs, const float* obs_bbox, int32_t iters,
                                   float lr, const float* start, float* init, float* params, float* loss,
                                   uint8_t* ok, dqo_stream stream);

/* Canonical parameters of each quadric (same ellipsoid, same Q*): semi-axes in descending
 * order (equal axes keep their order), the rotation's columns permuted with them (the third
 * negated if needed for det +1), and of the four rotations that differ by negating two
 * columns, the one with the largest trace.  The learned proposal regresses this form.
 * params, out: device [nq,9] (may alias).  Errors: DQO_EINVAL, DQO_ECUDA. */
DQO_API dqo_status dqo_quadric_canonical(int32_t nq, const float* params, float* out, dqo_stream stream);

/* ---------------------------------------------------------------------------------------
 * Batched optimisation step.  The paper's GPU side optimises several keyframes and many
 * quadrics per mapping round (Sec. III-D, IV); this entry point runs one step for a
 * batch of keyframes of any resolutions and scenes, plus a batch of quadric fits, with
 * every phase a single launch over the whole batch, and captures cleanly in a CUDA graph.
 * ------------------------------------------------------------------------------------- */

#define DQO_MAX_BATCH 16

/* One keyframe of a batch: its scene, camera, targets (required: the step optimises the
 * fused losses), outputs (as dqo_render_forward; NULL members are skipped) and the
 * gradient buffers its step ADDS to (several keyframes may share a scene and its
 * gradient buffers: additions are atomic).  With dqo_settings.grads_zero = 1 the step
 * overwrites each keyframe's gradient buffers instead: buffers no other keyframe of the
 * batch uses are written once by the adjoint, shared ones (the same array pointer) are
 * cleared at the start of the step and then added to; buffers that overlap without being
 * the same array are not supported in that mode. */
typedef struct dqo_keyframe {
  dqo_gaussians gaussians;
  dqo_camera camera;
  dqo_targets targets;
  dqo_render_out out;
  dqo_gaussian_grads grads;
} dqo_keyframe;

/* A batch of plain quadric fits, as the arguments of dqo_quadric_fit. */
typedef struct dqo_fit_batch {
  int32_t nq, nv, npairs, iters;
  float lr;
  const float* P;
  const int32_t* q_ptr;
  const int32_t* pair_v;
  const float* obs_bbox;
  const float* start;
  float *init, *params, *loss;
  uint8_t* ok;
} dqo_fit_batch;

/* One optimisation step for nkf keyframes (1 <= nkf <= DQO_MAX_BATCH) and, if fits is not
 * NULL, a batch of quadric fits.  Per keyframe: the forward render with the fused losses
 * of Eq. 7-10 and 15 (out->loss [4] if given) and the backward of those losses, added to
 * kf->grads.  Results are those of dqo_render_forward + dqo_render_backward (pixel
 * gradients = the saved loss derivatives) on each keyframe alone; images are bitwise the
 * same, gradients up to the order of floating-point additions.  The fits run concurrently
 * on a second stream of the context, joined into `stream` before the call's work ends.
 *   Phases: projection, depth sort, scan, pair emission, pair sort and tile ranges each
 *   run once over all keyframes; the blend as `schedule` says, tiles heaviest first; then
 *   the per-keyframe loss sums and the projection adjoint.
 * Sizing: the first call, and any call whose batch layout (keyframe count, Gaussian
 * counts, image sizes, tile shape) differs from the previous one, waits once on the host
 * for the pair count and sizes the pair buffers with 25% headroom; other calls do not
 * synchronise or allocate (so they can be captured in a CUDA graph) and read the pair
 * count on the device.  If a later step needs more pairs than that capacity, pairs past
 * it are dropped and dqo_batch_check reports it (and makes the next step a sizing call).
 * settings->tile_w/tile_h apply to every keyframe.  schedule selects how the blend runs:
 *   DQO_SCHEDULE_FUSED (0): one persistent kernel, each tile's forward then its backward;
 *   DQO_SCHEDULE_SPLIT (1): a persistent forward kernel then a persistent backward kernel,
 *     each on its own work queue;
 *   DQO_SCHEDULE_PER_KEYFRAME (2): the one-keyframe forward and backward kernels launched
 *     per keyframe.
 * ctas_per_sm bounds the persistent kernels' CTAs per SM (<= 0: as many as fit).
 * Errors: DQO_EINVAL (bad arguments, nkf out of range, missing targets, unknown schedule),
 * DQO_ENOMEM, DQO_ESTATE (a sizing call while the stream is being captured), DQO_ECUDA. */
#define DQO_SCHEDULE_FUSED 0
#define DQO_SCHEDULE_SPLIT 1
#define DQO_SCHEDULE_PER_KEYFRAME 2
DQO_API dqo_status dqo_batch_step(dqo_ctx* ctx, const dqo_settings* settings, int32_t nkf,
                                  const dqo_keyframe* kfs, const dqo_fit_batch* fits, int32_t ctas_per_sm,
                                  int32_t schedule, dqo_stream stream);

/* After the last dqo_batch_step has completed: pairs it needed and whether they exceeded
 * the capacity (synchronous). */
DQO_API dqo_status dqo_batch_check(dqo_ctx* ctx, uint64_t* pairs, int* overflow);

/* Autotuner of the batched step: times each of DQO_TUNE_CANDIDATES candidates over `reps`
 * steps on this batch (CUDA events on the stream; gradients accumulate into kfs' buffers
 * while it runs) and writes the fastest tile shape into settings, its CTAs per SM into
 * *ctas_per_sm and its schedule into *schedule.  Candidate i: tile shape i / 7 of
 * (16x16, 8x32, 32x8); j = i % 7: j < 3 fused with 2 + j CTAs per SM, 3 <= j < 6 split
 * with j - 1 CTAs per SM, j = 6 per keyframe.  ms [DQO_TUNE_CANDIDATES] (host, may be
 * NULL) receives each candidate's mean step time.  Errors: as dqo_batch_step. */
#define DQO_TUNE_CANDIDATES 21
DQO_API dqo_status dqo_batch_tune(dqo_ctx* ctx, dqo_settings* settings, int32_t nkf, const dqo_keyframe* kfs,
                                  const dqo_fit_batch* fits, int32_t reps, int32_t* ctas_per_sm,
                                  int32_t* schedule, float* ms, dqo_stream stream);

/* ---------------------------------------------------------------------------------------
 * Learned quadric proposal.  The paper initialises each quadric geometrically (Eq. 1);
 * this small network proposes the initial value from up to 8 views instead, including
 * from 2 views, where the Eq. 1 system is underdetermined, and dqo_quadric_fit (start =
 * the proposal) refines it on the Eq. 12 loss.  The plain fit stays the fallback and the
 * reference its error is measured against.
 * Network: 128 features -> 128 -> 128 -> 9 (ReLU after the two hidden layers), output =
 * canonical quadric parameters (dqo_quadric_canonical).  BF16 operands (features, weights,
 * activations, output gradients), FP32 accumulation on the tensor cores, FP32 biases,
 * master weights and Adam state.
 * BF16 arrays cross this interface as uint16_t (the bit pattern of bfloat16).
 * ------------------------------------------------------------------------------------- */

#define DQO_MLP_FEATURES 128
#define DQO_MLP_PARAMS 35088
/* Parameter vector (fp32, DQO_MLP_PARAMS): W1 [128][128] (row = output unit), b1 [128],
 * W2 [128][128], b2 [128], W3 [16][128] (rows 9..15 must be zero), b3 [16] (9..15 zero). */

typedef struct dqo_mlp_hparams {
  float lr;              /* Adam step at the start of the cosine schedule */
  float lr_final;        /* ... and at step total_steps and after */
  int64_t total_steps;   /* schedule length (<= 0: constant lr) */
  float beta1, beta2, eps;
  float loss_w[9];       /* per-output weights of the squared error */
} dqo_mlp_hparams;

/* Features of each quadric (device in, device out): view slot j < min(counts[q] (or 8 if
 * counts is NULL), views of q, 8) holds the j-th view of q in its CSR list; later slots
 * are zero.  For a slot, P = K [R | t] (K upper triangular with positive diagonal; the
 * overall scale and sign of P are normalised) gives camera axes r1, r2, r3 (rows of R)
 * and centre C = -R^T t; with the box centre in normalised image coordinates (xn, yn),
 * its half-extents (hw, hh) = ((u1-u0)/(2 fx), (v1-v0)/(2 fy)) and d the unit direction of
 * the ray through the box centre (xn r1 + yn r2 + r3, normalised), the slot is
 *   [xn, yn, hw, hh, r1, r2, d, C / length_scale]      (4 + 12 values).
 * X [nq][128] BF16; XT [128][ldt] BF16 (may be NULL), XT[f][q] = X[q][f]; ldt >= nq and a
 * multiple of 8.  Errors: DQO_EINVAL (bad sizes, NULL, length_scale <= 0), DQO_ECUDA. */
DQO_API dqo_status dqo_mlp_features(int32_t nq, int32_t nv, const float* P, const int32_t* q_ptr,
                                    const int32_t* pair_v, int32_t npairs, const float* obs_bbox,
                                    const int32_t* counts, float length_scale, uint16_t* X, uint16_t* XT,
                                    int64_t ldt, dqo_stream stream);

/* Size in bytes of an MLP state buffer (parameters, gradient, Adam moments, BF16 weight
 * copies, step count).  The caller allocates it on the device (256-byte aligned). */
DQO_API size_t dqo_mlp_state_bytes(void);
/* params (device, fp32 DQO_MLP_PARAMS) -> state; resets the Adam moments and step count. */
DQO_API dqo_status dqo_mlp_set_params(void* state, const float* params, dqo_stream stream);
/* state -> params (device, fp32 DQO_MLP_PARAMS). */
DQO_API dqo_status dqo_mlp_get_params(const void* state, float* params, dqo_stream stream);

/* Proposal for n quadrics: X [n][128] BF16 (device) -> out [n][9] fp32 (device). */
DQO_API dqo_status dqo_mlp_forward(dqo_ctx* ctx, const void* state, int64_t n, const uint16_t* X, float* out,
                                   dqo_stream stream);

/* Loss L = (1/n) sum_rows sum_j loss_w[j] (y_j - labels_j)^2 of a batch and its gradient
 * w.r.t. the parameter vector.  n > 0, n % 128 == 0.  X [n][128] BF16 and labels [n][9]
 * fp32 (device, 16-byte aligned); loss_w: 9 host floats.  grads (device, DQO_MLP_PARAMS,
 * 16-byte aligned) and loss (device, 1 float) are OVERWRITTEN.  Backward precision: dL/dy
 * rounded to BF16, hidden-layer gradients rounded to BF16 after the ReLU derivative (the
 * activation > 0); weight and bias gradients accumulate in FP32.  Each 128-sample tile's
 * gradient comes from one CTA (every product on tensor cores, intermediates in shared
 * memory); the tiles' gradients are summed in tile order, so the result is the same on
 * every run.  One cooperative launch of one CTA per SM (the GPU must be able to hold the
 * whole grid at once).
 * Errors: DQO_EINVAL, DQO_ECUDA (a wait that ran out is reported by dqo_mlp_check). */
DQO_API dqo_status dqo_mlp_gradients(dqo_ctx* ctx, void* state, int64_t n, const uint16_t* X, const float* labels,
                                     const float* loss_w, float* grads, float* loss, dqo_stream stream);

/* `steps` Adam steps, step k on rows [k batch, (k + 1) batch) of X [steps * batch][128]
 * BF16 and labels [steps * batch][9] fp32 (device, 16-byte aligned; batch % 128 == 0).
 * Each step is dqo_mlp_gradients' gradient of its batch followed by the Adam update (the
 * learning rate follows hp's cosine schedule at the state's step count, which advances by
 * one per step).  losses (device, `steps` floats, may be NULL) are OVERWRITTEN with each
 * step's batch loss before its update.  One cooperative launch runs all the steps: per step
 * the tiles' gradients, a grid-wide barrier, Adam on a slice of the parameters per CTA, a
 * grid-wide barrier.  The result equals `steps` calls of dqo_mlp_train_step on the same
 * batches.  Allocates nothing once the context has seen a batch of this size.
 * Errors: as dqo_mlp_gradients. */
DQO_API dqo_status dqo_mlp_train_steps(dqo_ctx* ctx, void* state, const dqo_mlp_hparams* hp, int32_t steps,
                                       int64_t batch, const uint16_t* X, const float* labels, float* losses,
                                       dqo_stream stream);

/* One Adam step on a batch of n rows: dqo_mlp_train_steps with steps = 1; loss (device,
 * 1 float, may be NULL) is OVERWRITTEN with the batch loss before the update. */
DQO_API dqo_status dqo_mlp_train_step(dqo_ctx* ctx, void* state, const dqo_mlp_hparams* hp, int64_t n,
                                      const uint16_t* X, const float* labels, float* loss, dqo_stream stream);

/* Error flag of the last tensor-core kernels on this context, read synchronously and
 * cleared: *timed_out = 1 and DQO_ETIMEOUT if a tensor-core completion wait ran out (the
 * kernel then skipped its epilogue, freed its tensor memory and returned). */
DQO_API dqo_status dqo_mlp_check(dqo_ctx* ctx, int* timed_out);

/* Exercises the bounded device waits the tensor-core kernels use: one kernel waits on an
 * mbarrier that nothing arrives at, then on the training kernel's grid barrier with a
 * count its single CTA never reaches; each gives up after about one second and records
 * it.  The call synchronises `stream` and returns DQO_ETIMEOUT when both gave up (DQO_OK
 * would mean one of them did not).  The context stays usable afterwards.  No counterpart
 * in the paper: this is how a stalled completion is reported instead of hanging the GPU. */
DQO_API dqo_status dqo_wait_probe(dqo_ctx* ctx, dqo_stream stream);

/* Throughput probe of one arithmetic pipe, for the roofline the blend kernels are quoted
 * against (no counterpart in the paper).  kind 0: FP32 fused multiply-add; kind 1: the
 * special-function unit's 2^x (ex2.approx), the exponential of every blend evaluation.
 * One launch fills every SM of the current device (8 CTAs of 256 threads per SM), each
 * thread running 8 independent chains of iters x 16 operations.  *ops (host) receives
 * the launch's operation count: flops for kind 0 (an FMA counts 2), exponentials for
 * kind 1; the caller times the launch on `stream` (CUDA events) and divides.  sink: one
 * device float, written only by an impossible outcome (it keeps the work live).
 * Errors: DQO_EINVAL (kind not 0/1, iters < 1, NULL pointers), DQO_ECUDA. */
DQO_API dqo_status dqo_alu_probe(int32_t kind, int32_t iters, float* sink, double* ops, dqo_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* DQO_H */
