/*
 * gsr.h -- C ABI of the GB300 Gaussian-splatting rasterizer with se(3) pose
 * gradient (libgsr.so).
 *
 * The operation is the rendering step of the dense render-and-match stage of
 * Hi^2-GSLoc (arXiv 2507.15683): Sec. 3.1 defines the scene as Gaussians
 * Theta_i = {centre (x, y, z), rotation q, scale s, opacity, colour c, feature
 * f}, rendered by tile-based rasterization with alpha blending, features going
 * through the identical blending; Sec. 3.4 renders feature, depth and colour
 * maps at a candidate pose on every refinement iteration; Algorithm 1 fixes the
 * projection (world -> camera by T, depth = camera z, perspective division,
 * then K) and Eq. 10 the pinhole map pi([x, y, z]) = [x/z, y/z].
 *
 * Conventions shared by every entry point
 *  - All functions return gs_status and never abort. On failure the
 *    thread-local message of gs_last_error() says why.
 *  - "device" pointers are CUDA device (or managed) memory of the current
 *    device; "host" pointers are ordinary host memory.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued on it; functions documented as synchronous also wait for
 *    it before returning.
 *  - Images are planar, row-major: channel c of pixel (x, y) sits at
 *    [c * H * W + y * W + x]. Pixel (x, y) has its centre at (x + 0.5, y + 0.5)
 *    in the frame of the projected coordinates.
 *  - A pose is a row-major 4x4 world-to-camera matrix T_cw (camera x right,
 *    y down, z forward), applied as p_cam = R X + t (Algorithm 1).
 *  - The pose tangent is xi = (rho, phi): T(xi) = Exp(xi^) T_cw (left
 *    perturbation, rho first), derivatives taken at xi = 0.
 *  - One scene may be used from one stream at a time (its workspace is shared
 *    by all calls on it); distinct scenes are independent.
 *
 * Fixed constants (the paper leaves them open): 16 x 16 tiles, near plane 0.2,
 * EWA footprint with 0.3 px dilation, 1.3 x half field of view guard on the
 * Jacobian and a 0.1 floor under the eigenvalue discriminant, radius =
 * ceil(3 sqrt(lambda_max)), alpha = min(0.99, o exp(power)), Gaussians with
 * alpha < 1/255 skipped, blending stops before a Gaussian that would take the
 * transmittance below 1e-4, background 0, depth = sum of w * z (not
 * normalised), colour = max(0, SH(dir) + 0.5) with dir = normalize(mean -
 * camera centre), real SH with the Condon-Shortley phase, coefficient index
 * l*l + l + m. Within a tile Gaussians are blended in ascending (binary32
 * camera depth bits, Gaussian index) order.
 */
#ifndef GSR_H
#define GSR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GS_OK = 0,
  GS_ERR_INVALID_ARG = 1, /* a pointer, size or enum is out of its documented range */
  GS_ERR_CUDA = 2,        /* a CUDA runtime call failed (message has the CUDA error) */
  GS_ERR_OOM = 3,         /* device or pinned host allocation failed */
  GS_ERR_CAPACITY = 4,    /* an asynchronous call outgrew the reserved workspace */
  GS_ERR_TIMEOUT = 5,     /* a bounded device wait ran out (gs_pmm_match); the context stays usable */
  GS_ERR_INTERNAL = 6     /* a device-side consistency check failed */
} gs_status;

typedef struct gs_scene gs_scene; /* opaque */

/* Scene description (Sec. 3.1 primitive). Arrays are row-major per Gaussian.
 * The scene copies what it needs into its own device arena: the caller may
 * free every array once gs_create_scene returns. */
typedef struct {
  int64_t n;                  /* number of Gaussians, >= 0 and < 2^31 */
  int sh_degree;              /* 0..3 */
  int feat_dim;               /* 0 or 32 */
  const float* means;         /* n x 3, world coordinates */
  const float* scales;        /* n x 3, linear standard deviations (> 0, not log) */
  const float* quats;         /* n x 4, (w, x, y, z); normalised inside; 0 -> identity */
  const float* opacities;     /* n, in (0, 1) (after the sigmoid) */
  const float* sh;            /* n x (deg+1)^2 x 3, coefficient-major */
  const uint16_t* feats_bf16; /* n x feat_dim bfloat16 bit patterns, NULL when feat_dim = 0 */
  int n_partitions;           /* 0 = one partition; else partition_offsets has n_partitions+1 entries */
  const int64_t* partition_offsets; /* host; ascending Gaussian index ranges, [0] = 0, [last] = n */
  int device_resident;        /* 1: the arrays above are device pointers; 0: host pointers */
} gs_scene_desc;

typedef struct {
  int width, height;          /* pixels, 1 .. 65535 * 16 */
  float fx, fy, cx, cy;       /* pinhole intrinsics K (Eq. 10) */
} gs_camera;

typedef struct {
  double T_cw[16];            /* row-major world-to-camera */
} gs_pose;

/* Caller-owned device output buffers of one view (H x W pixels). Any pointer
 * may be NULL to skip that output. */
typedef struct {
  float* rgb;        /* 3 x H x W */
  float* depth;      /* H x W, sum of w * z */
  float* alpha;      /* H x W, 1 - final transmittance */
  float* final_T;    /* H x W, final transmittance (>= 1e-4) */
  float* feats;      /* feat_dim x H x W, blended BF16 features accumulated in fp32 */
  uint32_t* last_idx;/* H x W, 1 + position in the tile list of the last blended Gaussian */
} gs_outputs;

/* Batch flags */
#define GS_BATCH_GRAPH 1u      /* capture the batch once into a CUDA graph and replay it */

/* Create a scene (Sec. 3.1). Packs the Gaussians into the device layout used by
 * the kernels (centre + max scale, binary32 3D covariance + opacity, SH
 * coefficients, features). Synchronous. *out receives the handle; destroy it
 * with gs_destroy_scene. Errors: INVALID_ARG (NULL pointer with n > 0, degree
 * or feature width out of range, bad partition table), OOM, CUDA. */
gs_status gs_create_scene(const gs_scene_desc* desc, gs_scene** out);

/* Release the scene and its device memory. Waits for its work. NULL is a no-op. */
void gs_destroy_scene(gs_scene* scene);

/* Reserve workspace for up to max_records projected (view, Gaussian) records
 * and max_pairs (tile, Gaussian) pairs, so that asynchronous calls and graph
 * replays never outgrow it. Synchronous. Errors: INVALID_ARG, OOM, CUDA. */
gs_status gs_scene_reserve(gs_scene* scene, int64_t max_records, int64_t max_pairs);

/* Render one view (Sec. 3.1 rasterization at the pose of Sec. 3.4).
 * Synchronous: waits for the stream, and when the workspace was too small
 * grows it and renders again, so the outputs are complete on return.
 * Errors: INVALID_ARG, OOM, CUDA. */
gs_status gs_render(gs_scene* scene, const gs_camera* cam, const gs_pose* pose, const gs_outputs* out,
                    void* stream);

/* Same as gs_render but only enqueues work. If the workspace is too small the
 * outputs are invalid and gs_scene_status() reports GS_ERR_CAPACITY. */
gs_status gs_render_async(gs_scene* scene, const gs_camera* cam, const gs_pose* pose,
                          const gs_outputs* out, void* stream);

/* Render one view and the gradient of
 *   L = 1/(3P) sum_px,c w_px |C - C*| + depth_weight * 1/P sum_px w_px |D - D*|
 * (P = W * H, w_px = pixel_weight or 1, sign(0) = 0) with respect to the pose
 * tangent xi = (rho, phi) (left perturbation, T(xi) = Exp(xi^) T_cw). One
 * compositing pass carries the six pose derivatives of colour, depth and
 * transmittance through the front-to-back blend; the per-pixel terms are
 * summed in fp32 per tile and in fp64 across tiles, in a fixed order.
 * target_rgb (3 x H x W), target_depth (H x W) and pixel_weight (H x W or
 * NULL) are device pointers. loss_out (1) and grad_xi_out (6) are host
 * pointers written before return (synchronous, with the same regrow rule as
 * gs_render). out may be NULL or have NULL members (those outputs are not
 * written). Errors: INVALID_ARG, OOM, CUDA. */
gs_status gs_render_pose_grad(gs_scene* scene, const gs_camera* cam, const gs_pose* pose,
                              const float* target_rgb, const float* target_depth, const float* pixel_weight,
                              float depth_weight, const gs_outputs* out, double* loss_out,
                              double* grad_xi_out, void* stream);

/* gs_render_pose_grad with the loss inputs in host memory: target_rgb
 * (3 x H x W), target_depth (H x W) and pixel_weight (H x W or NULL) are host
 * pointers. When all of them are page-locked (pinned) memory mapped into the
 * device's address space (cudaMallocHost / cudaHostRegister on a unified-
 * addressing system), the compositing pass reads them in place over the
 * CPU-GPU link, each pixel once at the end of its tile. Otherwise they are
 * copied into a scene-owned device buffer on a side stream, in bands of tile
 * rows, and each band of the compositing pass waits only for its rows. The
 * host buffers may be reused once the call returns. Everything else as
 * gs_render_pose_grad (the results are bit-identical to it). Errors:
 * INVALID_ARG, OOM, CUDA. */
gs_status gs_render_pose_grad_host(gs_scene* scene, const gs_camera* cam, const gs_pose* pose,
                                   const float* target_rgb, const float* target_depth, const float* pixel_weight,
                                   float depth_weight, const gs_outputs* out, double* loss_out,
                                   double* grad_xi_out, void* stream);

/* Asynchronous form of gs_render_pose_grad: result_dev (device, 7 doubles)
 * receives (loss, grad rho_x, rho_y, rho_z, phi_x, phi_y, phi_z). Capacity
 * overflow is reported by gs_scene_status(). */
gs_status gs_render_pose_grad_async(gs_scene* scene, const gs_camera* cam, const gs_pose* pose,
                                    const float* target_rgb, const float* target_depth,
                                    const float* pixel_weight, float depth_weight, const gs_outputs* out,
                                    double* result_dev, void* stream);

/* Render n_views views of possibly different sizes (candidate poses and
 * pyramid levels of Sec. 3.4) in one pass: one projection launch over all
 * (view, Gaussian) pairs, one global tile space, one persistent compositing
 * launch over every view's tiles. cams, poses and outs are host arrays of
 * n_views entries (outs hold device pointers). Each view's outputs equal those
 * of gs_render for that view. flags: 0 = synchronous (regrow rule of
 * gs_render); GS_BATCH_GRAPH = asynchronous replay of a CUDA graph captured on
 * the first call for this (n_views, cams, outs) layout -- poses may change
 * between calls; reserve the workspace first (gs_scene_reserve) and check
 * gs_scene_status(). Errors: INVALID_ARG, OOM, CUDA. */
gs_status gs_render_batch(gs_scene* scene, int n_views, const gs_camera* cams, const gs_pose* poses,
                          const gs_outputs* outs, unsigned flags, void* stream);

/* Batched pose gradient: the candidate poses / pyramid levels of Sec. 3.4
 * rendered and differentiated in one pass (one projection launch, one global
 * tile space, one persistent compositing launch and one persistent backward
 * launch over every view's tiles). For each view v the loss and gradient equal
 * those of gs_render_pose_grad for that view alone (bit for bit).
 * target_rgb, target_depth: host arrays of n_views device pointers (3 x H x W
 * and H x W of that view); pixel_weight: NULL or a host array of n_views device
 * pointers (entries may be NULL). outs: NULL or n_views output sets.
 * flags 0: synchronous (regrow rule of gs_render); loss_out (host, n_views)
 * and grad_out (host, n_views x 6) are written when not NULL; results_dev,
 * when not NULL, also receives them. GS_BATCH_GRAPH: asynchronous replay of a
 * CUDA graph captured on the first call for this layout (cameras, outputs,
 * targets, weights, results_dev); poses may change between calls; results_dev
 * (device, n_views x 8 doubles: loss, 6 gradient entries, 0) is required and
 * loss_out / grad_out are not written. Errors: INVALID_ARG, OOM, CUDA. */
gs_status gs_render_pose_grad_batch(gs_scene* scene, int n_views, const gs_camera* cams, const gs_pose* poses,
                                    const float* const* target_rgb, const float* const* target_depth,
                                    const float* const* pixel_weight, float depth_weight, const gs_outputs* outs,
                                    double* loss_out, double* grad_out, double* results_dev, unsigned flags,
                                    void* stream);

/* Pose refinement (the render-and-refine loop of Sec. 3.4, done by gradient
 * descent on the loss of gs_render_pose_grad). Every iteration renders,
 * differentiates, takes an Adam step s on the tangent xi = (rho, phi) --
 * per-component step size lr_trans for rho, lr_rot for phi, moments carried
 * across iterations -- and applies the left update T <- Exp(-s^) T, so the
 * tangent is re-linearised at the current pose. */
typedef struct {
  int iterations;      /* number of render + gradient + update steps (>= 0) */
  double lr_rot;       /* Adam step size of the rotation part (rad) */
  double lr_trans;     /* Adam step size of the translation part (scene units) */
  double beta1, beta2; /* Adam moment decays, in [0, 1) */
  double eps;          /* Adam denominator floor, > 0 */
  float depth_weight;  /* lambda_d of the loss */
} gs_refine_opts;

/* Defaults: 50 iterations, lr_rot 1e-3, lr_trans 0.5, betas 0.9 / 0.999,
 * eps 1e-8, depth weight 0.1. */
gs_refine_opts gs_refine_defaults(void);

/* Refine one pose in place (pose: host, updated). Targets and weights as in
 * gs_render_pose_grad. loss_history: host array of opts->iterations (the loss
 * before each update) or NULL. Synchronous.
 * On a scene of one partition that is not streamed, the Adam step and the pose
 * update run on the device (fp64) after every pass and the iterations after
 * the first replay one CUDA graph without a host round trip; the workspace is
 * sized by the first pass with 50% headroom, and a later pass that outgrows it
 * doubles it and restarts the refinement. Other scenes take the step on the
 * host after every pass (their partitions are culled per pose).
 * Errors: those of gs_render_pose_grad, INVALID_ARG for bad options, OOM. */
gs_status gs_refine_pose(gs_scene* scene, const gs_camera* cam, gs_pose* pose, const float* target_rgb,
                         const float* target_depth, const float* pixel_weight, const gs_refine_opts* opts,
                         double* loss_history, void* stream);

/* Refine n_views poses together (poses: host array, updated in place): every
 * iteration is one batched pose-gradient pass, then one Adam update per view,
 * on the device or the host as for gs_refine_pose. Each view's poses equal
 * those of gs_refine_pose on that view alone. Targets and weights as in
 * gs_render_pose_grad_batch. loss_history: host array n_views x iterations or
 * NULL. Synchronous. */
gs_status gs_refine_poses_batch(gs_scene* scene, int n_views, const gs_camera* cams, gs_pose* poses,
                                const float* const* target_rgb, const float* const* target_depth,
                                const float* const* pixel_weight, const gs_refine_opts* opts,
                                double* loss_history, void* stream);

/* Wait for the stream and return the device status of the last call (GS_OK,
 * or GS_ERR_CAPACITY / GS_ERR_INTERNAL from an asynchronous call).
 * needed_records / needed_pairs (host, may be NULL) receive the workspace the
 * last call needed (record capacity, pair count), to pass to
 * gs_scene_reserve. */
gs_status gs_scene_status(gs_scene* scene, void* stream, int64_t* needed_records, int64_t* needed_pairs);

/* Sorted tile lists of view `view` of the last render (parity/debugging).
 * Synchronous. keys (host, capacity) receive tile << 32 | depth bits, gids
 * (host, capacity) the Gaussian indices, tile_start (host, tiles + 1) the
 * list boundaries; *n_pairs (host) the list length. Errors: INVALID_ARG when
 * the view does not exist or capacity is too small (n_pairs still set). */
gs_status gs_get_tile_lists(gs_scene* scene, int view, uint64_t* keys, uint32_t* gids, int64_t* tile_start,
                            int64_t capacity, int64_t* n_pairs, void* stream);

/* Projected records of view `view` of the last render (parity/debugging).
 * Synchronous. For each of the *n_records visible Gaussians (in no particular
 * order) rec (host, capacity x 10 int32) receives: Gaussian index, x0, x1, y0,
 * y1 (inclusive tile rectangle), the bit pattern of the binary32 camera depth
 * (the sort key), then the projected centre used for blending as float-float
 * bit patterns u_hi, u_lo, v_hi, v_lo (u = u_hi + u_lo).
 * Errors: INVALID_ARG (bad view, capacity too small). */
gs_status gs_get_records(gs_scene* scene, int view, int32_t* rec, int64_t capacity, int64_t* n_records,
                         void* stream);

/* Partitions (Sec. 3.1: large scenes are split into cells). Every call walks
 * only the partitions whose padded bounding box can reach one of its views'
 * tiles (a conservative frustum test: the results are those of rendering every
 * Gaussian). A scene created with device_resident = 0 and a partition table
 * is streamed: it keeps a packed copy in pinned host memory and uploads a
 * partition to the device the first time a call needs it.
 * gs_scene_stream_stats reports the bytes uploaded so far, the partitions now
 * on the device and the partitions the last call walked (host pointers, any
 * may be NULL). gs_scene_evict marks every partition of a streamed scene as
 * not resident (they are uploaded again when needed; no memory is freed). */
gs_status gs_scene_stream_stats(gs_scene* scene, int64_t* h2d_bytes, int* resident_partitions,
                                int* active_partitions);
gs_status gs_scene_evict(gs_scene* scene);

/* Gaussian count, SH degree and feature channels of a scene (host pointers,
 * each may be NULL). Errors: INVALID_ARG (NULL scene). */
gs_status gs_scene_shape(const gs_scene* scene, int64_t* n, int* sh_degree, int* feat_dim);

/* Kernel timing (CUDA events recorded on the call's stream around every
 * launch of every call while enabled). Kernel order of the arrays below:
 * projection (discrete layer), shading (conic, colour, centre, Jacobian),
 * tile scan, scatter, warp sort of the short tile lists, compositing (block
 * sort of longer lists, blending, and for the pose gradient the tangent pass
 * with the fp64 reduction); then, in gs_visibility calls only, the reverse
 * pass (with the zeroing of its accumulators) and the per-Gaussian selection
 * (in-image test, chain rule, compaction). */
#define GS_KERNEL_COUNT 8
gs_status gs_scene_set_timing(gs_scene* scene, int enable);

/* Wait for the recorded calls and return, per kernel, the summed device time
 * (ms, host array of GS_KERNEL_COUNT) and the number of launches timed (host
 * array of GS_KERNEL_COUNT, may be NULL) since timing was enabled or last read;
 * then reset the sums. Errors: INVALID_ARG, CUDA. */
gs_status gs_scene_kernel_times(gs_scene* scene, double* total_ms, int64_t* launches);

/* Number of (pixel, Gaussian) pairs that the last pose-gradient call blended
 * (alpha accumulated into a pixel before its transmittance cutoff), summed
 * over its views: the work unit of the tangent pass, for roofline accounting.
 * 0 after a forward-only call. Waits for `stream`. `blended` is a host
 * pointer. Errors: INVALID_ARG, CUDA. */
gs_status gs_scene_blend_count(gs_scene* scene, void* stream, int64_t* blended);

/* Work units of the last call's backward walk, for roofline accounting:
 * blended = (pixel, Gaussian) pairs blended (as gs_scene_blend_count; after a
 * gs_visibility call, the pairs its reverse pass walked back through), and
 * evaluated = after a pose-gradient call, the tile-list entries its pixels
 * examined before their stop (each pixel's list up to and including the
 * entry that stopped it, else the whole list: the per-pixel walk of the
 * definition); after gs_visibility, the (pixel, Gaussian) pairs whose
 * footprint the reverse pass evaluated (a pair before the pixel's last
 * blended Gaussian whose tile entry hits the pixel's 8 x 4 block); 0 after a
 * forward-only call. Waits for `stream`; host pointers, either may be NULL.
 * Errors: INVALID_ARG, CUDA. */
gs_status gs_scene_work_counts(gs_scene* scene, void* stream, int64_t* blended, int64_t* evaluated);

/* ---- Launch configurations and the autotuner ----------------------------
 * The dense stage renders candidate poses at the levels of a coarse-to-fine
 * pyramid (Sec. 3.4: H_f / H_c = 8; 480x270 to 3840x2160 views here), and one
 * launch shape does not suit every level or batch. A launch configuration
 * applies to one call shape: the multiset of the call's view sizes (a
 * single view, or every view of a batch call), for one mode. It sets
 *   - the compositor variant (variant 0 is the default): the number of
 *     Gaussians staged in shared memory per batch, and the resident CTAs per
 *     SM its register allocation allows for;
 *   - the persistent compositor grid, in CTAs per SM (0: as many as the
 *     variant's occupancy allows);
 *   - the CTAs per SM of the projection, shading, scatter and sort kernels.
 * No configuration changes a result: the blending order and every reduction
 * order are fixed by the tile lists, so every configuration gives the same
 * bits. Shapes without a configuration use the defaults. Changing one makes
 * the next graph-mode batch call capture its graph again. */
#define GS_MODE_FORWARD 0     /* forward render without features */
#define GS_MODE_FEATURES 1    /* forward render with the feature map */
#define GS_MODE_POSE_GRAD 2   /* pose-gradient call (the tangent pass) */
#define GS_COMPOSITE_VARIANTS 4

typedef struct {
  int variant;      /* compositor variant, 0..GS_COMPOSITE_VARIANTS-1 */
  int ctas_per_sm;  /* persistent compositor CTAs per SM; 0 = the variant's occupancy */
  int grid_mult;    /* CTAs per SM of projection, shading, scatter and sort, 1..64 (default 8) */
  /* filled in by gs_scene_get_launch and gs_autotune, ignored on input: */
  int batch;        /* Gaussians the variant stages per batch */
  int min_blocks;   /* resident CTAs per SM its registers allow for */
  int occupancy;    /* resident CTAs per SM on this device */
} gs_launch;

/* Set (or read back, with the effective CTAs per SM and the variant's
 * figures) the configuration of `mode` for the call shape of cams[0..n_views)
 * (host array; only the sizes matter). Errors: INVALID_ARG (mode, sizes, a
 * field out of range), CUDA. */
gs_status gs_scene_set_launch(gs_scene* scene, int mode, int n_views, const gs_camera* cams, const gs_launch* cfg);
gs_status gs_scene_get_launch(gs_scene* scene, int mode, int n_views, const gs_camera* cams, gs_launch* cfg);

typedef struct {
  gs_launch best;     /* the configuration chosen (now set for the shape) */
  double ms_default;  /* median device time of one call under the defaults */
  double ms_best;     /* the same under the chosen configuration (<= ms_default) */
  int candidates;     /* configurations timed */
} gs_tune_result;

/* Autotuner: time one call of `mode` on the views (cams, poses: host arrays
 * of n_views) under candidate configurations -- every compositor variant
 * with its occupancy and the two next-smaller persistent grids, then the
 * projection-side grid at 2, 4, 16 and 32 CTAs per SM -- and keep the
 * fastest for the shape. Each candidate's time is the median of `reps`
 * (< 1: 5) asynchronous calls on `stream`, measured with CUDA events, after
 * one warm-up call. The views are rendered into buffers of the tuner's own;
 * GS_MODE_POSE_GRAD uses those renders as its targets. Synchronous; do not
 * call during stream capture. result (host) may be NULL. Errors: INVALID_ARG,
 * OOM, CUDA, CAPACITY. */
gs_status gs_autotune(gs_scene* scene, int mode, int n_views, const gs_camera* cams, const gs_pose* poses, int reps,
                      gs_tune_result* result, void* stream);

/* The configuration cache file: one text line per (device, mode, shape),
 * "device name/SM count|mode|shape|variant ctas_per_sm grid_mult". save
 * writes every configuration of the scene for its device and keeps the lines
 * of other devices and shapes; load applies the lines of this device (the
 * count in *loaded, may be NULL). Errors: INVALID_ARG (path unreadable or
 * unwritable, a malformed line). */
gs_status gs_tune_save(const gs_scene* scene, const char* path);
gs_status gs_tune_load(gs_scene* scene, const char* path, int* loaded);

/* Render-gradient visibility check with projection filtering (Sec. 3.2,
 * Algorithm 1) of every Gaussian of the scene from one pose.
 *
 * M^r[j] = the gradient of the summed rendered colours (sum over pixels and
 * channels of RGB, Sec. 3.1 rasterisation) with respect to Gaussian j's mean
 * is non-zero, i.e. j contributed to some pixel; M^i[j] = its projected centre
 * (U, V) = K (R X + t) / z lies in [0, W) x [0, H) (no depth test);
 * M = M^r and M^i. The gradient comes from one forward render, one reverse
 * pass over the same tile lists and a chain rule per Gaussian; it is fp32 and
 * its summation order varies between calls (the zero / non-zero test does
 * not, up to rounding of sums that cancel to within fp32 precision).
 *
 * Device outputs (n = the scene's Gaussian count):
 *   mask         required, n bytes: bit 0 = M, bit 1 = M^r, bit 2 = M^i
 *   uv           NULL or n x 2 floats (8-byte aligned): (U, V) of every Gaussian
 *   grad_mean    NULL or n x 3 floats: d sum(RGB) / d mean (0 for Gaussians
 *                that reach no tile)
 *   visible_ids  NULL or capacity n int32 (4-byte aligned): the Gaussians with
 *                M set, ascending -- the selection (U', V') = (U, V)[:, M]
 *   visible_uv   NULL or capacity n x 2 floats (8-byte aligned): their (U, V)
 * n_visible: host pointer or NULL, receives the number of Gaussians with M.
 * A streamed scene (partitions uploaded on demand) is made fully resident
 * first: the in-image test covers every Gaussian. Synchronous (waits for
 * `stream`). Errors: INVALID_ARG (NULL cam, pose or mask, misaligned array,
 * camera out of range, non-finite pose), OOM, CAPACITY, CUDA. */
gs_status gs_visibility(gs_scene* scene, const gs_camera* cam, const gs_pose* pose, uint8_t* mask, float* uv,
                        float* grad_mean, int32_t* visible_ids, float* visible_uv, int64_t* n_visible,
                        void* stream);

/* gs_render_noalloc -- the forward render of gs_render that allocates
 * nothing (the paper has no counterpart).
 *
 * Why: some callers cannot ask the CUDA allocator for memory when they render
 * -- a service that sized its device memory once at start-up and may not grow
 * it per request, a plug-in whose host application owns every device
 * allocation, or code that runs while another thread captures a CUDA graph in
 * global mode, where cudaMalloc is not permitted. gs_render needs a scene
 * (created with cudaMalloc) and grows its workspace on demand; this entry
 * point needs neither.
 *
 * What: renders one view exactly like gs_render (same kernels, same results),
 * reading the Gaussians straight from the caller's device arrays in desc
 * (desc->device_resident must be 1; partitions are ignored) and writing the
 * caller's device outputs. Every intermediate buffer (packed scene, projected
 * records, tile counts, pair lists, counters) lives in one fixed array of
 * GS_NOALLOC_SCRATCH_BYTES in device memory that the library reserves on every
 * GPU it is loaded on, for the lifetime of the process.
 *
 * Limits: at most GS_NOALLOC_MAX_GAUSSIANS Gaussians and GS_NOALLOC_MAX_TILES
 * 16x16 tiles (GS_ERR_INVALID_ARG, checked before any work), and at most
 * GS_NOALLOC_MAX_PAIRS (tile, Gaussian) pairs (GS_ERR_CAPACITY, detected on
 * the device; the outputs are then incomplete).
 *
 * Calls no cudaMalloc, cudaFree or allocating library routine. Synchronous:
 * waits for the stream to read the device counters. The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) for that device;
 * make that first call before any stream capture. All calls share the one
 * array: calls whose work overlaps on the GPU (different streams or host
 * threads at the same time) race and corrupt each other's results; serialize
 * them. Each call clears the parts that must start at zero. */
#define GS_NOALLOC_MAX_GAUSSIANS 32768
#define GS_NOALLOC_MAX_TILES 16384
#define GS_NOALLOC_MAX_PAIRS 524288
#define GS_NOALLOC_SCRATCH_BYTES (24u << 20)
gs_status gs_render_noalloc(const gs_scene_desc* desc, const gs_camera* cam, const gs_pose* pose,
                            const gs_outputs* out, void* stream);

/* Thread-local message describing the last error of this thread ("" if none). */
const char* gs_last_error(void);

/* Library version string. */
const char* gs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GSR_H */
