/* gsr_pnp.h -- dense 2D-3D PnP with RANSAC on rendered depth (Hi^2-GSLoc,
 * arXiv 2507.15683, Sec. 3.4, Eq. 10) on GB300 (sm_103a).
 *
 * Sec. 3.4 ends each coarse-to-fine round by lifting the rendered pixel of
 * every dense match to 3D with the depth rendered at the current pose, and
 * solving Eq. 10: the pose and inlier set minimising a robust reprojection
 * loss rho(||p_2D - pi(K [R|t] g_3D)||, tau), by PnP inside RANSAC.
 *
 * Readings (the paper is silent):
 *  - the query and rendered maps share the pinhole camera (they are matched
 *    pixel to pixel); pixel (x, y) has centre (x + 0.5, y + 0.5);
 *  - the depth of the surface seen at a rendered pixel is depth / alpha (the
 *    renderer's depth is the un-normalised sum of w z); a pixel with alpha <
 *    min_alpha gives no 3D point; the point is R_r^T (z K^-1 (x+.5, y+.5, 1)
 *    - t_r) in world coordinates;
 *  - rho is the truncated square min(e, tau)^2: RANSAC keeps the minimal-sample
 *    pose with the most inliers (e < tau with the point in front of the
 *    camera; ties to the lowest hypothesis, then the lowest solution), then
 *    Gauss-Newton steps on the squared errors of the inliers, re-selected
 *    before every step, refine it (left se(3) updates xi = (rho, phi));
 *  - minimal solver: P3P after Grunert (as reviewed by Haralick et al., 1994),
 *    solutions ordered by ascending ratio v = s3 / s1 of the distances along
 *    the first and third rays;
 *  - random numbers are inputs: hypothesis h takes three uint32 words w and
 *    the match indices floor(w K / 2^32) over the K matches with depth (in
 *    match order); a repeated index or a degenerate triangle gives no solution.
 *
 * Precision: lifting and P3P in fp64; inlier tests and the per-match
 * Gauss-Newton terms in fp32; the normal equations summed in fp64 in a fixed
 * order and solved in fp64. Device pointers are named *_dev or documented as
 * device memory. Thread safety: one solver per stream at a time.
 */
#ifndef GSR_PNP_H
#define GSR_PNP_H

#include "gsr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gs_pnp gs_pnp;

typedef struct {
  float tau_px;      /* inlier threshold tau in pixels, > 0 */
  float min_alpha;   /* rendered alpha below which a pixel has no depth, in (0, 1] */
  int refine_iters;  /* Gauss-Newton steps after RANSAC, 0 .. 100 */
} gs_pnp_opts;

/* Defaults: tau 2 px, min_alpha 0.5, 5 refinement steps. */
gs_pnp_opts gs_pnp_defaults(void);

/* A solver for up to max_matches matches and max_hypotheses RANSAC samples.
 * It owns its device workspace (about 80 bytes per match and 600 per
 * hypothesis). Errors: INVALID_ARG (max_matches outside [1, 2^30],
 * max_hypotheses outside [1, 65536]), OOM, CUDA. */
gs_status gs_pnp_create(int64_t max_matches, int max_hypotheses, gs_pnp** out);
void gs_pnp_destroy(gs_pnp* solver);

/* Result of the last gs_pnp_solve. Device arrays belong to the solver and
 * stay valid until its next call or destruction. */
typedef struct {
  double T_cw[16];            /* refined pose, row-major world-to-camera (the render pose when no hypothesis has a solution) */
  int64_t n_valid;            /* matches with depth (alpha >= min_alpha) */
  int64_t n_inliers;          /* inliers of the refined pose */
  int32_t best_hypothesis;    /* RANSAC winner, or -1 when no sample had a solution */
  int32_t best_solution;      /* its solution index (ascending v) */
  int64_t best_count;         /* its inlier count */
  int32_t refine_steps;       /* Gauss-Newton steps taken (stops early with < 3 inliers or a singular system) */
  const uint8_t* inlier;      /* device, n_matches: 1 = inlier of the refined pose */
  const int32_t* valid_index; /* device, n_valid: match index of each match with depth, ascending */
  const double* points;       /* device, n_valid x 3: world points of the matches with depth */
  const int32_t* hyp_counts;  /* device, n_hypotheses x 4: inlier count of each solution, -1 = no solution */
  const double* hyp_poses;    /* device, n_hypotheses x 4 x 12: (R row-major, t) of each solution */
} gs_pnp_result;

/* Lift, RANSAC and refine (Eq. 10) for one set of dense matches.
 *   cam        the shared camera (width x height pixels)
 *   T_render   the pose the depth and alpha were rendered at
 *   depth, alpha  device, height x width fp32: gs_outputs.depth and .alpha
 *   matches    device, n_matches x 3 int32 rows (any, query pixel, rendered
 *              pixel) with pixels y * width + x: the layout of
 *              gs_pmm_result.fine
 *   words      device, n_hypotheses x 3 uint32 random words (uniform)
 * Synchronous on `stream`; *out is valid on return. Errors: INVALID_ARG
 * (NULL pointers, counts above the solver's capacity, bad options, camera
 * out of range, non-finite pose; a match whose pixel index lies outside the
 * image is never read through and makes the call return INVALID_ARG after
 * it), CUDA. */
gs_status gs_pnp_solve(gs_pnp* solver, const gs_camera* cam, const gs_pose* T_render, const float* depth,
                       const float* alpha, const int32_t* matches, int64_t n_matches, const uint32_t* words,
                       int n_hypotheses, const gs_pnp_opts* opts, gs_pnp_result* out, void* stream);

/* Phase timing: while enabled, every gs_pnp_solve records CUDA events on its
 * stream around its GS_PNP_PHASES phases -- lifting (flags, scan, lift), P3P,
 * scoring, RANSAC argmax, Gauss-Newton refinement (all steps), final inliers --
 * and adds their durations. gs_pnp_phase_times returns the sums (ms, host
 * array of GS_PNP_PHASES) and the number of timed calls (may be NULL), then
 * resets them. Errors: INVALID_ARG, CUDA. */
#define GS_PNP_PHASES 6
gs_status gs_pnp_set_timing(gs_pnp* solver, int enable);
gs_status gs_pnp_phase_times(gs_pnp* solver, double* total_ms, int64_t* calls);

#ifdef __cplusplus
}
#endif

#endif /* GSR_PNP_H */
