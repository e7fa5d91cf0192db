/* gsr_localize.h -- the dense render-and-match stage of Hi^2-GSLoc (arXiv
 * 2507.15683, Sec. 3.4) with its pose consistency verification (Algorithm 2)
 * on GB300 (sm_103a).
 *
 * One round renders the feature map, depth and alpha of the scene at the
 * current pose (Sec. 3.1 rasteriser), matches the query feature map against
 * the rendered one coarse to fine (PMM, Eq. 11) and solves Eq. 10 on the fine
 * matches lifted through the rendered depth (PnP + RANSAC); its pose starts
 * the next round. After n rounds, Algorithm 2 compares the poses of the rounds
 * with its difference function Psi and declares the result unreliable when an
 * angle exceeds the threshold (20 degrees).
 *
 * Readings (the paper is silent or ambiguous):
 *  - Psi(T1, T2): angle of R1 R2^T from its trace clamped to [-1, 3], in
 *    degrees, and the distance between the translation columns t1, t2 of the
 *    world-to-camera matrices, as written;
 *  - Algorithm 2's loop evaluates Psi for every consecutive pair of rounds,
 *    (T_i, T_i+1) for i = 1 .. n-1 (its listing names (T_1, T_2) in every
 *    iteration); the translation distance is reported, not tested;
 *  - all n rounds run, then the check (as the listing orders them); the first
 *    round starts from the caller's initial pose.
 *
 * Host pointers unless named *_dev / documented as device memory.
 */
#ifndef GSR_LOCALIZE_H
#define GSR_LOCALIZE_H

#include "gsr.h"
#include "gsr_pmm.h"
#include "gsr_pnp.h"

#ifdef __cplusplus
extern "C" {
#endif

#define GS_LOCALIZE_MAX_ROUNDS 8

typedef struct {
  int n_rounds;         /* n of Algorithm 2: 1 .. GS_LOCALIZE_MAX_ROUNDS (3) */
  float pmm_tau;        /* PMM temperature (0.1), >= 0.025 */
  double max_angle_deg; /* Algorithm 2's threshold tau (20 degrees), > 0 */
  int n_hypotheses;     /* RANSAC samples per round, >= 0 */
  gs_pnp_opts pnp;      /* PnP options of every round */
} gs_localize_opts;

/* Defaults: 3 rounds, PMM tau 0.1, 20 degrees, 128 hypotheses, gs_pnp_defaults. */
gs_localize_opts gs_localize_defaults(void);

typedef struct {
  double T_cw[16];                              /* pose of the last round (T_n) */
  int reliable;                                 /* 1: every consecutive angle <= max_angle_deg */
  int n_rounds;                                 /* rounds run */
  double round_T[GS_LOCALIZE_MAX_ROUNDS][16];   /* pose after each round */
  double angle_deg[GS_LOCALIZE_MAX_ROUNDS];     /* Psi angle between rounds i and i + 1 (n_rounds - 1 entries) */
  double trans[GS_LOCALIZE_MAX_ROUNDS];         /* Psi translation distance, same pairs */
  int64_t n_matches[GS_LOCALIZE_MAX_ROUNDS];    /* fine PMM matches of each round */
  int64_t n_inliers[GS_LOCALIZE_MAX_ROUNDS];    /* PnP inliers of each round */
} gs_localize_result;

/* Algorithm 2's Psi on two row-major world-to-camera poses (host arithmetic,
 * no GPU): angle in degrees and translation distance. Errors: INVALID_ARG. */
gs_status gs_pose_difference(const gs_pose* T1, const gs_pose* T2, double* angle_deg, double* trans);

/* n rounds of render (features, depth, alpha) -> PMM -> PnP from T_init, then
 * Algorithm 2's consistency check.
 *   scene       feat_dim 32; cam its camera for every round
 *   matcher     created for (32, cam height, cam width)
 *   solver      capacity for the fine matches of a round (at most H W) and
 *               opts->n_hypotheses samples
 *   feat_query  device, 32 x height x width fp32 planar: the query image's
 *               feature map
 *   words       device, n_rounds x n_hypotheses x 3 uint32 random words
 *               (round r uses rows r * n_hypotheses ...)
 * Synchronous on `stream`. Errors: INVALID_ARG (NULL pointers, a scene
 * without features, shapes that disagree, options out of range), the errors
 * of gs_render, gs_pmm_match and gs_pnp_solve, OOM, CUDA. */
gs_status gs_dense_localize(gs_scene* scene, gs_pmm* matcher, gs_pnp* solver, const gs_camera* cam,
                            const gs_pose* T_init, const float* feat_query, const uint32_t* words,
                            const gs_localize_opts* opts, gs_localize_result* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GSR_LOCALIZE_H */
