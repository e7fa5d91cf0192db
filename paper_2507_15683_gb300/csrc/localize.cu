// Dense render-and-match rounds with Algorithm 2's pose consistency check,
// declared in include/gsr_localize.h. A host driver over the library's own
// entry points: each round renders the feature map, depth and alpha at the
// current pose (gs_render), matches the query features against them
// (gs_pmm_match, Eq. 11) and solves Eq. 10 on the fine matches
// (gs_pnp_solve); the rounds' poses are then compared with Psi.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "gsr_localize.h"

namespace gsr {
void set_last_error(const std::string& msg);
}

namespace {

gs_status loc_fail(gs_status s, const std::string& msg) {
  gsr::set_last_error(msg);
  return s;
}

void pose_of(const double* T, gs_pose* p) { std::memcpy(p->T_cw, T, 16 * sizeof(double)); }

}  // namespace

extern "C" {

gs_localize_opts gs_localize_defaults(void) {
  gs_localize_opts o;
  o.n_rounds = 3;
  o.pmm_tau = 0.1f;
  o.max_angle_deg = 20.0;
  o.n_hypotheses = 128;
  o.pnp = gs_pnp_defaults();
  return o;
}

gs_status gs_pose_difference(const gs_pose* T1, const gs_pose* T2, double* angle_deg, double* trans) {
  gsr::set_last_error("");
  if (!T1 || !T2 || !angle_deg || !trans) return loc_fail(GS_ERR_INVALID_ARG, "T1, T2, angle_deg and trans are required");
  const double* A = T1->T_cw;
  const double* B = T2->T_cw;
  double tr = 0.0;  // trace(R1 R2^T) = sum_ij R1_ij R2_ij
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) tr += A[4 * i + j] * B[4 * i + j];
  tr = std::min(3.0, std::max(tr, -1.0));
  *angle_deg = std::acos((tr - 1.0) / 2.0) * (180.0 / M_PI);
  const double d0 = A[3] - B[3], d1 = A[7] - B[7], d2 = A[11] - B[11];
  *trans = std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  return GS_OK;
}

gs_status gs_dense_localize(gs_scene* scene, gs_pmm* matcher, gs_pnp* solver, const gs_camera* cam,
                            const gs_pose* T_init, const float* feat_query, const uint32_t* words,
                            const gs_localize_opts* opts, gs_localize_result* out, void* stream) {
  gsr::set_last_error("");
  if (!scene || !matcher || !solver || !cam || !T_init || !feat_query || !opts || !out)
    return loc_fail(GS_ERR_INVALID_ARG, "scene, matcher, solver, cam, T_init, feat_query, opts and out are required");
  if (opts->n_rounds < 1 || opts->n_rounds > GS_LOCALIZE_MAX_ROUNDS || opts->n_hypotheses < 0 ||
      !(opts->max_angle_deg > 0.0) || !(opts->pmm_tau >= 0.025f))
    return loc_fail(GS_ERR_INVALID_ARG, "localisation options out of range");
  if (opts->n_hypotheses > 0 && !words) return loc_fail(GS_ERR_INVALID_ARG, "words are required");
  int feat_dim = 0;
  gs_status st = gs_scene_shape(scene, nullptr, nullptr, &feat_dim);
  if (st != GS_OK) return st;
  if (feat_dim != 32) return loc_fail(GS_ERR_INVALID_ARG, "the scene has no 32-channel features");
  int C = 0, H = 0, W = 0;
  if ((st = gs_pmm_shape(matcher, &C, &H, &W)) != GS_OK) return st;
  if (C != 32 || H != cam->height || W != cam->width)
    return loc_fail(GS_ERR_INVALID_ARG, "the matcher's shape differs from the camera's");
  const cudaStream_t cs = (cudaStream_t)stream;
  const size_t P = (size_t)H * W;
  float* buf = nullptr;  // rendered features (32 P), depth (P), alpha (P)
  cudaError_t e = cudaMallocAsync((void**)&buf, 34 * P * sizeof(float), cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return loc_fail(e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA,
                    std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  }
  gs_outputs o;
  std::memset(&o, 0, sizeof(o));
  o.feats = buf;
  o.depth = buf + 32 * P;
  o.alpha = buf + 33 * P;
  std::memset(out, 0, sizeof(*out));
  gs_pose T = *T_init;
  for (int r = 0; r < opts->n_rounds && st == GS_OK; ++r) {
    st = gs_render(scene, cam, &T, &o, stream);
    if (st != GS_OK) break;
    gs_pmm_result pm;
    st = gs_pmm_match(matcher, feat_query, o.feats, opts->pmm_tau, &pm, stream);
    if (st != GS_OK) break;
    gs_pnp_result pr;
    st = gs_pnp_solve(solver, cam, &T, o.depth, o.alpha, pm.fine, pm.n_fine,
                      words ? words + (size_t)r * opts->n_hypotheses * 3 : nullptr, opts->n_hypotheses, &opts->pnp,
                      &pr, stream);
    if (st != GS_OK) break;
    pose_of(pr.T_cw, &T);
    std::memcpy(out->round_T[r], pr.T_cw, 16 * sizeof(double));
    out->n_matches[r] = pm.n_fine;
    out->n_inliers[r] = pr.n_inliers;
    out->n_rounds = r + 1;
  }
  const cudaError_t fe = cudaFreeAsync(buf, cs);
  if (st != GS_OK) return st;
  if (fe != cudaSuccess) return loc_fail(GS_ERR_CUDA, std::string("cudaFreeAsync: ") + cudaGetErrorString(fe));
  out->reliable = 1;
  for (int i = 0; i + 1 < out->n_rounds; ++i) {
    gs_pose a, b;
    pose_of(out->round_T[i], &a);
    pose_of(out->round_T[i + 1], &b);
    gs_pose_difference(&a, &b, &out->angle_deg[i], &out->trans[i]);
    if (out->angle_deg[i] > opts->max_angle_deg) out->reliable = 0;
  }
  std::memcpy(out->T_cw, out->round_T[out->n_rounds - 1], 16 * sizeof(double));
  return GS_OK;
}

}  // extern "C"
