// Pose refinement driver: repeated render + se(3) gradient (gs_render_pose_grad
// / gs_render_pose_grad_batch) with an Adam step on the pose tangent and the
// left update T <- Exp(-step^) T, re-linearised at every iteration. This is
// the analysis-by-synthesis counterpart of the render-and-refine loop of
// Sec. 3.4 (the paper runs its dense stage for n = 3 rounds).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "gsr_internal.h"

namespace gsr {
void set_last_error(const std::string& msg);
}

namespace {

// Exp of the twist (rho, phi) as a 4x4 row-major matrix (Rodrigues' formula
// for the rotation, and V = I + b K + c K^2 applied to rho).
void se3_exp(const double xi[6], double E[16]) {
  const double* rho = xi;
  const double* w = xi + 3;
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  const double t = std::sqrt(t2);
  double a, b, c;
  if (t < 1e-6) {  // series: sin t / t, (1 - cos t) / t^2, (t - sin t) / t^3
    a = 1.0 - t2 / 6.0;
    b = 0.5 - t2 / 24.0;
    c = 1.0 / 6.0 - t2 / 120.0;
  } else {
    a = std::sin(t) / t;
    b = (1.0 - std::cos(t)) / t2;
    c = (t - std::sin(t)) / (t2 * t);
  }
  const double K[3][3] = {{0.0, -w[2], w[1]}, {w[2], 0.0, -w[0]}, {-w[1], w[0], 0.0}};
  double K2[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) K2[i][j] = K[i][0] * K[0][j] + K[i][1] * K[1][j] + K[i][2] * K[2][j];
  std::memset(E, 0, 16 * sizeof(double));
  for (int i = 0; i < 3; ++i) {
    double tv = 0.0;
    for (int j = 0; j < 3; ++j) {
      const double id = (i == j) ? 1.0 : 0.0;
      E[4 * i + j] = id + a * K[i][j] + b * K2[i][j];
      tv += (id + b * K[i][j] + c * K2[i][j]) * rho[j];
    }
    E[4 * i + 3] = tv;
  }
  E[15] = 1.0;
}

void left_update(const double step[6], double T[16]) {
  double neg[6], E[16], out[16];
  for (int k = 0; k < 6; ++k) neg[k] = -step[k];
  se3_exp(neg, E);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += E[4 * i + k] * T[4 * k + j];
      out[4 * i + j] = s;
    }
  std::memcpy(T, out, sizeof(out));
}

struct Adam {
  double m[6] = {0, 0, 0, 0, 0, 0}, v[6] = {0, 0, 0, 0, 0, 0};
  int t = 0;
  void step(const double g[6], const gs_refine_opts& o, double out[6]) {
    ++t;
    const double c1 = 1.0 - std::pow(o.beta1, t), c2 = 1.0 - std::pow(o.beta2, t);
    for (int k = 0; k < 6; ++k) {
      m[k] = o.beta1 * m[k] + (1.0 - o.beta1) * g[k];
      v[k] = o.beta2 * v[k] + (1.0 - o.beta2) * g[k] * g[k];
      const double lr = k < 3 ? o.lr_trans : o.lr_rot;
      out[k] = lr * (m[k] / c1) / (std::sqrt(v[k] / c2) + o.eps);
    }
  }
};

gs_status check_opts(const gs_refine_opts* o) {
  if (!o || o->iterations < 0 || !(o->lr_rot >= 0) || !(o->lr_trans >= 0) || !(o->beta1 >= 0 && o->beta1 < 1) ||
      !(o->beta2 >= 0 && o->beta2 < 1) || !(o->eps > 0)) {
    gsr::set_last_error("refine options out of range");
    return GS_ERR_INVALID_ARG;
  }
  return GS_OK;
}

}  // namespace

extern "C" {

gs_refine_opts gs_refine_defaults(void) {
  gs_refine_opts o;
  o.iterations = 50;
  o.lr_rot = 1e-3;
  o.lr_trans = 0.5;
  o.beta1 = 0.9;
  o.beta2 = 0.999;
  o.eps = 1e-8;
  o.depth_weight = 0.1f;
  return o;
}

gs_status gs_refine_pose(gs_scene* scene, const gs_camera* cam, gs_pose* pose, const float* target_rgb,
                         const float* target_depth, const float* pixel_weight, const gs_refine_opts* opts,
                         double* loss_history, void* stream) {
  if (!pose) {
    gsr::set_last_error("pose is required");
    return GS_ERR_INVALID_ARG;
  }
  const gs_status so = check_opts(opts);
  if (so != GS_OK) return so;
  if (scene && cam) {
    bool used = false;
    const gs_status sd = gsr::refine_on_device(scene, 1, cam, pose, &target_rgb, &target_depth,
                                               pixel_weight ? &pixel_weight : nullptr, opts, loss_history,
                                               (cudaStream_t)stream, &used);
    if (used) return sd;
  }
  Adam adam;
  for (int it = 0; it < opts->iterations; ++it) {
    double loss = 0.0, g[6], step[6];
    const gs_status st = gs_render_pose_grad(scene, cam, pose, target_rgb, target_depth, pixel_weight,
                                             opts->depth_weight, nullptr, &loss, g, stream);
    if (st != GS_OK) return st;
    if (loss_history) loss_history[it] = loss;
    adam.step(g, *opts, step);
    left_update(step, pose->T_cw);
  }
  return GS_OK;
}

gs_status gs_refine_poses_batch(gs_scene* scene, int n_views, const gs_camera* cams, gs_pose* poses,
                                const float* const* target_rgb, const float* const* target_depth,
                                const float* const* pixel_weight, const gs_refine_opts* opts,
                                double* loss_history, void* stream) {
  if (n_views < 1 || !poses) {
    gsr::set_last_error("n_views >= 1 and poses are required");
    return GS_ERR_INVALID_ARG;
  }
  const gs_status so = check_opts(opts);
  if (so != GS_OK) return so;
  const cudaStream_t st = (cudaStream_t)stream;
  if (scene && cams && target_rgb && target_depth) {
    bool used = false;
    const gs_status sd = gsr::refine_on_device(scene, n_views, cams, poses, target_rgb, target_depth, pixel_weight,
                                               opts, loss_history, st, &used);
    if (used) return sd;
  }
  // first iteration synchronously (sizes the workspace), then graph replays
  std::vector<Adam> adam(n_views);
  std::vector<double> loss(n_views), grad(6 * (size_t)n_views), res(8 * (size_t)n_views);
  double* dres = nullptr;
  cudaError_t e = cudaMalloc(&dres, res.size() * sizeof(double));
  if (e != cudaSuccess) {
    gsr::set_last_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return GS_ERR_OOM;
  }
  gs_status status = GS_OK;
  for (int it = 0; it < opts->iterations && status == GS_OK; ++it) {
    if (it == 0) {
      status = gs_render_pose_grad_batch(scene, n_views, cams, poses, target_rgb, target_depth, pixel_weight,
                                         opts->depth_weight, nullptr, loss.data(), grad.data(), nullptr, 0, stream);
    } else {
      status = gs_render_pose_grad_batch(scene, n_views, cams, poses, target_rgb, target_depth, pixel_weight,
                                         opts->depth_weight, nullptr, nullptr, nullptr, dres, GS_BATCH_GRAPH, stream);
      if (status == GS_OK) status = gs_scene_status(scene, stream, nullptr, nullptr);
      if (status == GS_OK) {
        e = cudaMemcpyAsync(res.data(), dres, res.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
          gsr::set_last_error(std::string("result copy: ") + cudaGetErrorString(e));
          status = GS_ERR_CUDA;
        }
        for (int v = 0; v < n_views; ++v) {
          loss[v] = res[8 * (size_t)v];
          for (int k = 0; k < 6; ++k) grad[6 * (size_t)v + k] = res[8 * (size_t)v + 1 + k];
        }
      }
    }
    if (status != GS_OK) break;
    for (int v = 0; v < n_views; ++v) {
      if (loss_history) loss_history[(size_t)v * opts->iterations + it] = loss[v];
      double step[6];
      adam[v].step(&grad[6 * (size_t)v], *opts, step);
      left_update(step, poses[v].T_cw);
    }
  }
  cudaFree(dres);
  return status;
}

}  // extern "C"
