/*
 * gs_oracle.h -- plain, slow CPU oracle for the tile-based Gaussian-splatting
 * rasterizer and its pose gradient (Hi^2-GSLoc, arXiv 2507.15683, Sec. 3.1
 * and Sec. 3.4; Algorithm 1 for the projection).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. The product path (the
 * CUDA library under paper_2507_15683_gb300/) never links, calls or includes
 * anything here, and this file includes nothing from there.
 *
 * Precision contract
 *   - Discrete layer (camera-space depth, projected centre, 2D covariance,
 *     radius, tile rectangle, sort key) is evaluated in IEEE binary32 in one
 *     fixed operation order with no contraction, so that tile lists can be
 *     compared bit for bit.
 *   - Continuous layer (conic, colour, compositing, loss, gradient) is binary64.
 *     With geom64 = 0 the conic and the centre are taken from the binary32
 *     covariance/centre; with geom64 = 1 they are recomputed in binary64 from
 *     the inputs (needed for finite differences and the gradient).
 *   - The pose gradient is computed in forward (tangent) mode: every quantity
 *     carries its six derivatives with respect to the left se(3) perturbation
 *     xi = (rho, phi), T(xi) = Exp(xi^) T_cw.
 */
#ifndef GS_ORACLE_H
#define GS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int width, height;     /* pixels */
  float fx, fy, cx, cy;  /* pinhole intrinsics K (Eq. 10: pi([x,y,z]) = [x/z, y/z]) */
} orc_camera;

typedef struct {
  int64_t n;               /* number of Gaussians */
  int sh_degree;           /* 0..3 */
  int feat_dim;            /* 0 or more feature channels */
  const float* means;      /* n x 3, world */
  const float* scales;     /* n x 3, linear, > 0 */
  const float* quats;      /* n x 4, (w, x, y, z), normalised inside */
  const float* opacities;  /* n, in (0, 1) */
  const float* sh;         /* n x (deg+1)^2 x 3, coefficient-major */
  const uint16_t* feats_bf16; /* n x feat_dim bfloat16 bit patterns, or NULL */
  const float* feats_f32;  /* n x feat_dim binary32 features, or NULL; when given they are blended
                              instead of feats_bf16 (the unrounded vectors, to separate the error of
                              bf16 storage from that of the blending) */
} orc_scene;

/* Per-Gaussian discrete record written by orc_project_f32. */
enum { ORC_VISIBLE = 0, ORC_CULL_NEAR = 1, ORC_CULL_DET = 2, ORC_CULL_RADIUS = 3,
       ORC_CULL_EMPTY = 4 };
/* int32 fields per Gaussian (ORC_NI of them) */
enum { ORC_I_STATUS = 0, ORC_I_X0, ORC_I_X1, ORC_I_Y0, ORC_I_Y1, ORC_I_COUNT, ORC_NI };
/* float fields per Gaussian (ORC_NF of them) */
enum { ORC_F_Z = 0, ORC_F_U, ORC_F_V, ORC_F_A, ORC_F_B, ORC_F_C, ORC_F_DET, ORC_F_R, ORC_NF };

/* Near-tie flags per pixel (a decision whose margin is below the test's
 * resolution; either outcome is a valid rendering of the definition). */
enum { ORC_TIE_POWER = 1, ORC_TIE_ALPHA_FLOOR = 2, ORC_TIE_T_CUTOFF = 4,
       ORC_TIE_ALPHA_CAP = 8, ORC_TIE_RGB_CLAMP = 16, ORC_TIE_J_CLAMP = 32,
       ORC_TIE_RESIDUAL = 64 };

typedef struct {
  int geom64;               /* 0: conic/centre from the binary32 layer; 1: binary64 */
  int want_grad;            /* 1: compute loss gradient w.r.t. xi (requires geom64) */
  int n_threads;            /* worker threads over pixels (>= 1) */
  const int64_t* pixels;    /* subset of linear pixel indices y*W+x, or NULL = all */
  int64_t n_pixels;         /* length of pixels[] (ignored when pixels == NULL) */
  const float* target_rgb;  /* 3 x H x W planar, or NULL (no loss) */
  const float* target_depth;/* H x W, required with target_rgb */
  const float* pixel_weight;/* H x W, or NULL = all 1 */
  double depth_weight;      /* lambda_d of the loss */
  double tie_rel;           /* relative margin for near-tie flags (alpha floor, cap) */
  double tie_rel_T;         /* relative margin for the transmittance cutoff */
  int64_t mean_tangent_gid; /* >= 0: tangents 1..3 are d/d(mean x, y, z) of this Gaussian alone, and
                               loss / grad are sum_px,c C and its tangents (Algorithm 1's RGB.sum());
                               -1: pose tangents and the L1 loss of the targets */
} orc_opts;

typedef struct {
  /* per evaluated pixel (in the order of opts.pixels, or y*W+x for all) */
  double* rgb;        /* n_pix x 3, or NULL */
  double* depth;      /* n_pix, or NULL */
  double* alpha;      /* n_pix, or NULL */
  double* final_T;    /* n_pix, or NULL */
  int32_t* last_idx;  /* n_pix: 1 + list position of the last blended Gaussian (0 = none) */
  int32_t* n_eval;    /* n_pix: list entries examined, or NULL */
  int32_t* n_blend;   /* n_pix: Gaussians blended (accumulated before the cutoff), or NULL */
  uint8_t* flags;     /* n_pix: ORC_TIE_* bits, or NULL */
  double* feats;      /* n_pix x feat_dim, or NULL */
  double* loss;       /* 1, or NULL */
  double* grad;       /* 6 (rho, phi), or NULL */
  uint64_t* signature;/* 1: hash of every discrete decision taken, or NULL */
  int64_t* n_pairs;   /* 1: number of (tile, Gaussian) pairs, or NULL */
} orc_out;

/* Sec. 3.1 primitive: 3D covariance Sigma = R(q) diag(s)^2 R(q)^T in binary32. */
void orc_cov3d_f32(int64_t n, const float* scales, const float* quats, float* cov6);

/* Algorithm 1 projection plus EWA footprint, binary32 discrete layer.
 * T_cw: row-major 4x4 world-to-camera pose (double). Writes n x ORC_NI ints
 * and n x ORC_NF floats. */
void orc_project_f32(int64_t n, const float* means, const float* cov6,
                     const orc_camera* cam, const double* T_cw,
                     int32_t* rec_i, float* rec_f);

/* Tile binning: for every 16x16 tile (row-major) the Gaussians whose rectangle
 * covers it, ordered by (binary32 depth bits, Gaussian index). Writes
 * tile_start[n_tiles + 1], keys[pairs] = tile << 32 | depth bits, gids[pairs].
 * Returns the pair count, or -(pair count) if capacity is too small. */
int64_t orc_bin(int64_t n, const int32_t* rec_i, const float* rec_f,
                int tiles_x, int tiles_y, int64_t* tile_start, uint64_t* keys,
                uint32_t* gids, int64_t capacity);

/* Real spherical harmonics (Condon-Shortley phase), index l*l + l + m,
 * built from the Legendre polynomials; Y[(deg+1)^2], dY[(deg+1)^2 x 3] is the
 * gradient of the Cartesian polynomial form (may be NULL). */
void orc_sh_basis(int deg, const double* dir, double* Y, double* dY);

/* Full render: projection, binning, compositing (and loss / gradient). */
int orc_render(const orc_scene* sc, const orc_camera* cam, const double* T_cw,
               const orc_opts* opts, orc_out* out);

/* Brute force: every pixel walks ALL Gaussians in global (depth bits, index)
 * order, keeping those whose tile rectangle contains the pixel's tile. Same
 * outputs as orc_render without loss/gradient. */
int orc_render_brute(const orc_scene* sc, const orc_camera* cam, const double* T_cw,
                     const orc_opts* opts, orc_out* out);

/* Left se(3) update: T_out = Exp(xi^) T_in, xi = (rho, phi). */
void orc_se3_exp_left(const double* xi, const double* T_in, double* T_out);

/* Algorithm 2 pose difference: angle in degrees (trace clamped to [-1, 3])
 * and translation distance. */
void orc_pose_diff(const double* T1, const double* T2, double* angle_deg, double* dtrans);

#ifdef __cplusplus
}
#endif
#endif
