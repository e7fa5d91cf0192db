/*
 * gs_oracle.c -- plain, slow CPU oracle of the Gaussian-splatting rasterizer
 * and its pose gradient. TEST INFRASTRUCTURE ONLY (see gs_oracle.h): only the
 * tests, the smoke check and the benchmark's CPU-baseline leg use it; it shares
 * no code, header, table or constant with the CUDA library.
 *
 * What is computed, and where it comes from:
 *  - Sec. 3.1 of the paper: Gaussians Theta_i = {mean, rotation q, scale s,
 *    opacity, colour c, feature f}; colour is alpha-blended by a tile-based
 *    rasterizer and features go through the identical blending.
 *  - Algorithm 1: p_cam = (T [X, 1])[:3], depth d = p_cam.z, perspective
 *    division, then K; Eq. 10 gives pi([x, y, z]) = [x/z, y/z].
 *  - Everything the paper leaves open (EWA footprint, 0.3 px dilation, 1.3
 *    field-of-view guard, 0.1 eigenvalue floor, 3-sigma radius, 16 x 16 tiles,
 *    alpha floor 1/255, alpha cap 0.99, transmittance cutoff 1e-4, near plane
 *    0.2, stop-before-blend, background 0, un-normalised depth, L1 loss with
 *    0.1 depth weight, left perturbation xi = (rho, phi)) follows the readings
 *    written down for this project; each is marked [R] where it is used.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no -ffast-math).
 * The binary32 layer relies on IEEE single precision with no contraction.
 */
#include "gs_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TILE 16
#define ORC_CHUNK 4096          /* pixels per work chunk (fixed: sums do not depend on threads) */
#define ORC_ND 7                /* value + 6 tangents */
static const double kAlphaFloor = 1.0 / 255.0;  /* [R] */
static const double kAlphaCap = 0.99;           /* [R] */
static const double kTCutoff = 1e-4;            /* [R] */
static const double kResidualTie = 1e-5;        /* |I - I*| below this: sign undecided */
static const double kPi = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* binary32 discrete layer                                                   */
/* ------------------------------------------------------------------------ */

static uint32_t f32_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}

void orc_cov3d_f32(int64_t n, const float* scales, const float* quats, float* cov6) {
  for (int64_t i = 0; i < n; ++i) {
    const float qw = quats[4 * i + 0], qx = quats[4 * i + 1];
    const float qy = quats[4 * i + 2], qz = quats[4 * i + 3];
    /* |q|^2 summed left to right, then divide by |q| */
    const float n2 = qw * qw + qx * qx + qy * qy + qz * qz;
    float w = 1.0f, x = 0.0f, y = 0.0f, z = 0.0f;
    if (n2 > 0.0f) {
      const float nr = sqrtf(n2);
      w = qw / nr;
      x = qx / nr;
      y = qy / nr;
      z = qz / nr;
    }
    const float xx = x * x, yy = y * y, zz = z * z;
    const float xy = x * y, xz = x * z, yz = y * z;
    const float wx = w * x, wy = w * y, wz = w * z;
    float r[3][3];
    r[0][0] = 1.0f - 2.0f * (yy + zz);
    r[0][1] = 2.0f * (xy - wz);
    r[0][2] = 2.0f * (xz + wy);
    r[1][0] = 2.0f * (xy + wz);
    r[1][1] = 1.0f - 2.0f * (xx + zz);
    r[1][2] = 2.0f * (yz - wx);
    r[2][0] = 2.0f * (xz - wy);
    r[2][1] = 2.0f * (yz + wx);
    r[2][2] = 1.0f - 2.0f * (xx + yy);
    const float s[3] = {scales[3 * i + 0], scales[3 * i + 1], scales[3 * i + 2]};
    float m[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) m[a][b] = r[a][b] * s[b];
    /* Sigma_ab = (m_a0 m_b0 + m_a1 m_b1) + m_a2 m_b2 */
    float sg[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) sg[a][b] = m[a][0] * m[b][0] + m[a][1] * m[b][1] + m[a][2] * m[b][2];
    cov6[6 * i + 0] = sg[0][0];
    cov6[6 * i + 1] = sg[0][1];
    cov6[6 * i + 2] = sg[0][2];
    cov6[6 * i + 3] = sg[1][1];
    cov6[6 * i + 4] = sg[1][2];
    cov6[6 * i + 5] = sg[2][2];
  }
}

void orc_project_f32(int64_t n, const float* means, const float* cov6, const orc_camera* cam,
                     const double* T_cw, int32_t* rec_i, float* rec_f) {
  float R[3][3], t[3];
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) R[a][b] = (float)T_cw[4 * a + b];
    t[a] = (float)T_cw[4 * a + 3];
  }
  const float fx = cam->fx, fy = cam->fy, cx = cam->cx, cy = cam->cy;
  const int tiles_x = (cam->width + ORC_TILE - 1) / ORC_TILE;
  const int tiles_y = (cam->height + ORC_TILE - 1) / ORC_TILE;
  /* [R] 1.3 x half field of view guard on the Jacobian */
  const float limx = 1.3f * ((0.5f * (float)cam->width) / fx);
  const float limy = 1.3f * ((0.5f * (float)cam->height) / fy);
  const float txmax = (float)(tiles_x - 1), tymax = (float)(tiles_y - 1);

  for (int64_t i = 0; i < n; ++i) {
    int32_t* oi = rec_i + ORC_NI * i;
    float* of = rec_f + ORC_NF * i;
    memset(oi, 0, sizeof(int32_t) * ORC_NI);
    memset(of, 0, sizeof(float) * ORC_NF);
    const float mx = means[3 * i + 0], my = means[3 * i + 1], mz = means[3 * i + 2];
    /* Algorithm 1: homogeneous transform, depth = third camera coordinate */
    const float px = R[0][0] * mx + R[0][1] * my + R[0][2] * mz + t[0];
    const float py = R[1][0] * mx + R[1][1] * my + R[1][2] * mz + t[1];
    const float pz = R[2][0] * mx + R[2][1] * my + R[2][2] * mz + t[2];
    of[ORC_F_Z] = pz;
    if (!(pz >= 0.2f)) { /* [R] near plane 0.2 */
      oi[ORC_I_STATUS] = ORC_CULL_NEAR;
      continue;
    }
    /* perspective division then K (Algorithm 1, Eq. 10) */
    const float ix = px / pz, iy = py / pz;
    const float u = fx * ix + cx;
    const float v = fy * iy + cy;
    of[ORC_F_U] = u;
    of[ORC_F_V] = v;
    /* EWA: Jacobian of the perspective map at the (guard-clamped) centre */
    const float xh = fminf(limx, fmaxf(-limx, ix)) * pz;
    const float yh = fminf(limy, fmaxf(-limy, iy)) * pz;
    const float pz2 = pz * pz;
    const float j00 = fx / pz, j02 = -((fx * xh) / pz2);
    const float j11 = fy / pz, j12 = -((fy * yh) / pz2);
    float T[2][3];
    for (int k = 0; k < 3; ++k) {
      T[0][k] = j00 * R[0][k] + j02 * R[2][k];
      T[1][k] = j11 * R[1][k] + j12 * R[2][k];
    }
    const float* c = cov6 + 6 * i;
    const float S[3][3] = {{c[0], c[1], c[2]}, {c[1], c[3], c[4]}, {c[2], c[4], c[5]}};
    float U[2][3];
    for (int a = 0; a < 2; ++a)
      for (int k = 0; k < 3; ++k) U[a][k] = T[a][0] * S[0][k] + T[a][1] * S[1][k] + T[a][2] * S[2][k];
    /* [R] 0.3 px low-pass dilation */
    const float ca = U[0][0] * T[0][0] + U[0][1] * T[0][1] + U[0][2] * T[0][2] + 0.3f;
    const float cb = U[0][0] * T[1][0] + U[0][1] * T[1][1] + U[0][2] * T[1][2];
    const float cc = U[1][0] * T[1][0] + U[1][1] * T[1][1] + U[1][2] * T[1][2] + 0.3f;
    of[ORC_F_A] = ca;
    of[ORC_F_B] = cb;
    of[ORC_F_C] = cc;
    const float det = ca * cc - cb * cb;
    of[ORC_F_DET] = det;
    if (!(det > 0.0f)) {
      oi[ORC_I_STATUS] = ORC_CULL_DET;
      continue;
    }
    /* [R] largest eigenvalue with a 0.1 floor under the discriminant; 3 sigma */
    const float mid = 0.5f * (ca + cc);
    const float disc = mid * mid - det;
    const float lam = mid + sqrtf(fmaxf(0.1f, disc));
    const float r = ceilf(3.0f * sqrtf(lam));
    of[ORC_F_R] = r;
    if (!(r > 0.0f)) {
      oi[ORC_I_STATUS] = ORC_CULL_RADIUS;
      continue;
    }
    /* tile rectangle, inclusive bounds, clamped to the image's tiles */
    float x0 = floorf((u - r) / 16.0f), x1 = floorf((u + r) / 16.0f);
    float y0 = floorf((v - r) / 16.0f), y1 = floorf((v + r) / 16.0f);
    x0 = fmaxf(x0, 0.0f);
    y0 = fmaxf(y0, 0.0f);
    x1 = fminf(x1, txmax);
    y1 = fminf(y1, tymax);
    if (x0 > x1 || y0 > y1) {
      oi[ORC_I_STATUS] = ORC_CULL_EMPTY;
      continue;
    }
    oi[ORC_I_STATUS] = ORC_VISIBLE;
    oi[ORC_I_X0] = (int32_t)x0;
    oi[ORC_I_X1] = (int32_t)x1;
    oi[ORC_I_Y0] = (int32_t)y0;
    oi[ORC_I_Y1] = (int32_t)y1;
    oi[ORC_I_COUNT] = (oi[ORC_I_X1] - oi[ORC_I_X0] + 1) * (oi[ORC_I_Y1] - oi[ORC_I_Y0] + 1);
  }
}

static int cmp_u64(const void* a, const void* b) {
  const uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return (x > y) - (x < y);
}

int64_t orc_bin(int64_t n, const int32_t* rec_i, const float* rec_f, int tiles_x, int tiles_y,
                int64_t* tile_start, uint64_t* keys, uint32_t* gids, int64_t capacity) {
  const int64_t n_tiles = (int64_t)tiles_x * tiles_y;
  int64_t* cnt = (int64_t*)calloc((size_t)n_tiles + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) {
    const int32_t* oi = rec_i + ORC_NI * i;
    if (oi[ORC_I_STATUS] != ORC_VISIBLE) continue;
    for (int ty = oi[ORC_I_Y0]; ty <= oi[ORC_I_Y1]; ++ty)
      for (int tx = oi[ORC_I_X0]; tx <= oi[ORC_I_X1]; ++tx) cnt[(int64_t)ty * tiles_x + tx] += 1;
  }
  tile_start[0] = 0;
  for (int64_t t = 0; t < n_tiles; ++t) tile_start[t + 1] = tile_start[t] + cnt[t];
  const int64_t total = tile_start[n_tiles];
  if (total > capacity) {
    free(cnt);
    return -total;
  }
  for (int64_t t = 0; t < n_tiles; ++t) cnt[t] = tile_start[t];
  for (int64_t i = 0; i < n; ++i) {
    const int32_t* oi = rec_i + ORC_NI * i;
    if (oi[ORC_I_STATUS] != ORC_VISIBLE) continue;
    for (int ty = oi[ORC_I_Y0]; ty <= oi[ORC_I_Y1]; ++ty)
      for (int tx = oi[ORC_I_X0]; tx <= oi[ORC_I_X1]; ++tx) gids[cnt[(int64_t)ty * tiles_x + tx]++] = (uint32_t)i;
  }
  /* within a tile: ascending (depth bits, index); depth > 0 so bit order = value order */
  uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(total > 0 ? total : 1));
  for (int64_t t = 0; t < n_tiles; ++t) {
    const int64_t s = tile_start[t], e = tile_start[t + 1];
    for (int64_t j = s; j < e; ++j) tmp[j] = ((uint64_t)f32_bits(rec_f[ORC_NF * gids[j] + ORC_F_Z]) << 32) | gids[j];
    qsort(tmp + s, (size_t)(e - s), sizeof(uint64_t), cmp_u64);
    for (int64_t j = s; j < e; ++j) {
      gids[j] = (uint32_t)(tmp[j] & 0xffffffffu);
      keys[j] = ((uint64_t)t << 32) | (tmp[j] >> 32);
    }
  }
  free(tmp);
  free(cnt);
  return total;
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics from their definition                            */
/* Y_l^m = N_lm Q_lm(z) A_m(x, y):                                           */
/*   Q_lm = (-1)^|m| d^|m| P_l / dz^|m|   (Condon-Shortley phase)            */
/*   A_m  = Re (x + i y)^m (m > 0), Im (x + i y)^|m| (m < 0), 1 (m = 0)       */
/*   N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) * (sqrt 2 if m != 0)        */
/* ------------------------------------------------------------------------ */

static double factorial(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= i;
  return f;
}

void orc_sh_basis(int deg, const double* dir, double* Y, double* dY) {
  double P[4][4];  /* Legendre coefficients P_l(z) = sum_k P[l][k] z^k */
  memset(P, 0, sizeof(P));
  P[0][0] = 1.0;
  P[1][1] = 1.0;
  for (int l = 1; l < 3; ++l) /* (l+1) P_{l+1} = (2l+1) z P_l - l P_{l-1} */
    for (int k = 0; k < 4; ++k) {
      const double zp = (k > 0) ? P[l][k - 1] : 0.0;
      P[l + 1][k] = ((2.0 * l + 1.0) * zp - l * P[l - 1][k]) / (l + 1.0);
    }
  const double x = dir[0], y = dir[1], z = dir[2];
  for (int l = 0; l <= deg; ++l) {
    for (int m = -l; m <= l; ++m) {
      const int am = m < 0 ? -m : m;
      /* m-th derivative of P_l, and its derivative */
      double q = 0.0, dq = 0.0;
      for (int k = 0; k + am <= 3; ++k) {
        const double d = P[l][k + am] * factorial(k + am) / factorial(k);
        q += d * pow(z, k);
        if (k > 0) dq += d * k * pow(z, k - 1);
      }
      if (am & 1) {
        q = -q;
        dq = -dq;
      }
      /* (x + i y)^am and (x + i y)^(am - 1) */
      double re = 1.0, im = 0.0, re1 = 0.0, im1 = 0.0;
      for (int k = 0; k < am; ++k) {
        re1 = re;
        im1 = im;
        const double nr = re * x - im * y, ni = re * y + im * x;
        re = nr;
        im = ni;
      }
      double A, Ax, Ay;
      if (m > 0) {
        A = re;
        Ax = am * re1;
        Ay = -am * im1;
      } else if (m < 0) {
        A = im;
        Ax = am * im1;
        Ay = am * re1;
      } else {
        A = 1.0;
        Ax = 0.0;
        Ay = 0.0;
      }
      double N = sqrt((2.0 * l + 1.0) / (4.0 * kPi) * factorial(l - am) / factorial(l + am));
      if (m != 0) N *= sqrt(2.0);
      const int idx = l * l + l + m;
      Y[idx] = N * q * A;
      if (dY) {
        dY[3 * idx + 0] = N * q * Ax;
        dY[3 * idx + 1] = N * q * Ay;
        dY[3 * idx + 2] = N * dq * A;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Continuous layer: per-Gaussian quantities with 6 pose tangents            */
/* ------------------------------------------------------------------------ */

enum { Q_U = 0, Q_V, Q_A, Q_B, Q_C, Q_Z, Q_R, Q_G, Q_BL, NQ };

typedef struct {
  double q[NQ][ORC_ND]; /* value + d/dxi_k */
  double opacity;
  uint32_t clamp_bits;  /* bit0/1: x guard low/high, bit2/3: y guard, bit4..6: rgb clamped */
  uint8_t tie;          /* ORC_TIE_J_CLAMP / ORC_TIE_RGB_CLAMP */
} gprep;

static void mat3_mul(const double a[3][3], const double b[3][3], double c[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += a[i][k] * b[k][j];
      c[i][j] = s;
    }
}

static void skew(const double w[3], double S[3][3]) {
  S[0][0] = 0.0;   S[0][1] = -w[2]; S[0][2] = w[1];
  S[1][0] = w[2];  S[1][1] = 0.0;   S[1][2] = -w[0];
  S[2][0] = -w[1]; S[2][1] = w[0];  S[2][2] = 0.0;
}

typedef struct {
  const orc_scene* sc;
  const orc_camera* cam;
  const double* T_cw;
  const int32_t* rec_i;
  const float* rec_f;
  int geom64, nd;
  double tie_rel;
  int64_t mean_gid;  /* >= 0: tangents along this Gaussian's mean only */
} prep_ctx;

/* colour from SH at dir = normalize(mean - camera centre) [R: +0.5, clamp >= 0] */
static void prep_colour(const prep_ctx* cx, int64_t g, const double mu[3], const double cw[3],
                        const double dd[6][3], gprep* o) {
  const orc_scene* sc = cx->sc;
  const int K = (sc->sh_degree + 1) * (sc->sh_degree + 1);
  double d[3] = {mu[0] - cw[0], mu[1] - cw[1], mu[2] - cw[2]};
  const double nrm = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  double dir[3] = {d[0] / nrm, d[1] / nrm, d[2] / nrm};
  double Y[16], dY[48];
  orc_sh_basis(sc->sh_degree, dir, Y, dY);
  const float* sh = sc->sh + (int64_t)g * K * 3;
  for (int ch = 0; ch < 3; ++ch) {
    double val = 0.5;
    for (int k = 0; k < K; ++k) val += Y[k] * (double)sh[3 * k + ch];
    double* q = o->q[Q_R + ch];
    for (int j = 0; j < cx->nd; ++j) q[j] = 0.0;
    if (fabs(val) <= 1e-9 + cx->tie_rel * 1e-3) o->tie |= ORC_TIE_RGB_CLAMP;
    if (val < 0.0) {
      o->clamp_bits |= 1u << (4 + ch);
      continue;
    }
    q[0] = val;
    for (int k = 1; k < cx->nd; ++k) {
      /* d dir = (dd - dir (dir . dd)) / |d| */
      const double* e = dd[k - 1];
      const double pr = dir[0] * e[0] + dir[1] * e[1] + dir[2] * e[2];
      const double ddir[3] = {(e[0] - dir[0] * pr) / nrm, (e[1] - dir[1] * pr) / nrm,
                              (e[2] - dir[2] * pr) / nrm};
      double s = 0.0;
      for (int b = 0; b < K; ++b)
        s += (dY[3 * b] * ddir[0] + dY[3 * b + 1] * ddir[1] + dY[3 * b + 2] * ddir[2]) * (double)sh[3 * b + ch];
      q[k] = s;
    }
  }
}

static void prep_gauss(const prep_ctx* cx, int64_t g, gprep* o) {
  const orc_scene* sc = cx->sc;
  const orc_camera* cam = cx->cam;
  const int nd = cx->nd;
  memset(o, 0, sizeof(*o));
  o->opacity = (double)sc->opacities[g];
  double R[3][3], t[3];
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) R[a][b] = cx->T_cw[4 * a + b];
    t[a] = cx->T_cw[4 * a + 3];
  }
  const double mu[3] = {sc->means[3 * g], sc->means[3 * g + 1], sc->means[3 * g + 2]};
  /* camera centre c_w = -R^T t; under the left perturbation d c_w = -R^T rho */
  double cw[3];
  for (int a = 0; a < 3; ++a) cw[a] = -(R[0][a] * t[0] + R[1][a] * t[1] + R[2][a] * t[2]);
  double dd[6][3]; /* tangent of (mu - c_w) = R^T rho */
  for (int k = 0; k < 6; ++k)
    for (int a = 0; a < 3; ++a) dd[k][a] = (k < 3) ? R[k][a] : 0.0;
  /* mean tangents (Algorithm 1): d (mu - c_w) / d mu_k = e_k for the chosen Gaussian, 0 for the rest */
  const int mean_mode = cx->mean_gid >= 0;
  const int own = mean_mode && cx->mean_gid == g;
  if (mean_mode)
    for (int k = 0; k < 6; ++k)
      for (int a = 0; a < 3; ++a) dd[k][a] = (own && k < 3 && a == k) ? 1.0 : 0.0;

  if (!cx->geom64) {
    const float* of = cx->rec_f + ORC_NF * g;
    const double a = of[ORC_F_A], b = of[ORC_F_B], c = of[ORC_F_C];
    const double det = a * c - b * b;
    o->q[Q_U][0] = of[ORC_F_U];
    o->q[Q_V][0] = of[ORC_F_V];
    o->q[Q_A][0] = c / det;
    o->q[Q_B][0] = -b / det;
    o->q[Q_C][0] = a / det;
    o->q[Q_Z][0] = of[ORC_F_Z];
    prep_colour(cx, g, mu, cw, dd, o);
    return;
  }

  /* camera-space mean and its tangents: d p = rho + phi x p */
  double p[3];
  for (int a = 0; a < 3; ++a) p[a] = R[a][0] * mu[0] + R[a][1] * mu[1] + R[a][2] * mu[2] + t[a];
  double dp[6][3];
  for (int k = 0; k < 6; ++k) {
    if (mean_mode) {  /* d p / d mu_k = R e_k for the chosen Gaussian */
      for (int a = 0; a < 3; ++a) dp[k][a] = (own && k < 3) ? R[a][k] : 0.0;
    } else if (k < 3) {
      for (int a = 0; a < 3; ++a) dp[k][a] = (a == k) ? 1.0 : 0.0;
    } else {
      double w[3] = {0, 0, 0};
      w[k - 3] = 1.0;
      dp[k][0] = w[1] * p[2] - w[2] * p[1];
      dp[k][1] = w[2] * p[0] - w[0] * p[2];
      dp[k][2] = w[0] * p[1] - w[1] * p[0];
    }
  }
  /* world covariance from (s, q) in binary64, then camera covariance R Sigma R^T */
  double qw = sc->quats[4 * g], qx = sc->quats[4 * g + 1], qy = sc->quats[4 * g + 2], qz = sc->quats[4 * g + 3];
  const double qn = sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
  if (qn > 0.0) {
    qw /= qn; qx /= qn; qy /= qn; qz /= qn;
  } else {
    qw = 1.0; qx = qy = qz = 0.0;
  }
  const double Rq[3][3] = {
      {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
      {2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)},
      {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)}};
  double S2[3][3] = {{0}};
  for (int a = 0; a < 3; ++a) S2[a][a] = (double)sc->scales[3 * g + a] * (double)sc->scales[3 * g + a];
  double RqT[3][3], tmp[3][3], Sw[3][3], RT[3][3], Sc[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      RqT[a][b] = Rq[b][a];
      RT[a][b] = R[b][a];
    }
  mat3_mul(Rq, S2, tmp);
  mat3_mul(tmp, RqT, Sw);
  mat3_mul(R, Sw, tmp);
  mat3_mul(tmp, RT, Sc);
  double dSc[6][3][3];
  for (int k = 0; k < 6; ++k) {
    if (k < 3 || mean_mode) {  /* the covariance does not depend on the mean */
      memset(dSc[k], 0, sizeof(dSc[k]));
      continue;
    }
    double w[3] = {0, 0, 0}, W[3][3], A1[3][3], A2[3][3];
    w[k - 3] = 1.0;
    skew(w, W);
    mat3_mul(W, Sc, A1);
    mat3_mul(Sc, W, A2);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) dSc[k][a][b] = A1[a][b] - A2[a][b];
  }
  const double fx = cam->fx, fy = cam->fy;
  const double pz = p[2];
  /* Algorithm 1 projection */
  o->q[Q_U][0] = fx * p[0] / pz + cam->cx;
  o->q[Q_V][0] = fy * p[1] / pz + cam->cy;
  o->q[Q_Z][0] = pz;
  for (int k = 1; k < nd; ++k) {
    const double* e = dp[k - 1];
    o->q[Q_U][k] = fx * (e[0] * pz - p[0] * e[2]) / (pz * pz);
    o->q[Q_V][k] = fy * (e[1] * pz - p[1] * e[2]) / (pz * pz);
    o->q[Q_Z][k] = e[2];
  }
  /* guard-clamped Jacobian (exact derivative of the clamped expression) */
  const double lim[2] = {1.3 * (0.5 * cam->width / fx), 1.3 * (0.5 * cam->height / fy)};
  double h[2][ORC_ND];
  for (int a = 0; a < 2; ++a) {
    const double ratio = p[a] / pz;
    if (fabs(fabs(ratio) - lim[a]) <= cx->tie_rel * lim[a]) o->tie |= ORC_TIE_J_CLAMP;
    if (ratio < -lim[a] || ratio > lim[a]) {
      const double L = ratio < 0 ? -lim[a] : lim[a];
      o->clamp_bits |= 1u << (2 * a + (ratio < 0 ? 0 : 1));
      h[a][0] = L * pz;
      for (int k = 1; k < nd; ++k) h[a][k] = L * dp[k - 1][2];
    } else {
      h[a][0] = p[a];
      for (int k = 1; k < nd; ++k) h[a][k] = dp[k - 1][a];
    }
  }
  double J[ORC_ND][2][3];
  memset(J, 0, sizeof(J));
  J[0][0][0] = fx / pz;
  J[0][0][2] = -fx * h[0][0] / (pz * pz);
  J[0][1][1] = fy / pz;
  J[0][1][2] = -fy * h[1][0] / (pz * pz);
  for (int k = 1; k < nd; ++k) {
    const double dz = dp[k - 1][2];
    J[k][0][0] = -fx * dz / (pz * pz);
    J[k][0][2] = -fx * (h[0][k] / (pz * pz) - 2.0 * h[0][0] * dz / (pz * pz * pz));
    J[k][1][1] = -fy * dz / (pz * pz);
    J[k][1][2] = -fy * (h[1][k] / (pz * pz) - 2.0 * h[1][0] * dz / (pz * pz * pz));
  }
  /* M = J Sc J^T + 0.3 I and its tangents (product rule over the three factors) */
  double M[ORC_ND][2][2];
  memset(M, 0, sizeof(M));
  for (int k = 0; k < nd; ++k) {
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        double s = 0.0;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            if (k == 0) {
              s += J[0][a][i] * Sc[i][j] * J[0][b][j];
            } else {
              s += J[k][a][i] * Sc[i][j] * J[0][b][j] + J[0][a][i] * dSc[k - 1][i][j] * J[0][b][j] +
                   J[0][a][i] * Sc[i][j] * J[k][b][j];
            }
          }
        M[k][a][b] = s;
      }
  }
  M[0][0][0] += 0.3;
  M[0][1][1] += 0.3;
  const double det = M[0][0][0] * M[0][1][1] - M[0][0][1] * M[0][0][1];
  o->q[Q_A][0] = M[0][1][1] / det;
  o->q[Q_B][0] = -M[0][0][1] / det;
  o->q[Q_C][0] = M[0][0][0] / det;
  for (int k = 1; k < nd; ++k) {
    const double dd_ = M[k][0][0] * M[0][1][1] + M[0][0][0] * M[k][1][1] - 2.0 * M[0][0][1] * M[k][0][1];
    o->q[Q_A][k] = (M[k][1][1] * det - M[0][1][1] * dd_) / (det * det);
    o->q[Q_B][k] = -(M[k][0][1] * det - M[0][0][1] * dd_) / (det * det);
    o->q[Q_C][k] = (M[k][0][0] * det - M[0][0][0] * dd_) / (det * det);
  }
  prep_colour(cx, g, mu, cw, dd, o);
}

/* ------------------------------------------------------------------------ */
/* Compositing of one pixel (binary64, with tangents when nd == 7)           */
/* ------------------------------------------------------------------------ */

typedef struct {
  double rgb[3][ORC_ND], depth[ORC_ND], T[ORC_ND];
  int32_t last_idx, n_eval, n_blend;
  uint8_t flags;
  uint64_t hash;
} pix_result;

static uint64_t mix64(uint64_t h, uint64_t v) {
  h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
  h *= 0xff51afd7ed558ccdull;
  return h ^ (h >> 29);
}

/* list[0..len): Gaussian indices in blending order; vis[gid] -> prep index */
static void composite_pixel(const gprep* prep, const int32_t* vis, const uint32_t* list, int64_t len,
                            double pxc, double pyc, int nd, double tie_rel, double tie_rel_T,
                            const orc_scene* sc, double* feat_out, pix_result* r) {
  memset(r, 0, sizeof(*r));
  r->T[0] = 1.0;
  r->hash = 1469598103934665603ull;
  const int fd = (feat_out && (sc->feats_bf16 || sc->feats_f32)) ? sc->feat_dim : 0;
  for (int c = 0; c < fd; ++c) feat_out[c] = 0.0;
  for (int64_t j = 0; j < len; ++j) {
    const uint32_t gid = list[j];
    const gprep* g = prep + vis[gid];
    r->n_eval += 1;
    const double* U = g->q[Q_U];
    const double* V = g->q[Q_V];
    const double* A = g->q[Q_A];
    const double* B = g->q[Q_B];
    const double* C = g->q[Q_C];
    const double dx = U[0] - pxc, dy = V[0] - pyc;
    const double power = -0.5 * (A[0] * dx * dx + C[0] * dy * dy) - B[0] * dx * dy;
    const double scale = 0.5 * (fabs(A[0]) * dx * dx + fabs(C[0]) * dy * dy) + fabs(B[0] * dx * dy);
    if (power > -1e-6 * scale) r->flags |= ORC_TIE_POWER;
    if (power > 0.0) {
      r->hash = mix64(r->hash, ((uint64_t)gid << 3) | 1);
      continue;
    }
    const double oe = g->opacity * exp(power);
    if (fabs(oe - kAlphaCap) <= tie_rel * kAlphaCap) r->flags |= ORC_TIE_ALPHA_CAP;
    if (fabs(oe - kAlphaFloor) <= tie_rel * kAlphaFloor) r->flags |= ORC_TIE_ALPHA_FLOOR;
    const int capped = oe >= kAlphaCap;
    const double alpha = capped ? kAlphaCap : oe;
    if (alpha < kAlphaFloor) {
      r->hash = mix64(r->hash, ((uint64_t)gid << 3) | 2);
      continue;
    }
    double dalpha[ORC_ND] = {0};
    if (!capped)
      for (int k = 1; k < nd; ++k) {
        const double dpow = -0.5 * (A[k] * dx * dx + 2.0 * A[0] * dx * U[k] + C[k] * dy * dy +
                                    2.0 * C[0] * dy * V[k]) -
                            B[k] * dx * dy - B[0] * (U[k] * dy + dx * V[k]);
        dalpha[k] = oe * dpow;
      }
    const double Tn = r->T[0] * (1.0 - alpha);
    if (fabs(Tn - kTCutoff) <= tie_rel_T * kTCutoff) r->flags |= ORC_TIE_T_CUTOFF;
    if (Tn < kTCutoff) { /* [R] stop before blending this Gaussian */
      r->hash = mix64(r->hash, ((uint64_t)gid << 3) | 3);
      break;
    }
    double w[ORC_ND], dT[ORC_ND];
    w[0] = alpha * r->T[0];
    for (int k = 1; k < nd; ++k) {
      w[k] = dalpha[k] * r->T[0] + alpha * r->T[k];
      dT[k] = r->T[k] * (1.0 - alpha) - r->T[0] * dalpha[k];
    }
    for (int ch = 0; ch < 3; ++ch) {
      const double* c = g->q[Q_R + ch];
      r->rgb[ch][0] += w[0] * c[0];
      for (int k = 1; k < nd; ++k) r->rgb[ch][k] += w[k] * c[0] + w[0] * c[k];
    }
    const double* z = g->q[Q_Z];
    r->depth[0] += w[0] * z[0];
    for (int k = 1; k < nd; ++k) r->depth[k] += w[k] * z[0] + w[0] * z[k];
    if (fd) {
      if (sc->feats_f32) {
        const float* f = sc->feats_f32 + (int64_t)gid * sc->feat_dim;
        for (int c = 0; c < fd; ++c) feat_out[c] += w[0] * (double)f[c];
      } else {
        const uint16_t* f = sc->feats_bf16 + (int64_t)gid * sc->feat_dim;
        for (int c = 0; c < fd; ++c) {
          uint32_t bits = (uint32_t)f[c] << 16;
          float fv;
          memcpy(&fv, &bits, 4);
          feat_out[c] += w[0] * (double)fv;
        }
      }
    }
    r->T[0] = Tn;
    for (int k = 1; k < nd; ++k) r->T[k] = dT[k];
    r->last_idx = (int32_t)(j + 1);
    r->n_blend += 1;
    r->hash = mix64(r->hash, ((uint64_t)gid << 3) | 4 | (capped ? 8 : 0));
  }
}

/* ------------------------------------------------------------------------ */
/* Render driver                                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
  const orc_scene* sc;
  const orc_camera* cam;
  const orc_opts* opts;
  orc_out* out;
  const gprep* prep;
  const int32_t* vis;
  /* binned lists */
  const int64_t* tile_start;
  const uint32_t* gids;
  /* brute force: global order of visible Gaussians + their rects */
  int brute;
  const uint32_t* order;
  int64_t n_order;
  const int32_t* rec_i;
  int tiles_x;
  int nd;
  int64_t n_pix;
  int64_t n_chunks;
  double* chunk_loss;   /* n_chunks */
  double* chunk_grad;   /* n_chunks x 6 */
  uint64_t* pix_hash;   /* n_pix */
  pthread_mutex_t lock;
  int64_t next_chunk;
} render_job;

static void* render_worker(void* arg) {
  render_job* jb = (render_job*)arg;
  const orc_camera* cam = jb->cam;
  const orc_opts* op = jb->opts;
  orc_out* out = jb->out;
  const int W = cam->width, H = cam->height;
  const double P = (double)W * (double)H;
  const int fd = (jb->sc->feats_bf16 || jb->sc->feats_f32) ? jb->sc->feat_dim : 0;
  uint32_t* tmp_list = NULL;
  if (jb->brute) tmp_list = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(jb->n_order > 0 ? jb->n_order : 1));
  double* fbuf = (double*)malloc(sizeof(double) * (size_t)(fd > 0 ? fd : 1));
  for (;;) {
    pthread_mutex_lock(&jb->lock);
    const int64_t ck = jb->next_chunk++;
    pthread_mutex_unlock(&jb->lock);
    if (ck >= jb->n_chunks) break;
    double closs = 0.0, cgrad[6] = {0, 0, 0, 0, 0, 0};
    const int64_t s = ck * ORC_CHUNK;
    const int64_t e = (s + ORC_CHUNK < jb->n_pix) ? s + ORC_CHUNK : jb->n_pix;
    for (int64_t i = s; i < e; ++i) {
      const int64_t lin = op->pixels ? op->pixels[i] : i;
      const int x = (int)(lin % W), y = (int)(lin / W);
      const int64_t tile = (int64_t)(y / ORC_TILE) * jb->tiles_x + (x / ORC_TILE);
      const uint32_t* list;
      int64_t len;
      if (!jb->brute) {
        list = jb->gids + jb->tile_start[tile];
        len = jb->tile_start[tile + 1] - jb->tile_start[tile];
      } else {
        const int tx = x / ORC_TILE, ty = y / ORC_TILE;
        len = 0;
        for (int64_t k = 0; k < jb->n_order; ++k) {
          const int32_t* oi = jb->rec_i + ORC_NI * (int64_t)jb->order[k];
          if (tx >= oi[ORC_I_X0] && tx <= oi[ORC_I_X1] && ty >= oi[ORC_I_Y0] && ty <= oi[ORC_I_Y1])
            tmp_list[len++] = jb->order[k];
        }
        list = tmp_list;
      }
      pix_result r;
      composite_pixel(jb->prep, jb->vis, list, len, x + 0.5, y + 0.5, jb->nd, op->tie_rel, op->tie_rel_T,
                      jb->sc, fd ? fbuf : NULL, &r);
      uint8_t flags = r.flags;
      for (int64_t j = 0; j < r.n_eval; ++j) flags |= jb->prep[jb->vis[list[j]]].tie;
      uint64_t h = r.hash;
      for (int64_t j = 0; j < r.n_eval; ++j) h = mix64(h, jb->prep[jb->vis[list[j]]].clamp_bits);
      if (op->mean_tangent_gid >= 0) {  /* Algorithm 1: sum of the rendered colours */
        for (int ch = 0; ch < 3; ++ch) {
          closs += r.rgb[ch][0];
          for (int k = 1; k < jb->nd; ++k) cgrad[k - 1] += r.rgb[ch][k];
        }
      } else if (op->target_rgb) {
        const double wpx = op->pixel_weight ? (double)op->pixel_weight[lin] : 1.0;
        for (int ch = 0; ch < 3; ++ch) {
          const double res = r.rgb[ch][0] - (double)op->target_rgb[(int64_t)ch * W * H + lin];
          if (fabs(res) <= kResidualTie) flags |= ORC_TIE_RESIDUAL;
          const double sg = (res > 0) - (res < 0);
          h = mix64(h, (uint64_t)(sg + 1));
          closs += wpx * fabs(res) / (3.0 * P);
          for (int k = 1; k < jb->nd; ++k) cgrad[k - 1] += wpx * sg * r.rgb[ch][k] / (3.0 * P);
        }
        const double res = r.depth[0] - (double)op->target_depth[lin];
        if (fabs(res) <= kResidualTie) flags |= ORC_TIE_RESIDUAL;
        const double sg = (res > 0) - (res < 0);
        h = mix64(h, (uint64_t)(sg + 1));
        closs += op->depth_weight * wpx * fabs(res) / P;
        for (int k = 1; k < jb->nd; ++k) cgrad[k - 1] += op->depth_weight * wpx * sg * r.depth[k] / P;
      }
      if (out->rgb)
        for (int ch = 0; ch < 3; ++ch) out->rgb[3 * i + ch] = r.rgb[ch][0];
      if (out->depth) out->depth[i] = r.depth[0];
      if (out->alpha) out->alpha[i] = 1.0 - r.T[0];
      if (out->final_T) out->final_T[i] = r.T[0];
      if (out->last_idx) out->last_idx[i] = r.last_idx;
      if (out->n_eval) out->n_eval[i] = r.n_eval;
      if (out->n_blend) out->n_blend[i] = r.n_blend;
      if (out->flags) out->flags[i] = flags;
      if (out->feats && fd)
        for (int c = 0; c < fd; ++c) out->feats[i * fd + c] = fbuf[c];
      /* a pixel with zero weight cannot change the loss: leave it out of the signature */
      jb->pix_hash[i] = (op->target_rgb && op->pixel_weight && op->pixel_weight[lin] == 0.0f) ? 0 : h;
    }
    jb->chunk_loss[ck] = closs;
    for (int k = 0; k < 6; ++k) jb->chunk_grad[6 * ck + k] = cgrad[k];
  }
  free(tmp_list);
  free(fbuf);
  return NULL;
}

static int render_impl(const orc_scene* sc, const orc_camera* cam, const double* T_cw, const orc_opts* op,
                       orc_out* out, int brute) {
  if (!sc || !cam || !T_cw || !op || !out) return -1;
  if (op->want_grad && !op->geom64) return -2;
  if (sc->sh_degree < 0 || sc->sh_degree > 3) return -3;
  if (op->target_rgb && !op->target_depth) return -4;
  const int64_t n = sc->n;
  const int W = cam->width, H = cam->height;
  const int tiles_x = (W + ORC_TILE - 1) / ORC_TILE, tiles_y = (H + ORC_TILE - 1) / ORC_TILE;
  const int64_t n_tiles = (int64_t)tiles_x * tiles_y;
  float* cov6 = (float*)malloc(sizeof(float) * 6 * (size_t)(n > 0 ? n : 1));
  int32_t* rec_i = (int32_t*)malloc(sizeof(int32_t) * ORC_NI * (size_t)(n > 0 ? n : 1));
  float* rec_f = (float*)malloc(sizeof(float) * ORC_NF * (size_t)(n > 0 ? n : 1));
  orc_cov3d_f32(n, sc->scales, sc->quats, cov6);
  orc_project_f32(n, sc->means, cov6, cam, T_cw, rec_i, rec_f);

  int64_t total = 0;
  for (int64_t i = 0; i < n; ++i)
    if (rec_i[ORC_NI * i] == ORC_VISIBLE) total += rec_i[ORC_NI * i + ORC_I_COUNT];
  int64_t* tile_start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_tiles + 1));
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(total > 0 ? total : 1));
  uint32_t* gids = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(total > 0 ? total : 1));
  orc_bin(n, rec_i, rec_f, tiles_x, tiles_y, tile_start, keys, gids, total);
  if (out->n_pairs) *out->n_pairs = total;

  /* continuous per-Gaussian layer for the visible ones */
  int32_t* vis = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int64_t n_vis = 0;
  for (int64_t i = 0; i < n; ++i) vis[i] = (rec_i[ORC_NI * i] == ORC_VISIBLE) ? (int32_t)n_vis++ : -1;
  gprep* prep = (gprep*)malloc(sizeof(gprep) * (size_t)(n_vis > 0 ? n_vis : 1));
  prep_ctx pc = {sc, cam, T_cw, rec_i, rec_f, op->geom64, op->want_grad ? ORC_ND : 1, op->tie_rel,
                 op->mean_tangent_gid};
  for (int64_t i = 0; i < n; ++i)
    if (vis[i] >= 0) prep_gauss(&pc, i, prep + vis[i]);

  /* brute-force order: every visible Gaussian by (depth bits, index) */
  uint32_t* order = NULL;
  if (brute) {
    uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n_vis > 0 ? n_vis : 1));
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i)
      if (vis[i] >= 0) tmp[k++] = ((uint64_t)f32_bits(rec_f[ORC_NF * i + ORC_F_Z]) << 32) | (uint64_t)i;
    qsort(tmp, (size_t)n_vis, sizeof(uint64_t), cmp_u64);
    order = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n_vis > 0 ? n_vis : 1));
    for (int64_t i = 0; i < n_vis; ++i) order[i] = (uint32_t)(tmp[i] & 0xffffffffu);
    free(tmp);
  }

  render_job jb;
  memset(&jb, 0, sizeof(jb));
  jb.sc = sc;
  jb.cam = cam;
  jb.opts = op;
  jb.out = out;
  jb.prep = prep;
  jb.vis = vis;
  jb.tile_start = tile_start;
  jb.gids = gids;
  jb.brute = brute;
  jb.order = order;
  jb.n_order = n_vis;
  jb.rec_i = rec_i;
  jb.tiles_x = tiles_x;
  jb.nd = op->want_grad ? ORC_ND : 1;
  jb.n_pix = op->pixels ? op->n_pixels : (int64_t)W * H;
  jb.n_chunks = (jb.n_pix + ORC_CHUNK - 1) / ORC_CHUNK;
  jb.chunk_loss = (double*)calloc((size_t)(jb.n_chunks > 0 ? jb.n_chunks : 1), sizeof(double));
  jb.chunk_grad = (double*)calloc((size_t)(jb.n_chunks > 0 ? jb.n_chunks : 1) * 6, sizeof(double));
  jb.pix_hash = (uint64_t*)calloc((size_t)(jb.n_pix > 0 ? jb.n_pix : 1), sizeof(uint64_t));
  pthread_mutex_init(&jb.lock, NULL);
  int nt = op->n_threads > 0 ? op->n_threads : 1;
  if (nt > 256) nt = 256;
  pthread_t th[256];
  for (int i = 1; i < nt; ++i) pthread_create(&th[i], NULL, render_worker, &jb);
  render_worker(&jb);
  for (int i = 1; i < nt; ++i) pthread_join(th[i], NULL);
  pthread_mutex_destroy(&jb.lock);

  double loss = 0.0, grad[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t c = 0; c < jb.n_chunks; ++c) {
    loss += jb.chunk_loss[c];
    for (int k = 0; k < 6; ++k) grad[k] += jb.chunk_grad[6 * c + k];
  }
  if (out->loss) *out->loss = loss;
  if (out->grad)
    for (int k = 0; k < 6; ++k) out->grad[k] = grad[k];
  if (out->signature) {
    uint64_t h = 88172645463325252ull;
    /* tile membership and order only (not the depth bits, which move with any pose change) */
    for (int64_t j = 0; j < total; ++j) h = mix64(h, (keys[j] >> 32) ^ ((uint64_t)gids[j] << 24));
    for (int64_t i = 0; i < jb.n_pix; ++i) h = mix64(h, jb.pix_hash[i]);
    *out->signature = h;
  }
  free(jb.chunk_loss);
  free(jb.chunk_grad);
  free(jb.pix_hash);
  free(order);
  free(prep);
  free(vis);
  free(keys);
  free(gids);
  free(tile_start);
  free(rec_f);
  free(rec_i);
  free(cov6);
  return 0;
}

int orc_render(const orc_scene* sc, const orc_camera* cam, const double* T_cw, const orc_opts* opts,
               orc_out* out) {
  return render_impl(sc, cam, T_cw, opts, out, 0);
}

int orc_render_brute(const orc_scene* sc, const orc_camera* cam, const double* T_cw, const orc_opts* opts,
                     orc_out* out) {
  if (opts && opts->want_grad) return -5;
  return render_impl(sc, cam, T_cw, opts, out, 1);
}

/* ------------------------------------------------------------------------ */
/* Pose utilities                                                             */
/* ------------------------------------------------------------------------ */

void orc_se3_exp_left(const double* xi, const double* T_in, double* T_out) {
  const double* rho = xi;
  const double* phi = xi + 3;
  const double th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
  const double th = sqrt(th2);
  double a, b, c; /* sin/th, (1-cos)/th^2, (th - sin)/th^3 */
  if (th < 1e-5) {
    a = 1.0 - th2 / 6.0;
    b = 0.5 - th2 / 24.0;
    c = 1.0 / 6.0 - th2 / 120.0;
  } else {
    a = sin(th) / th;
    b = (1.0 - cos(th)) / th2;
    c = (th - sin(th)) / (th2 * th);
  }
  double K[3][3], K2[3][3];
  skew(phi, K);
  mat3_mul(K, K, K2);
  double Rx[3][3], V[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double I = (i == j) ? 1.0 : 0.0;
      Rx[i][j] = I + a * K[i][j] + b * K2[i][j];
      V[i][j] = I + b * K[i][j] + c * K2[i][j];
    }
  double E[4][4] = {{0}};
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) E[i][j] = Rx[i][j];
    E[i][3] = V[i][0] * rho[0] + V[i][1] * rho[1] + V[i][2] * rho[2];
  }
  E[3][3] = 1.0;
  double out[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += E[i][k] * T_in[4 * k + j];
      out[4 * i + j] = s;
    }
  memcpy(T_out, out, sizeof(out));
}

void orc_pose_diff(const double* T1, const double* T2, double* angle_deg, double* dtrans) {
  /* Algorithm 2: R_rel = R1 R2^T, trace clamped to [-1, 3], angle = acos((tr - 1)/2) */
  double tr = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) tr += T1[4 * i + k] * T2[4 * i + k];
  tr = fmin(3.0, fmax(tr, -1.0));
  *angle_deg = 180.0 / kPi * acos((tr - 1.0) / 2.0);
  double d2 = 0.0;
  for (int i = 0; i < 3; ++i) {
    const double d = T1[4 * i + 3] - T2[4 * i + 3];
    d2 += d * d;
  }
  *dtrans = sqrt(d2);
}
