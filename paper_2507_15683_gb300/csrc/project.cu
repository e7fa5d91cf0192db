// Scene packing and per-Gaussian projection (EWA footprint, tile rectangle,
// SH colour and, for the pose gradient, the per-Gaussian pose Jacobian).
//
// The projection follows Algorithm 1 of the paper (p = R X + t, depth = p.z,
// perspective division, then K; Eq. 10). The "discrete layer" -- camera
// depth, projected centre, 2D covariance, radius and tile rectangle -- is
// evaluated with explicitly rounded binary32 operations (__fmul_rn,
// __fadd_rn, ...) in one fixed order, so that the tile lists and sort keys are
// reproducible bit for bit by any IEEE binary32 evaluation of the same
// sequence. Everything after it (conic, colour, Jacobian) is ordinary fp32.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "gsr_internal.h"

namespace gsr {
namespace {

__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float dvd(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float sqr(float a) { return __fsqrt_rn(a); }
// ((a0 b0 + a1 b1) + a2 b2), each operation rounded
__device__ __forceinline__ float dot3(float a0, float b0, float a1, float b1, float a2, float b2) {
  return add(add(mul(a0, b0), mul(a1, b1)), mul(a2, b2));
}

// ---------------------------------------------------------------------------
// Float-float (double-single) arithmetic for the blending centre: world
// coordinates of a few hundred metres leave binary32 camera coordinates with
// ~1e-4 px of error, which the cancellation-heavy pose gradient amplifies.
// Error-free transformations (Knuth two-sum, FMA two-product) keep ~44 bits.
// ---------------------------------------------------------------------------
struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = add(a, b);
  const float bb = sub(s, a);
  return {s, add(sub(a, sub(s, bb)), sub(b, bb))};
}

// (Rh + Rl) . m + (th + tl)
__device__ __forceinline__ ff ff_row(const float* Rh, const float* Rl, float th, float tl, float m0, float m1,
                                     float m2) {
  const float m[3] = {m0, m1, m2};
  float s = th, err = tl;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float ph = mul(Rh[j], m[j]);
    const float pe = __fmaf_rn(Rh[j], m[j], -ph);
    const ff q = two_sum(s, ph);
    s = q.hi;
    err = add(err, add(q.lo, __fmaf_rn(Rl[j], m[j], pe)));
  }
  return two_sum(s, err);
}

// c + f * (num / den) in float-float
__device__ __forceinline__ ff ff_project(ff num, ff den, float f, float c) {
  const float qh = dvd(num.hi, den.hi);
  const float r = add(add(__fmaf_rn(-qh, den.hi, num.hi), num.lo), -mul(qh, den.lo));
  const float ql = dvd(r, den.hi);
  const float ph = mul(f, qh);
  const float pe = __fmaf_rn(f, qh, -ph);
  const ff s = two_sum(c, ph);
  return two_sum(s.hi, add(s.lo, __fmaf_rn(f, ql, pe)));
}

// ---------------------------------------------------------------------------
// Scene packing: binary32 covariance Sigma = R(q) diag(s)^2 R(q)^T
// ---------------------------------------------------------------------------
__global__ void k_pack_scene(const float* __restrict__ means, const float* __restrict__ scales,
                             const float* __restrict__ quats, const float* __restrict__ opacities,
                             const float* __restrict__ sh, int sh_k3, const uint16_t* __restrict__ feats,
                             int feat_dim, int n, int nsh4, float4* __restrict__ pos, float4* __restrict__ cov,
                             float4* __restrict__ sh_out, uint4* __restrict__ feat_out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float qw = quats[4 * i + 0], qx = quats[4 * i + 1], qy = quats[4 * i + 2], qz = quats[4 * i + 3];
    const float n2 = add(add(add(mul(qw, qw), mul(qx, qx)), mul(qy, qy)), mul(qz, qz));
    float w = 1.0f, x = 0.0f, y = 0.0f, z = 0.0f;
    if (n2 > 0.0f) {
      const float nr = sqr(n2);
      w = dvd(qw, nr);
      x = dvd(qx, nr);
      y = dvd(qy, nr);
      z = dvd(qz, nr);
    }
    const float xx = mul(x, x), yy = mul(y, y), zz = mul(z, z);
    const float xy = mul(x, y), xz = mul(x, z), yz = mul(y, z);
    const float wx = mul(w, x), wy = mul(w, y), wz = mul(w, z);
    float r[3][3];
    r[0][0] = sub(1.0f, mul(2.0f, add(yy, zz)));
    r[0][1] = mul(2.0f, sub(xy, wz));
    r[0][2] = mul(2.0f, add(xz, wy));
    r[1][0] = mul(2.0f, add(xy, wz));
    r[1][1] = sub(1.0f, mul(2.0f, add(xx, zz)));
    r[1][2] = mul(2.0f, sub(yz, wx));
    r[2][0] = mul(2.0f, sub(xz, wy));
    r[2][1] = mul(2.0f, add(yz, wx));
    r[2][2] = sub(1.0f, mul(2.0f, add(xx, yy)));
    const float s[3] = {scales[3 * i + 0], scales[3 * i + 1], scales[3 * i + 2]};
    float m[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) m[a][b] = mul(r[a][b], s[b]);
    float S[6];
    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int k = 0; k < 6; ++k)
      S[k] = dot3(m[ia[k]][0], m[ib[k]][0], m[ia[k]][1], m[ib[k]][1], m[ia[k]][2], m[ib[k]][2]);
    const float smax = fmaxf(s[0], fmaxf(s[1], s[2]));
    pos[i] = make_float4(means[3 * i], means[3 * i + 1], means[3 * i + 2], smax);
    cov[2 * i] = make_float4(S[0], S[1], S[2], S[3]);
    cov[2 * i + 1] = make_float4(S[4], S[5], opacities[i], 0.0f);
    float* so = reinterpret_cast<float*>(sh_out + (size_t)i * nsh4);
    for (int k = 0; k < 4 * nsh4; ++k) so[k] = (k < sh_k3) ? sh[(size_t)i * sh_k3 + k] : 0.0f;
    if (feat_dim) {
      uint16_t* fo = reinterpret_cast<uint16_t*>(feat_out + (size_t)i * 4);
      for (int k = 0; k < 32; ++k) fo[k] = feats[(size_t)i * feat_dim + k];
    }
  }
}

// ---------------------------------------------------------------------------
// Real spherical harmonics (Condon-Shortley phase), index l*l + l + m, as
// Cartesian polynomials; values are only used on the unit sphere and their
// gradients only after projection onto the sphere's tangent plane.
//   l=1: -c1 y, c1 z, -c1 x                        c1 = sqrt(3/(4pi))
//   l=2: c2a xy, -c2a yz, c20 (3z^2-1), -c2a xz, c2c (x^2-y^2)
//        c2a = sqrt(15/(4pi)), c20 = sqrt(5/(16pi)), c2c = sqrt(15/(16pi))
//   l=3: -c3a (3x^2 y - y^3), c3b xyz, -c3c y(5z^2-1), c30 z(5z^2-3),
//        -c3c x(5z^2-1), c3d z(x^2-y^2), -c3a (x^3 - 3x y^2)
//        c3a = sqrt(35/(32pi)), c3b = sqrt(105/(4pi)), c3c = sqrt(21/(32pi)),
//        c30 = sqrt(7/(16pi)), c3d = sqrt(105/(16pi))
// ---------------------------------------------------------------------------
constexpr float kC0 = 0.28209479177387814f;
constexpr float kC1 = 0.48860251190291992f;
constexpr float kC2a = 1.0925484305920792f;
constexpr float kC20 = 0.31539156525252005f;
constexpr float kC2c = 0.54627421529603959f;
constexpr float kC3a = 0.59004358992664352f;
constexpr float kC3b = 2.8906114426405538f;
constexpr float kC3c = 0.45704579946446572f;
constexpr float kC30 = 0.37317633259011540f;
constexpr float kC3d = 1.4453057213202769f;

// Accumulates colour (value) and, when GRADC, the Cartesian gradient of each
// channel's polynomial G[ch][0..2].
template <int DEG, bool GRADC>
__device__ __forceinline__ void eval_sh(const float4* __restrict__ shp, float x, float y, float z, float rgb[3],
                                        float G[3][3]) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  constexpr int NF4 = (3 * K + 3) / 4;
  float c[4 * NF4];
#pragma unroll
  for (int k = 0; k < NF4; ++k) {
    const float4 v = __ldg(shp + k);
    c[4 * k] = v.x;
    c[4 * k + 1] = v.y;
    c[4 * k + 2] = v.z;
    c[4 * k + 3] = v.w;
  }
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    rgb[ch] = kC0 * c[ch] + 0.5f;
    if (GRADC) G[ch][0] = G[ch][1] = G[ch][2] = 0.0f;
  }
#define GS_ACC(k, Y, gx, gy, gz)                                  \
  _Pragma("unroll") for (int ch = 0; ch < 3; ++ch) {               \
    const float co = c[3 * (k) + ch];                              \
    rgb[ch] = fmaf(co, (Y), rgb[ch]);                              \
    if (GRADC) {                                                   \
      G[ch][0] = fmaf(co, (gx), G[ch][0]);                         \
      G[ch][1] = fmaf(co, (gy), G[ch][1]);                         \
      G[ch][2] = fmaf(co, (gz), G[ch][2]);                         \
    }                                                              \
  }
  if (DEG >= 1) {
    GS_ACC(1, -kC1 * y, 0.0f, -kC1, 0.0f);
    GS_ACC(2, kC1 * z, 0.0f, 0.0f, kC1);
    GS_ACC(3, -kC1 * x, -kC1, 0.0f, 0.0f);
  }
  if (DEG >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    GS_ACC(4, kC2a * x * y, kC2a * y, kC2a * x, 0.0f);
    GS_ACC(5, -kC2a * y * z, 0.0f, -kC2a * z, -kC2a * y);
    GS_ACC(6, kC20 * (3.0f * zz - 1.0f), 0.0f, 0.0f, 6.0f * kC20 * z);
    GS_ACC(7, -kC2a * x * z, -kC2a * z, 0.0f, -kC2a * x);
    GS_ACC(8, kC2c * (xx - yy), 2.0f * kC2c * x, -2.0f * kC2c * y, 0.0f);
    if (DEG >= 3) {
      GS_ACC(9, -kC3a * (3.0f * xx * y - yy * y), -kC3a * 6.0f * x * y, -kC3a * (3.0f * xx - 3.0f * yy), 0.0f);
      GS_ACC(10, kC3b * x * y * z, kC3b * y * z, kC3b * x * z, kC3b * x * y);
      GS_ACC(11, -kC3c * y * (5.0f * zz - 1.0f), 0.0f, -kC3c * (5.0f * zz - 1.0f), -kC3c * 10.0f * y * z);
      GS_ACC(12, kC30 * z * (5.0f * zz - 3.0f), 0.0f, 0.0f, kC30 * (15.0f * zz - 3.0f));
      GS_ACC(13, -kC3c * x * (5.0f * zz - 1.0f), -kC3c * (5.0f * zz - 1.0f), 0.0f, -kC3c * 10.0f * x * z);
      GS_ACC(14, kC3d * z * (xx - yy), kC3d * 2.0f * x * z, -kC3d * 2.0f * y * z, kC3d * (xx - yy));
      GS_ACC(15, -kC3a * (xx * x - 3.0f * x * yy), -kC3a * (3.0f * xx - 3.0f * yy), kC3a * 6.0f * x * y, 0.0f);
    }
  }
#undef GS_ACC
}

template <bool GRADC>
__device__ __forceinline__ void eval_sh_deg(int deg, const float4* shp, float x, float y, float z, float rgb[3],
                                            float G[3][3]) {
  switch (deg) {
    case 0: eval_sh<0, GRADC>(shp, x, y, z, rgb, G); break;
    case 1: eval_sh<1, GRADC>(shp, x, y, z, rgb, G); break;
    case 2: eval_sh<2, GRADC>(shp, x, y, z, rgb, G); break;
    default: eval_sh<3, GRADC>(shp, x, y, z, rgb, G); break;
  }
}

// ---------------------------------------------------------------------------
// Projection, discrete pass. Decides visibility, the tile rectangle and the
// sort key, counts pairs per tile and appends a record; the continuous
// quantities are filled in by k_shade over the compact records. Record fields
// written here: rec_m = (rect, view, depth bits), rec_a = (binary32
// covariance a, b, c, -), rec_b.w = Gaussian index.
//
// Every warp works on its own: it walks chunks of 32 Gaussians (means loaded
// one chunk ahead), runs a cheap conservative test (camera transform, near
// plane, reach of the footprint) of each against every view of the call, and
// appends the surviving (Gaussian, view) pairs to its own queue in shared
// memory; whenever 32 are queued (and at the end) it drains them through the
// exact discrete layer with all of its lanes busy. No barrier joins the warps
// of a block. Block b appends its
// records to segment b % kRecRegions, and its warps take the Gaussians
// [256 b, 256 b + 256) first (then every gridDim.x * 256).
// ---------------------------------------------------------------------------
constexpr int kWarpQ = 64;  // (Gaussian, view) queue entries per warp: a drain of 32 leaves at most 31

// 16-byte asynchronous copy global -> shared (both 16-byte aligned)
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}

// camera-space position in the binary32 operation order of the oracle
__device__ __forceinline__ void cam_xyz(const View& V, float4 p4, float& px, float& py, float& pz) {
  px = add(add(add(mul(V.R[0], p4.x), mul(V.R[1], p4.y)), mul(V.R[2], p4.z)), V.t[0]);
  py = add(add(add(mul(V.R[3], p4.x), mul(V.R[4], p4.y)), mul(V.R[5], p4.z)), V.t[1]);
  pz = add(add(add(mul(V.R[6], p4.x), mul(V.R[7], p4.y)), mul(V.R[8], p4.z)), V.t[2]);
}

// Conservative reach: radius <= 3 sqrt(s_max^2 |J|_F^2 + 0.3 + sqrt(0.1)) + 1,
// with margins for rounding; a Gaussian that fails it has an empty rectangle
// under the exact rule, so skipping it changes nothing. The test runs for
// every (Gaussian, view): the camera transform and the near-plane test are
// the exact layer's, bit for bit, while the division and the square root are
// the fast approximate ones. Their relative errors (a few 1e-7) move u and v
// by far less than the test's margins (1 px on the image bounds, 1 % and
// 3 px on the reach).
__device__ __forceinline__ bool may_reach(const View& V, float4 p4) {
  float px, py, pz;
  cam_xyz(V, p4, px, py, pz);
  if (!(pz >= 0.2f)) return false;
  const float iz = __fdividef(1.0f, pz);
  const float u = fmaf(V.fx * px, iz, V.cx);
  const float v = fmaf(V.fy * py, iz, V.cy);
  const float r2 = (p4.w * p4.w * V.jb2 * (iz * iz) + 0.62f) * 1.01f;
  const float reach = 3.0f * (r2 * rsqrtf(r2)) + 3.0f;
  const float wx = (float)(kTile * V.tiles_x), wy = (float)(kTile * V.tiles_y);
  return u + reach >= -1.0f && u - reach <= wx + 1.0f && v + reach >= -1.0f && v - reach <= wy + 1.0f;
}

// The exact binary32 discrete layer (Sec. 3.1 projection, EWA footprint,
// 3-sigma radius and tile rectangle). Returns false when the Gaussian has no
// tile in this view.
__device__ __forceinline__ bool discrete_layer(const View& V, float4 p4, float4 c0, float4 c1, float& pz, float& ca,
                                               float& cb, float& cc, int& x0, int& x1, int& y0, int& y1) {
  float px, py;
  cam_xyz(V, p4, px, py, pz);
  if (!(pz >= 0.2f)) return false;
  const float ix = dvd(px, pz), iy = dvd(py, pz);
  const float u = add(mul(V.fx, ix), V.cx);
  const float v = add(mul(V.fy, iy), V.cy);
  const float xh = mul(fminf(V.limx, fmaxf(-V.limx, ix)), pz);
  const float yh = mul(fminf(V.limy, fmaxf(-V.limy, iy)), pz);
  const float pz2 = mul(pz, pz);
  const float j00 = dvd(V.fx, pz), j02 = -dvd(mul(V.fx, xh), pz2);
  const float j11 = dvd(V.fy, pz), j12 = -dvd(mul(V.fy, yh), pz2);
  float T[2][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T[0][k] = add(mul(j00, V.R[k]), mul(j02, V.R[6 + k]));
    T[1][k] = add(mul(j11, V.R[3 + k]), mul(j12, V.R[6 + k]));
  }
  const float S[3][3] = {{c0.x, c0.y, c0.z}, {c0.y, c0.w, c1.x}, {c0.z, c1.x, c1.y}};
  float U[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k) U[a][k] = dot3(T[a][0], S[0][k], T[a][1], S[1][k], T[a][2], S[2][k]);
  ca = add(dot3(U[0][0], T[0][0], U[0][1], T[0][1], U[0][2], T[0][2]), 0.3f);
  cb = dot3(U[0][0], T[1][0], U[0][1], T[1][1], U[0][2], T[1][2]);
  cc = add(dot3(U[1][0], T[1][0], U[1][1], T[1][1], U[1][2], T[1][2]), 0.3f);
  const float det = sub(mul(ca, cc), mul(cb, cb));
  if (!(det > 0.0f)) return false;
  const float mid = mul(0.5f, add(ca, cc));
  const float disc = sub(mul(mid, mid), det);
  const float lam = add(mid, sqr(fmaxf(0.1f, disc)));
  const float r = ceilf(mul(3.0f, sqr(lam)));
  if (!(r > 0.0f)) return false;
  // division by 16 is exact: multiply by 1/16
  float fx0 = floorf(mul(sub(u, r), 0.0625f)), fx1 = floorf(mul(add(u, r), 0.0625f));
  float fy0 = floorf(mul(sub(v, r), 0.0625f)), fy1 = floorf(mul(add(v, r), 0.0625f));
  fx0 = fmaxf(fx0, 0.0f);
  fy0 = fmaxf(fy0, 0.0f);
  fx1 = fminf(fx1, (float)(V.tiles_x - 1));
  fy1 = fminf(fy1, (float)(V.tiles_y - 1));
  if (fx0 > fx1 || fy0 > fy1) return false;
  x0 = (int)fx0;
  x1 = (int)fx1;
  y0 = (int)fy0;
  y1 = (int)fy1;
  return true;
}

__global__ void __launch_bounds__(256) k_project(SceneDev sc, const View* __restrict__ views, int n_views, Work w) {
  // per warp, a ring of kWarpQ (Gaussian, view) entries with the Gaussian's
  // mean and its covariance, copied (cp.async) when the entry is queued so that
  // a drain finds them in shared memory
  __shared__ int2 s_q[kTileThreads / 32][kWarpQ];
  __shared__ float4 s_qp[kTileThreads / 32][kWarpQ];
  __shared__ float4 s_qc[kTileThreads / 32][kWarpQ][2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  const unsigned region = blockIdx.x % kRecRegions;
  const int4 hdr = w.ranges[0];  // (ranges, total length): only partitions in view are walked
  int2* q = s_q[wid];
  float4* qp = s_qp[wid];
  float4(*qc)[2] = s_qc[wid];
  unsigned qh = 0, qn = 0;  // ring head and queued entries (warp-uniform)
  // the exact layer over the cnt <= 32 entries at the head, one per lane
  auto drain = [&](unsigned cnt) {
    asm volatile("cp.async.wait_all;" ::: "memory");  // this lane's covariance copies
    __syncwarp();                                      // ... and every other lane's
    bool vis = false;
    int i = 0, vi = 0, x0 = 0, x1 = 0, y0 = 0, y1 = 0;
    float pz = 0.f, ca = 0.f, cb = 0.f, cc = 0.f;
    if ((unsigned)lane < cnt) {
      const unsigned e = (qh + (unsigned)lane) & (kWarpQ - 1);
      const int2 qe = q[e];
      i = qe.x;
      vi = qe.y;
      vis = discrete_layer(views[vi], qp[e], qc[e][0], qc[e][1], pz, ca, cb, cc, x0, x1, y0, y1);
    }
    const unsigned vmask = __ballot_sync(0xffffffffu, vis);
    if (vmask == 0u) return;
    // warp-aggregated append into this block's record segment
    unsigned slot0 = 0;
    const int leader = __ffs(vmask) - 1;
    if (lane == leader) slot0 = atomicAdd(&w.ctr->rec_region[region], (unsigned)__popc(vmask));
    slot0 = __shfl_sync(0xffffffffu, slot0, leader);
    if (!vis) return;
    const unsigned local = slot0 + __popc(vmask & lt_mask);
    if (local >= w.rec_seg) {
      atomicOr(&w.ctr->overflow, 1u);
      return;
    }
    const unsigned slot = region * w.rec_seg + local;
    w.rec_a[slot] = make_float4(ca, cb, cc, 0.0f);
    w.rec_b[slot] = make_float4(0.0f, 0.0f, 0.0f, __int_as_float(i));
    w.rec_m[slot] = make_uint4((unsigned)x0 | ((unsigned)x1 << 16), (unsigned)y0 | ((unsigned)y1 << 16),
                               (unsigned)vi, __float_as_uint(pz));
    const View& V = views[vi];
    for (int ty = y0; ty <= y1; ++ty)
      for (int tx = x0; tx <= x1; ++tx) atomicAdd(&w.tile_count[V.tile_base + ty * V.tiles_x + tx], 1u);
  };
  // Gaussian index of flat position f over the active ranges, or -1 (one
  // range, the common call: read once, so that the means' loads do not wait
  // on it)
  const int4 rg1 = hdr.x == 1 ? w.ranges[1] : make_int4(0, 0, 0, 0);
  auto gaussian_of = [&](int f) -> int {
    if (f >= hdr.y) return -1;
    if (hdr.x == 1) return rg1.x + (f - rg1.z);
    int lo = 1, hi = hdr.x;  // last range whose prefix is <= f
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (w.ranges[mid].z <= f) lo = mid; else hi = mid - 1;
    }
    const int4 rg = w.ranges[lo];
    return rg.x + (f - rg.z);
  };
  // chunks of 32 Gaussians: this warp's first is 256 blockIdx.x + 32 wid; the
  // next chunk's means are loaded before the current one is tested
  const int stride = gridDim.x * kTileThreads;
  int i_next = gaussian_of(blockIdx.x * kTileThreads + wid * 32 + lane);
  float4 p_next = i_next >= 0 ? __ldg(sc.pos + i_next) : make_float4(0.f, 0.f, 0.f, 0.f);
  for (int base = blockIdx.x * kTileThreads + wid * 32; base < hdr.y; base += stride) {  // warp-uniform loop
    const int i = i_next;
    const bool valid = i >= 0;
    const float4 p4 = p_next;
    i_next = gaussian_of(base + stride + lane);
    if (i_next >= 0) p_next = __ldg(sc.pos + i_next);
    for (int vi = 0; vi < n_views; ++vi) {
      const bool pass = valid && may_reach(views[vi], p4);
      const unsigned pm = __ballot_sync(0xffffffffu, pass);
      if (pass) {
        const unsigned e = (qh + qn + (unsigned)__popc(pm & lt_mask)) & (kWarpQ - 1);
        q[e] = make_int2(i, vi);
        qp[e] = p4;
        cp_async16(&qc[e][0], sc.cov + 2 * i);
        cp_async16(&qc[e][1], sc.cov + 2 * i + 1);
      }
      qn += __popc(pm);
      if (qn >= 32u) {  // a full warp of work
        __syncwarp();
        drain(32u);
        __syncwarp();  // the drained slots are free again
        qh = (qh + 32u) & (kWarpQ - 1);
        qn -= 32u;
      }
    }
  }
  __syncwarp();
  if (qn) drain(qn);
}

// ---------------------------------------------------------------------------
// Shading pass over the compact records: conic, SH colour, float-float
// blending centre and, for the pose gradient, the per-record pose Jacobian.
// ---------------------------------------------------------------------------
template <bool GRAD>
__global__ void __launch_bounds__(256, 3) k_shade(SceneDev sc, const View* __restrict__ views, Work w) {
  if (w.ctr->overflow) return;
  for (uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x; slot < w.rec_cap; slot += gridDim.x * blockDim.x) {
    const uint32_t reg = slot / w.rec_seg, loc = slot - reg * w.rec_seg;
    if (loc >= min(w.ctr->rec_region[reg], w.rec_seg)) continue;
    const float4 ra = w.rec_a[slot];
    const int i = __float_as_int(w.rec_b[slot].w);
    const uint4 m = w.rec_m[slot];
    const View& V = views[m.z];
    const float ca = ra.x, cb = ra.y, cc = ra.z;
    const float4 p4 = __ldg(sc.pos + i);
    const float4 c0 = __ldg(sc.cov + 2 * i);
    const float4 c1 = __ldg(sc.cov + 2 * i + 1);
    const float pz = __uint_as_float(m.w);
    // conic from the binary32 covariance; determinant with one compensated step
    const float bb = cb * cb;
    const float e = __fmaf_rn(-cb, cb, bb);
    const float f = __fmaf_rn(ca, cc, -bb);
    const float detc = f + e;
    const float inv = 1.0f / detc;
    const float A = cc * inv, B = -cb * inv, C = ca * inv;
    // colour from SH at dir = normalize(mean - camera centre)
    const float dxw = p4.x - V.cw[0], dyw = p4.y - V.cw[1], dzw = p4.z - V.cw[2];
    const float dn = sqrtf(dxw * dxw + dyw * dyw + dzw * dzw);
    const float rn = 1.0f / dn;
    const float dirx = dxw * rn, diry = dyw * rn, dirz = dzw * rn;
    float rgb[3], G[3][3];
    eval_sh_deg<GRAD>(sc.sh_degree, sc.sh + (size_t)i * sc.nsh4, dirx, diry, dirz, rgb, G);
    bool clampc[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      clampc[ch] = rgb[ch] < 0.0f;
      rgb[ch] = fmaxf(rgb[ch], 0.0f);
    }
    // blending centre in float-float; high parts in rec_a, low parts as half2
    const ff fpx = ff_row(V.R, V.Rl, V.t[0], V.tl[0], p4.x, p4.y, p4.z);
    const ff fpy = ff_row(V.R + 3, V.Rl + 3, V.t[1], V.tl[1], p4.x, p4.y, p4.z);
    const ff fpz = ff_row(V.R + 6, V.Rl + 6, V.t[2], V.tl[2], p4.x, p4.y, p4.z);
    const ff fu = ff_project(fpx, fpz, V.fx, V.cx);
    const ff fv = ff_project(fpy, fpz, V.fy, V.cy);
    const __half2 lo2 = __floats2half2_rn(fu.lo, fv.lo);
    w.rec_a[slot] = make_float4(fu.hi, fv.hi, A, B);
    // rec_b.w (the Gaussian index, the sort's tie key) stays as the projection wrote it
    float* rb = reinterpret_cast<float*>(w.rec_b + slot);
    *reinterpret_cast<float2*>(rb) = make_float2(C, c1.z);
    rb[2] = pz;
    w.rec_c[slot] = make_float4(rgb[0], rgb[1], rgb[2], *reinterpret_cast<const float*>(&lo2));

    if (GRAD) {
      // Pose Jacobian of (u, v, A, B, C, z) w.r.t. xi = (rho, phi) and of (r, g, b)
      // w.r.t. rho, by forward differentiation along the six tangent directions:
      // d p = rho + phi x p; d Sigma_cam = [phi]x Sigma_cam - Sigma_cam [phi]x;
      // d (mean - camera centre) = R^T rho.
      const float* R = V.R;
      const float px = fpx.hi, py = fpy.hi;
      const float ix = px / pz, iy = py / pz;
      const float Sw[3][3] = {{c0.x, c0.y, c0.z}, {c0.y, c0.w, c1.x}, {c0.z, c1.x, c1.y}};
      float Q[3][3], Sc[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) Q[a][b] = R[3 * a] * Sw[0][b] + R[3 * a + 1] * Sw[1][b] + R[3 * a + 2] * Sw[2][b];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) Sc[a][b] = Q[a][0] * R[3 * b] + Q[a][1] * R[3 * b + 1] + Q[a][2] * R[3 * b + 2];
      const bool clx = (ix < -V.limx) || (ix > V.limx);
      const bool cly = (iy < -V.limy) || (iy > V.limy);
      const float Lx = ix < 0.0f ? -V.limx : V.limx, Ly = iy < 0.0f ? -V.limy : V.limy;
      const float zi = 1.0f / pz;
      const float xh = clx ? Lx * pz : px, yh = cly ? Ly * pz : py;
      const float j00 = V.fx * zi, j02 = -V.fx * xh * zi * zi;
      const float j11 = V.fy * zi, j12 = -V.fy * yh * zi * zi;
      float K[2][3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        K[0][k] = j00 * Sc[0][k] + j02 * Sc[2][k];
        K[1][k] = j11 * Sc[1][k] + j12 * Sc[2][k];
      }
      const float di = 1.0f / detc;
      float jac[45];
      const float pc[3] = {px, py, pz};
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        float dp[3];
        if (k < 3) {
          dp[0] = (k == 0) ? 1.f : 0.f;
          dp[1] = (k == 1) ? 1.f : 0.f;
          dp[2] = (k == 2) ? 1.f : 0.f;
        } else {
          const int e3 = k - 3;  // e x p
          dp[0] = (e3 == 1) ? pc[2] : (e3 == 2) ? -pc[1] : 0.f;
          dp[1] = (e3 == 0) ? -pc[2] : (e3 == 2) ? pc[0] : 0.f;
          dp[2] = (e3 == 0) ? pc[1] : (e3 == 1) ? -pc[0] : 0.f;
        }
        const float du = V.fx * (dp[0] - ix * dp[2]) * zi;
        const float dv = V.fy * (dp[1] - iy * dp[2]) * zi;
        const float dxh = clx ? Lx * dp[2] : dp[0];
        const float dyh = cly ? Ly * dp[2] : dp[1];
        const float dj00 = -j00 * dp[2] * zi;
        const float dj02 = -V.fx * (dxh - 2.0f * xh * dp[2] * zi) * zi * zi;
        const float dj11 = -j11 * dp[2] * zi;
        const float dj12 = -V.fy * (dyh - 2.0f * yh * dp[2] * zi) * zi * zi;
        // S = dJ K^T
        const float S00 = dj00 * K[0][0] + dj02 * K[0][2];
        const float S01 = dj00 * K[1][0] + dj02 * K[1][2];
        const float S10 = dj11 * K[0][1] + dj12 * K[0][2];
        const float S11 = dj11 * K[1][1] + dj12 * K[1][2];
        float dm00 = 2.0f * S00, dm01 = S01 + S10, dm11 = 2.0f * S11;
        if (k >= 3) {
          // D = X + X^T with X = [e]x Sc
          const int e3 = k - 3;
          float X[3][3];
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            if (e3 == 0) { X[0][b] = 0.f; X[1][b] = -Sc[2][b]; X[2][b] = Sc[1][b]; }
            else if (e3 == 1) { X[0][b] = Sc[2][b]; X[1][b] = 0.f; X[2][b] = -Sc[0][b]; }
            else { X[0][b] = -Sc[1][b]; X[1][b] = Sc[0][b]; X[2][b] = 0.f; }
          }
          float D[3][3];
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) D[a][b] = X[a][b] + X[b][a];
          float JD[2][3];
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            JD[0][b] = j00 * D[0][b] + j02 * D[2][b];
            JD[1][b] = j11 * D[1][b] + j12 * D[2][b];
          }
          dm00 += JD[0][0] * j00 + JD[0][2] * j02;
          dm01 += JD[0][1] * j11 + JD[0][2] * j12;
          dm11 += JD[1][1] * j11 + JD[1][2] * j12;
        }
        const float ddet = dm00 * cc + ca * dm11 - 2.0f * cb * dm01;
        const float dA = (dm11 - cc * ddet * di) * di;
        const float dB = -(dm01 - cb * ddet * di) * di;
        const float dC = (dm00 - ca * ddet * di) * di;
        jac[0 * 6 + k] = du;
        jac[1 * 6 + k] = dv;
        jac[2 * 6 + k] = dA;
        jac[3 * 6 + k] = dB;
        jac[4 * 6 + k] = dC;
        jac[5 * 6 + k] = dp[2];
      }
      // colour rows (rho only): d rgb_ch / d rho_k = G_ch . (I - dir dir^T) R^T e_k / |d|
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const float gd = G[ch][0] * dirx + G[ch][1] * diry + G[ch][2] * dirz;
        const float gp0 = (G[ch][0] - gd * dirx) * rn, gp1 = (G[ch][1] - gd * diry) * rn,
                    gp2 = (G[ch][2] - gd * dirz) * rn;
#pragma unroll
        for (int k = 0; k < 3; ++k)
          jac[36 + 3 * ch + k] = clampc[ch] ? 0.0f : gp0 * R[3 * k] + gp1 * R[3 * k + 1] + gp2 * R[3 * k + 2];
      }
      // Stored for the compositor's packed FMAs over the direction pairs
      // (0,1), (2,3), (4,5). With the pixel offset (dx, dy) = centre - pixel,
      //   -dpower/dxi = dx (A du + B dv) + dy (B du + C dv) + dx^2 dA/2
      //                 + dx dy dB + dy^2 dC/2,
      // so pair k holds three float4: (P, Q), (dA/2, dB), (dC/2, dz), each
      // as the two directions of the pair, with P = A du + B dv and
      // Q = B du + C dv; then d(r, g, b)/d rho in three float4 (three
      // directions and a zero).
      float jt[48];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int d = 2 * k + h;
          jt[12 * k + h] = A * jac[d] + B * jac[6 + d];
          jt[12 * k + 2 + h] = B * jac[d] + C * jac[6 + d];
          jt[12 * k + 4 + h] = 0.5f * jac[12 + d];
          jt[12 * k + 6 + h] = jac[18 + d];
          jt[12 * k + 8 + h] = 0.5f * jac[24 + d];
          jt[12 * k + 10 + h] = jac[30 + d];
        }
      }
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
#pragma unroll
        for (int k = 0; k < 3; ++k) jt[36 + 4 * ch + k] = jac[36 + 3 * ch + k];
        jt[39 + 4 * ch] = 0.0f;
      }
      float4* jo = reinterpret_cast<float4*>(w.rec_j + (size_t)slot * kJacStride);
#pragma unroll
      for (int q = 0; q < 12; ++q) jo[q] = make_float4(jt[4 * q], jt[4 * q + 1], jt[4 * q + 2], jt[4 * q + 3]);
    }
  }
}

// ---------------------------------------------------------------------------
// Algorithm 1 (render-gradient visibility check), per-Gaussian parts.
//
// In-image test: (U, V) = K (p / z) with p = R X + t in float-float (the
// blending centre's arithmetic), M^i = U in [0, W) and V in [0, H). No depth
// test: the algorithm has none, and M^r is false behind the near plane.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_vis_inimage(SceneDev sc, const View* __restrict__ views,
                                                     uint8_t* __restrict__ mask, float2* __restrict__ uv,
                                                     float* __restrict__ grad) {
  const View& V = views[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < sc.n; i += gridDim.x * blockDim.x) {
    const float4 p4 = __ldg(sc.pos + i);
    const ff fpx = ff_row(V.R, V.Rl, V.t[0], V.tl[0], p4.x, p4.y, p4.z);
    const ff fpy = ff_row(V.R + 3, V.Rl + 3, V.t[1], V.tl[1], p4.x, p4.y, p4.z);
    const ff fpz = ff_row(V.R + 6, V.Rl + 6, V.t[2], V.tl[2], p4.x, p4.y, p4.z);
    const float u = ff_project(fpx, fpz, V.fx, V.cx).hi;
    const float v = ff_project(fpy, fpz, V.fy, V.cy).hi;
    const bool in = u >= 0.0f && u < (float)V.width && v >= 0.0f && v < (float)V.height;
    mask[i] = in ? 4u : 0u;
    uv[i] = make_float2(u, v);
    if (grad) {
      grad[3 * (size_t)i] = 0.0f;
      grad[3 * (size_t)i + 1] = 0.0f;
      grad[3 * (size_t)i + 2] = 0.0f;
    }
  }
}

// Chain rule from the reverse pass's per-record sums to the mean. Moving the
// mean by d moves the camera-frame centre by R d exactly as a translation
// rho = R d of the pose does, and the view direction by d exactly as that
// translation does (d(X - c) = R^T rho), while the camera-frame covariance is
// unchanged in both; so dL/dX = R^T dL/drho restricted to this Gaussian, and
// dL/drho_k = -(P_k s_x + Q_k s_y + dA_k/2 s_xx + dB_k s_xy + dC_k/2 s_yy)
//             + (dr_k + dg_k + db_k) s_w
// with the record's pose Jacobian rows and accumulated sums. M^r = some
// component of the gradient is non-zero; M = M^r and M^i (bit 2 set by
// k_vis_inimage).
__global__ void __launch_bounds__(256) k_vis_chain(const View* __restrict__ views, Work w,
                                                   const float* __restrict__ acc, uint8_t* __restrict__ mask,
                                                   float* __restrict__ grad) {
  if (w.ctr->overflow) return;
  const View& V = views[0];
  const int lane = threadIdx.x & 31;
  for (uint32_t base = blockIdx.x * blockDim.x; base < w.rec_cap; base += gridDim.x * blockDim.x) {
    const uint32_t slot = base + threadIdx.x;
    bool keep = false;
    if (slot < w.rec_cap) {
      const uint32_t reg = slot / w.rec_seg, loc = slot - reg * w.rec_seg;
      if (loc < min(w.ctr->rec_region[reg], w.rec_seg)) {
        const float4 a0 = reinterpret_cast<const float4*>(acc)[2 * (size_t)slot];
        const float4 a1 = reinterpret_cast<const float4*>(acc)[2 * (size_t)slot + 1];
        if (a0.x != 0.0f || a0.y != 0.0f || a0.z != 0.0f || a0.w != 0.0f || a1.x != 0.0f || a1.y != 0.0f) {
          const float* J = w.rec_j + (size_t)slot * kJacStride;
          float gr[3];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const int o = 12 * (d >> 1) + (d & 1);  // direction d of pair d / 2
            const float sp = J[o] * a0.x + J[o + 2] * a0.y + J[o + 4] * a0.z + J[o + 6] * a0.w + J[o + 8] * a1.x;
            gr[d] = (J[36 + d] + J[40 + d] + J[44 + d]) * a1.y - sp;
          }
          float g[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) g[a] = V.R[a] * gr[0] + V.R[3 + a] * gr[1] + V.R[6 + a] * gr[2];
          const int i = __float_as_int(w.rec_b[slot].w);
          if (grad) {
            grad[3 * (size_t)i] = g[0];
            grad[3 * (size_t)i + 1] = g[1];
            grad[3 * (size_t)i + 2] = g[2];
          }
          if (g[0] != 0.0f || g[1] != 0.0f || g[2] != 0.0f) {
            const uint8_t m = mask[i];
            keep = (m & 4u) != 0;
            mask[i] = (uint8_t)(m | 2u | (keep ? 1u : 0u));
          }
        }
      }
    }
    const unsigned km = __ballot_sync(0xffffffffu, keep);
    if (lane == 0 && km) atomicAdd(&w.ctr->vis_count, (unsigned)__popc(km));
  }
}

// Order-preserving compaction of the kept Gaussians: per-block counts, one
// scan block, scatter (blocks of kVisBlock Gaussians, 256 threads).
__global__ void __launch_bounds__(256) k_vis_count(const uint8_t* __restrict__ mask, int n,
                                                   uint32_t* __restrict__ blk) {
  __shared__ uint32_t s_w[8];
  const int base = blockIdx.x * kVisBlock;
  uint32_t c = 0;
#pragma unroll
  for (int k = 0; k < kVisBlock / 256; ++k) {
    const int i = base + k * 256 + threadIdx.x;
    c += (i < n && (mask[i] & 1u)) ? 1u : 0u;
  }
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int k = 0; k < 8; ++k) t += s_w[k];
    blk[blockIdx.x] = t;
  }
}

// exclusive scan of nb counters in place (one block of 1024 threads)
__global__ void __launch_bounds__(1024) k_vis_scan(uint32_t* __restrict__ blk, int nb) {
  __shared__ uint32_t s_w[32];
  __shared__ uint32_t s_carry;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nb; b0 += 1024) {
    const int i = b0 + tid;
    const uint32_t x = i < nb ? blk[i] : 0u;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      uint32_t t = s_w[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      s_w[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    const uint32_t carry = s_carry;
    const uint32_t excl = carry + (wid ? s_w[wid - 1] : 0u) + inc - x;
    if (i < nb) blk[i] = excl;
    __syncthreads();
    if (tid == 0) s_carry = carry + s_w[31];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_vis_scatter(const uint8_t* __restrict__ mask, const float2* __restrict__ uv,
                                                     int n, const uint32_t* __restrict__ blk,
                                                     int32_t* __restrict__ vis_gid, float2* __restrict__ vis_uv) {
  __shared__ uint32_t s_w[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int base = blockIdx.x * kVisBlock;
  uint32_t off = blk[blockIdx.x];
  for (int k = 0; k < kVisBlock / 256; ++k) {
    const int i = base + k * 256 + threadIdx.x;
    const bool m = i < n && (mask[i] & 1u);
    const unsigned b = __ballot_sync(0xffffffffu, m);
    if (lane == 0) s_w[wid] = (uint32_t)__popc(b);
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      before += q < wid ? s_w[q] : 0u;
      total += s_w[q];
    }
    if (m) {
      const uint32_t o = off + before + (uint32_t)__popc(b & ((1u << lane) - 1u));
      if (vis_gid) vis_gid[o] = i;
      if (vis_uv) vis_uv[o] = uv[i];
    }
    off += total;
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_pack_scene(const float* means, const float* scales, const float* quats,
                              const float* opacities, const float* sh, int sh_k3, const uint16_t* feats,
                              int feat_dim, int n, int nsh4, float4* pos, float4* cov, float4* sh_out,
                              uint4* feat_out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
  k_pack_scene<<<grid, 256, 0, st>>>(means, scales, quats, opacities, sh, sh_k3, feats, feat_dim, n, nsh4, pos,
                                     cov, sh_out, feat_out);
  return cudaGetLastError();
}

cudaError_t launch_project(const SceneDev& sc, const View* views, int n_views, const Work& w, int grid,
                           cudaStream_t st) {
  if (sc.n <= 0 || n_views <= 0) return cudaSuccess;
  const int need = (sc.n + 255) / 256;  // the active ranges never exceed the scene
  const int g = need < grid ? need : grid;
  k_project<<<g, 256, 0, st>>>(sc, views, n_views, w);
  return cudaGetLastError();
}

cudaError_t launch_shade(const SceneDev& sc, const View* views, const Work& w, bool grad, int grid,
                         cudaStream_t st) {
  if (sc.n <= 0 || w.rec_cap == 0) return cudaSuccess;
  const int need = (int)((w.rec_cap + 255) / 256);
  const int g = need < grid ? need : grid;
  if (grad)
    k_shade<true><<<g, 256, 0, st>>>(sc, views, w);
  else
    k_shade<false><<<g, 256, 0, st>>>(sc, views, w);
  return cudaGetLastError();
}

cudaError_t launch_vis_inimage(const SceneDev& sc, const View* views, uint8_t* mask, float2* uv, float* grad,
                               int grid, cudaStream_t st) {
  if (sc.n <= 0) return cudaSuccess;
  const int need = (sc.n + 255) / 256;
  k_vis_inimage<<<need < grid ? need : grid, 256, 0, st>>>(sc, views, mask, uv, grad);
  return cudaGetLastError();
}

cudaError_t launch_vis_chain(const View* views, const Work& w, const float* acc, uint8_t* mask, float* grad,
                             int grid, cudaStream_t st) {
  if (w.rec_cap == 0) return cudaSuccess;
  const int need = (int)((w.rec_cap + 255) / 256);
  k_vis_chain<<<need < grid ? need : grid, 256, 0, st>>>(views, w, acc, mask, grad);
  return cudaGetLastError();
}

cudaError_t launch_vis_compact(const uint8_t* mask, const float2* uv, int n, uint32_t* blk, int32_t* vis_gid,
                               float2* vis_uv, cudaStream_t st) {
  if (n <= 0 || (!vis_gid && !vis_uv)) return cudaSuccess;
  const int nb = (n + kVisBlock - 1) / kVisBlock;
  k_vis_count<<<nb, 256, 0, st>>>(mask, n, blk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_vis_scan<<<1, 1024, 0, st>>>(blk, nb);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_vis_scatter<<<nb, 256, 0, st>>>(mask, uv, n, blk, vis_gid, vis_uv);
  return cudaGetLastError();
}

}  // namespace gsr
