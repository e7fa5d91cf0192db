// Dense PnP + RANSAC on rendered depth (Sec. 3.4, Eq. 10), declared in
// include/gsr_pnp.h:
//   1. lifting: every match whose rendered pixel has alpha >= min_alpha gets
//      the world point R_r^T (z K^-1 (x + .5, y + .5, 1) - t_r), z = depth /
//      alpha (fp64), compacted in match order;
//   2. hypotheses: one thread per RANSAC sample solves P3P in fp64 (Grunert's
//      quartic in v = s3 / s1, Ferrari's closed form polished by Newton,
//      triad absolute orientation);
//   3. scoring: every solution against every lifted match, packed fp32
//      (__ffma2_rn on pairs of matches), inlier counts per solution;
//   4. the RANSAC argmax (most inliers, lowest index on ties);
//   5. Gauss-Newton: per-match J^T J, J^T r of the current inliers in fp32,
//      per-block sums in a fixed order, an fp64 6x6 Cholesky solve and the left
//      update T <- Exp(xi) T on the device;
//   6. the inlier mask and count of the refined pose.
// Everything after the argument checks is asynchronous on the caller's
// stream; one read-back of the solver state ends the call.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>

#include "gsr_pnp.h"

namespace gsr {
void set_last_error(const std::string& msg);
}

namespace {

constexpr int kThreads = 256;
constexpr int kCompact = 2048;    // matches per compaction block (8 per thread)
constexpr int kSol = 4;           // P3P solutions per hypothesis, at most
constexpr int kPose = 12;         // (R row-major, t)
constexpr int kRow = 4;           // matches per thread in the scoring kernel
constexpr int kScorePoses = 128;  // solutions staged per scoring CTA
constexpr int kGnVals = 29;       // J^T J upper triangle (21), J^T r (6), inlier count, squared error
constexpr int kGnBlocks = 304;    // accumulation blocks (fixed, so the summation order is fixed)

struct Cam {
  double fx, fy, cx, cy;
  double ifx, ify;  // 1 / fx, 1 / fy
  int W, H;
};

struct Pose12 {
  double v[kPose];
};

// Device-resident solver state (read back once at the end of a call).
struct State {
  double T[kPose];       // current pose
  int active;            // refinement continues
  int steps;             // Gauss-Newton updates taken
  int best_h, best_s;
  long long best_count;
  unsigned int n_valid;
  unsigned int n_inliers;
  unsigned int bad_pixel;
  unsigned int pad;
};

// ------------------------------------------------------------------ lifting
__device__ __forceinline__ bool match_valid(const int32_t* __restrict__ m, long long i, const float* __restrict__ alpha,
                                            int npix, float min_alpha, bool* bad) {
  const int q = m[3 * i + 1], r = m[3 * i + 2];
  if (q < 0 || q >= npix || r < 0 || r >= npix) {
    *bad = true;
    return false;
  }
  *bad = false;
  return alpha[r] >= min_alpha;
}

__global__ void __launch_bounds__(kThreads) k_pnp_flags(const int32_t* __restrict__ m, long long n,
                                                        const float* __restrict__ alpha, int npix, float min_alpha,
                                                        unsigned* __restrict__ blk, State* __restrict__ st) {
  __shared__ unsigned s_w[kThreads / 32];
  const long long base = (long long)blockIdx.x * kCompact;
  unsigned c = 0, nbad = 0;
  for (int k = 0; k < kCompact / kThreads; ++k) {
    const long long i = base + k * kThreads + threadIdx.x;
    if (i < n) {
      bool bad;
      c += match_valid(m, i, alpha, npix, min_alpha, &bad) ? 1u : 0u;
      nbad += bad ? 1u : 0u;
    }
  }
  c = __reduce_add_sync(0xffffffffu, c);
  nbad = __reduce_add_sync(0xffffffffu, nbad);
  if ((threadIdx.x & 31) == 0) {
    s_w[threadIdx.x >> 5] = c;
    if (nbad) atomicAdd(&st->bad_pixel, nbad);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int k = 0; k < kThreads / 32; ++k) t += s_w[k];
    blk[blockIdx.x] = t;
  }
}

// exclusive scan of nb block counts in place; the total is the valid count
__global__ void __launch_bounds__(1024) k_pnp_scan(unsigned* __restrict__ blk, int nb, State* __restrict__ st) {
  __shared__ unsigned s_w[32];
  __shared__ unsigned s_carry;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nb; b0 += 1024) {
    const int i = b0 + tid;
    const unsigned x = i < nb ? blk[i] : 0u;
    unsigned inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      unsigned t = s_w[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      s_w[lane] = t;
    }
    __syncthreads();
    const unsigned carry = s_carry;
    if (i < nb) blk[i] = carry + (wid ? s_w[wid - 1] : 0u) + inc - x;
    __syncthreads();
    if (tid == 0) s_carry = carry + s_w[31];
    __syncthreads();
  }
  if (tid == 0) st->n_valid = s_carry;
}

__global__ void __launch_bounds__(kThreads) k_pnp_lift(const int32_t* __restrict__ m, long long n,
                                                       const float* __restrict__ depth,
                                                       const float* __restrict__ alpha, Cam cam, Pose12 Tr,
                                                       float min_alpha, const unsigned* __restrict__ blk,
                                                       double* __restrict__ X64, float4* __restrict__ X32,
                                                       float2* __restrict__ nab, float2* __restrict__ pix,
                                                       int32_t* __restrict__ vidx) {
  __shared__ unsigned s_w[kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long base = (long long)blockIdx.x * kCompact;
  const int npix = cam.W * cam.H;
  unsigned off = blk[blockIdx.x];
  for (int k = 0; k < kCompact / kThreads; ++k) {
    const long long i = base + k * kThreads + threadIdx.x;
    bool bad = false;
    const bool v = i < n && match_valid(m, i, alpha, npix, min_alpha, &bad);
    const unsigned b = __ballot_sync(0xffffffffu, v);
    if (lane == 0) s_w[wid] = (unsigned)__popc(b);
    __syncthreads();
    unsigned before = 0, total = 0;
#pragma unroll
    for (int q = 0; q < kThreads / 32; ++q) {
      before += q < wid ? s_w[q] : 0u;
      total += s_w[q];
    }
    if (v) {
      const unsigned o = off + before + (unsigned)__popc(b & ((1u << lane) - 1u));
      const int qp = m[3 * i + 1], rp = m[3 * i + 2];
      // z = depth / alpha in fp64 without a division: the binary32 reciprocal
      // refined by one Newton step (48 bits), then one correction of the quotient
      const double A = alpha[rp], D = depth[rp];
      double rcp = (double)(1.0f / alpha[rp]);
      rcp = rcp * (2.0 - A * rcp);
      double z = D * rcp;
      z = fma(rcp, fma(-z, A, D), z);
      const double xc = z * (((double)(rp % cam.W) + 0.5 - cam.cx) * cam.ifx);
      const double yc = z * (((double)(rp / cam.W) + 0.5 - cam.cy) * cam.ify);
      const double d0 = xc - Tr.v[9], d1 = yc - Tr.v[10], d2 = z - Tr.v[11];
      const double* R = Tr.v;
      const double X = R[0] * d0 + R[3] * d1 + R[6] * d2;  // R^T d
      const double Y = R[1] * d0 + R[4] * d1 + R[7] * d2;
      const double Z = R[2] * d0 + R[5] * d1 + R[8] * d2;
      X64[3 * (size_t)o] = X;
      X64[3 * (size_t)o + 1] = Y;
      X64[3 * (size_t)o + 2] = Z;
      X32[o] = make_float4((float)X, (float)Y, (float)Z, 0.0f);
      const double px = (double)(qp % cam.W) + 0.5, py = (double)(qp / cam.W) + 0.5;
      pix[o] = make_float2((float)px, (float)py);
      nab[o] = make_float2((float)(-(px - cam.cx) * cam.ifx), (float)(-(py - cam.cy) * cam.ify));
      vidx[o] = (int32_t)i;
    }
    off += total;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ P3P (fp64)
// Real roots of the monic quartic x^4 + a x^3 + b x^2 + c x + d by Ferrari's
// method in fp64: with x = y - a/4 the depressed quartic y^4 + p y^2 + q y + r
// equals (y^2 + m)^2 - (s y - q / (2 s))^2, s^2 = 2 m - p, for the largest root
// m of the resolvent cubic 8 m^3 - 4 p m^2 - 8 r m + 4 p r - q^2 (Cardano or the
// trigonometric form, then Newton-polished); y solves y^2 +- s y + m -+ q/(2 s)
// = 0 (for q = 0: y^2 = the roots of z^2 + p z + r). The closed form runs in a
// few hundred fp64 operations, against thousands for bracketing: fp64 is slow
// on this part. Each real root is then polished by two Newton steps on the
// original quartic. Returns the count; roots ascending.
__device__ int quartic_real_roots(const double* q4, double* out) {
  const double a = q4[3] / q4[4], b = q4[2] / q4[4], c = q4[1] / q4[4], d = q4[0] / q4[4];
  const double a2 = a * a;
  const double p = b - 0.375 * a2;
  const double q = c - 0.5 * a * b + 0.125 * a2 * a;
  const double r = d - 0.25 * a * c + 0.0625 * a2 * b - (3.0 / 256.0) * a2 * a2;
  // resolvent m^3 + A m^2 + B m + C, A = -p/2, B = -r, C = (4 p r - q^2) / 8
  const double A = -0.5 * p, B = -r, C = 0.125 * (4.0 * p * r - q * q);
  const double P3 = B - A * A / 3.0, Q3 = 2.0 * A * A * A / 27.0 - A * B / 3.0 + C;
  const double disc = 0.25 * Q3 * Q3 + P3 * P3 * P3 / 27.0;
  double t;
  if (disc > 0.0) {  // one real root
    const double sq = sqrt(disc);
    const double u = cbrt(-0.5 * Q3 - copysign(sq, Q3));
    t = (u != 0.0) ? u - P3 / (3.0 * u) : 0.0;
  } else {  // three real roots: the largest
    const double rr = sqrt(fmax(-P3 / 3.0, 0.0));
    double ca = (rr > 0.0) ? -0.5 * Q3 / (rr * rr * rr) : 0.0;
    ca = fmin(1.0, fmax(-1.0, ca));
    t = 2.0 * rr * cos(acos(ca) / 3.0);
  }
  double m = t - A / 3.0;
  for (int it = 0; it < 2; ++it) {  // polish on the resolvent
    const double f = ((m + A) * m + B) * m + C, df = (3.0 * m + 2.0 * A) * m + B;
    if (df != 0.0) m -= f / df;
  }
  double y[4];
  int ny = 0;
  const double s2 = 2.0 * m - p;
  if (s2 > 1e-14 * (fabs(p) + fabs(m) + 1e-300)) {
    const double s = sqrt(s2), h = q / (2.0 * s);
    const double d1 = s2 - 4.0 * (m - h), d2 = s2 - 4.0 * (m + h);
    if (d1 >= 0.0) {
      const double e = sqrt(d1);
      y[ny++] = 0.5 * (-s - e);
      y[ny++] = 0.5 * (-s + e);
    }
    if (d2 >= 0.0) {
      const double e = sqrt(d2);
      y[ny++] = 0.5 * (s - e);
      y[ny++] = 0.5 * (s + e);
    }
  } else {  // biquadratic
    const double dz = p * p - 4.0 * r;
    if (dz >= 0.0) {
      const double e = sqrt(dz);
      const double z1 = 0.5 * (-p - e), z2 = 0.5 * (-p + e);
      for (double z : {z1, z2})
        if (z >= 0.0) {
          const double w = sqrt(z);
          y[ny++] = -w;
          y[ny++] = w;
        }
    }
  }
  int n = 0;
  for (int k = 0; k < ny; ++k) {
    double x = y[k] - 0.25 * a;
    for (int it = 0; it < 2; ++it) {
      const double f = (((x + a) * x + b) * x + c) * x + d;
      const double df = ((4.0 * x + 3.0 * a) * x + 2.0 * b) * x + c;
      if (df != 0.0) x -= f / df;
    }
    out[n++] = x;
  }
  for (int i = 1; i < n; ++i)  // ascending (insertion sort, n <= 4)
    for (int j = i; j > 0 && out[j - 1] > out[j]; --j) {
      const double tmp = out[j];
      out[j] = out[j - 1];
      out[j - 1] = tmp;
    }
  return n;
}

__device__ void frame3(const double* P0, const double* P1, const double* P2, double F[3][3], bool* ok) {
  double e1[3] = {P1[0] - P0[0], P1[1] - P0[1], P1[2] - P0[2]};
  const double f[3] = {P2[0] - P0[0], P2[1] - P0[1], P2[2] - P0[2]};
  double n[3] = {e1[1] * f[2] - e1[2] * f[1], e1[2] * f[0] - e1[0] * f[2], e1[0] * f[1] - e1[1] * f[0]};
  const double le = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  const double ln = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  *ok = le > 0.0 && ln > 0.0;
  for (int k = 0; k < 3; ++k) {
    e1[k] /= le;
    n[k] /= ln;
  }
  const double e2[3] = {n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2], n[0] * e1[1] - n[1] * e1[0]};
  for (int r = 0; r < 3; ++r) {  // columns e1, e2, n
    F[r][0] = e1[r];
    F[r][1] = e2[r];
    F[r][2] = n[r];
  }
}

__global__ void __launch_bounds__(32) k_pnp_p3p(const double* __restrict__ X64, const float2* __restrict__ pix,
                                                 const State* __restrict__ st, const uint32_t* __restrict__ words,
                                                 int n_hyp, Cam cam, double* __restrict__ poses64,
                                                 float4* __restrict__ poses32, int* __restrict__ counts) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= n_hyp) return;
#pragma unroll
  for (int s = 0; s < kSol; ++s) counts[kSol * h + s] = -1;
  const unsigned long long K = st->n_valid;
  if (K < 3) return;
  int idx[3];
  for (int k = 0; k < 3; ++k) idx[k] = (int)(((unsigned long long)words[3 * h + k] * K) >> 32);
  if (idx[0] == idx[1] || idx[0] == idx[2] || idx[1] == idx[2]) return;
  double X[3][3], f[3][3];
  for (int k = 0; k < 3; ++k) {
    for (int a = 0; a < 3; ++a) X[k][a] = X64[3 * (size_t)idx[k] + a];
    const float2 p = pix[idx[k]];
    const double bx = ((double)p.x - cam.cx) / cam.fx, by = ((double)p.y - cam.cy) / cam.fy;
    const double nb = sqrt(bx * bx + by * by + 1.0);
    f[k][0] = bx / nb;
    f[k][1] = by / nb;
    f[k][2] = 1.0 / nb;
  }
  auto d2 = [&](int i, int j) {
    const double a = X[i][0] - X[j][0], b = X[i][1] - X[j][1], c = X[i][2] - X[j][2];
    return a * a + b * b + c * c;
  };
  const double a2 = d2(1, 2), b2 = d2(0, 2), c2 = d2(0, 1);
  if (!(a2 > 0.0 && b2 > 0.0 && c2 > 0.0)) return;
  {  // collinear world points
    const double u[3] = {X[1][0] - X[0][0], X[1][1] - X[0][1], X[1][2] - X[0][2]};
    const double w[3] = {X[2][0] - X[0][0], X[2][1] - X[0][1], X[2][2] - X[0][2]};
    const double cx = u[1] * w[2] - u[2] * w[1], cy = u[2] * w[0] - u[0] * w[2], cz = u[0] * w[1] - u[1] * w[0];
    if (sqrt(cx * cx + cy * cy + cz * cz) <= 1e-12 * (a2 + b2 + c2)) return;
  }
  const double ca = f[1][0] * f[2][0] + f[1][1] * f[2][1] + f[1][2] * f[2][2];
  const double cb = f[0][0] * f[2][0] + f[0][1] * f[2][1] + f[0][2] * f[2][2];
  const double cg = f[0][0] * f[1][0] + f[0][1] * f[1][1] + f[0][2] * f[1][2];
  const double k = (a2 - c2) / b2, cr = c2 / b2;
  // D = cg - ca v, N = (1 + k) - 2 k cb v + (k - 1) v^2, E = (1 - cr) + 2 cr cb v - cr v^2;
  // Q = 4 D^2 E + N^2 - 4 cg N D
  const double D[2] = {cg, -ca};
  const double N[3] = {1.0 + k, -2.0 * k * cb, k - 1.0};
  const double E[3] = {1.0 - cr, 2.0 * cr * cb, -cr};
  double D2[3] = {D[0] * D[0], 2.0 * D[0] * D[1], D[1] * D[1]};
  double Q[5] = {0, 0, 0, 0, 0};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Q[i + j] += 4.0 * D2[i] * E[j] + N[i] * N[j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 2; ++j) Q[i + j] -= 4.0 * cg * N[i] * D[j];
  if (Q[4] == 0.0) return;
  double roots[4];
  const int nr = quartic_real_roots(Q, roots);
  int ns = 0;
  double FX[3][3];
  bool okx;
  frame3(X[0], X[1], X[2], FX, &okx);
  if (!okx) return;
  for (int r = 0; r < nr && ns < kSol; ++r) {
    const double v = roots[r];
    if (!(v > 0.0)) continue;
    const double Dv = D[0] + D[1] * v;
    if (Dv == 0.0) continue;
    const double u = (N[0] + v * (N[1] + v * N[2])) / (2.0 * Dv);
    if (!(u > 0.0)) continue;
    const double s1 = sqrt(b2 / (1.0 + v * v - 2.0 * v * cb));
    const double s[3] = {s1, u * s1, v * s1};
    double Qc[3][3];
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < 3; ++a) Qc[i][a] = s[i] * f[i][a];
    double FQ[3][3];
    bool okq;
    frame3(Qc[0], Qc[1], Qc[2], FQ, &okq);
    if (!okq) continue;
    double R[9], t[3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) R[3 * i + j] = FQ[i][0] * FX[j][0] + FQ[i][1] * FX[j][1] + FQ[i][2] * FX[j][2];
    for (int i = 0; i < 3; ++i)
      t[i] = Qc[0][i] - (R[3 * i] * X[0][0] + R[3 * i + 1] * X[0][1] + R[3 * i + 2] * X[0][2]);
    double* o = poses64 + ((size_t)kSol * h + ns) * kPose;
    for (int q = 0; q < 9; ++q) o[q] = R[q];
    for (int q = 0; q < 3; ++q) o[9 + q] = t[q];
    float4* o32 = poses32 + ((size_t)kSol * h + ns) * 3;
    for (int i = 0; i < 3; ++i) o32[i] = make_float4((float)R[3 * i], (float)R[3 * i + 1], (float)R[3 * i + 2], (float)t[i]);
    counts[kSol * h + ns] = 0;
    ++ns;
  }
}

// ------------------------------------------------------------------ scoring (fp32, packed pairs)
__device__ __forceinline__ unsigned inl2(float2 px, float2 py, float2 pz, float2 na, float2 nb, float2 FX,
                                         float2 FY, float2 TA, float2 NTA, bool v0, bool v1) {
  const float2 du = __ffma2_rn(na, pz, px);  // x - a z
  const float2 dv = __ffma2_rn(nb, pz, py);
  const float2 fu = __fmul2_rn(FX, du), fv = __fmul2_rn(FY, dv);
  const float2 e2 = __ffma2_rn(fu, fu, __fmul2_rn(fv, fv));  // (|e| z)^2
  const float2 diff = __ffma2_rn(__fmul2_rn(TA, pz), __fmul2_rn(NTA, pz), e2);  // (|e| z)^2 - (tau z)^2
  return ((v0 && pz.x > 0.0f && diff.x < 0.0f) ? 1u : 0u) + ((v1 && pz.y > 0.0f && diff.y < 0.0f) ? 1u : 0u);
}

__device__ __forceinline__ void cam_pair(float4 r, float2 x, float2 y, float2 z, float2& out) {
  out = __ffma2_rn(make_float2(r.x, r.x), x,
                   __ffma2_rn(make_float2(r.y, r.y), y, __ffma2_rn(make_float2(r.z, r.z), z, make_float2(r.w, r.w))));
}

__global__ void __launch_bounds__(kThreads) k_pnp_score(const float4* __restrict__ X32, const float2* __restrict__ nab,
                                                        const State* __restrict__ st,
                                                        const float4* __restrict__ poses32, int* __restrict__ counts,
                                                        int n_poses, float fx, float fy, float tau) {
  __shared__ float4 sp[kScorePoses][3];
  __shared__ int sc[kScorePoses];
  __shared__ int sok[kScorePoses];
  const int p0 = blockIdx.y * kScorePoses;
  const int np = min(kScorePoses, n_poses - p0);
  for (int i = threadIdx.x; i < np; i += kThreads) {
    sok[i] = counts[p0 + i] >= 0;
    sc[i] = 0;
    for (int r = 0; r < 3; ++r) sp[i][r] = poses32[(size_t)(p0 + i) * 3 + r];
  }
  __syncthreads();
  const unsigned K = st->n_valid;
  const size_t base = (size_t)blockIdx.x * kThreads * kRow + threadIdx.x;
  float4 Xm[kRow];
  float2 ab[kRow];
  bool v[kRow];
#pragma unroll
  for (int j = 0; j < kRow; ++j) {
    const size_t i = base + (size_t)j * kThreads;
    v[j] = i < K;
    Xm[j] = v[j] ? X32[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    ab[j] = v[j] ? nab[i] : make_float2(0.f, 0.f);
  }
  const float2 xA = make_float2(Xm[0].x, Xm[1].x), yA = make_float2(Xm[0].y, Xm[1].y), zA = make_float2(Xm[0].z, Xm[1].z);
  const float2 xB = make_float2(Xm[2].x, Xm[3].x), yB = make_float2(Xm[2].y, Xm[3].y), zB = make_float2(Xm[2].z, Xm[3].z);
  const float2 naA = make_float2(ab[0].x, ab[1].x), nbA = make_float2(ab[0].y, ab[1].y);
  const float2 naB = make_float2(ab[2].x, ab[3].x), nbB = make_float2(ab[2].y, ab[3].y);
  const float2 FX = make_float2(fx, fx), FY = make_float2(fy, fy), TA = make_float2(tau, tau),
               NTA = make_float2(-tau, -tau);
  const bool any = __any_sync(0xffffffffu, v[0]);
  if (any) {
    for (int pi = 0; pi < np; ++pi) {
      if (!sok[pi]) continue;
      const float4 r0 = sp[pi][0], r1 = sp[pi][1], r2 = sp[pi][2];
      float2 px, py, pz;
      cam_pair(r0, xA, yA, zA, px);
      cam_pair(r1, xA, yA, zA, py);
      cam_pair(r2, xA, yA, zA, pz);
      unsigned c = inl2(px, py, pz, naA, nbA, FX, FY, TA, NTA, v[0], v[1]);
      cam_pair(r0, xB, yB, zB, px);
      cam_pair(r1, xB, yB, zB, py);
      cam_pair(r2, xB, yB, zB, pz);
      c += inl2(px, py, pz, naB, nbB, FX, FY, TA, NTA, v[2], v[3]);
      c = __reduce_add_sync(0xffffffffu, c);
      if ((threadIdx.x & 31) == 0 && c) atomicAdd(&sc[pi], (int)c);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < np; i += kThreads)
    if (sok[i] && sc[i]) atomicAdd(&counts[p0 + i], sc[i]);
}

// ------------------------------------------------------------------ RANSAC argmax
__global__ void __launch_bounds__(1024) k_pnp_best(const int* __restrict__ counts, int n_poses,
                                                   const double* __restrict__ poses64, Pose12 Tr,
                                                   State* __restrict__ st) {
  __shared__ int s_c[32], s_i[32];
  int bc = -1, bi = 0x7fffffff;
  for (int i = threadIdx.x; i < n_poses; i += 1024) {
    const int c = counts[i];
    if (c > bc) {  // ascending i per thread: the first maximum is kept
      bc = c;
      bi = i;
    }
  }
  auto better = [](int c1, int i1, int c2, int i2) { return c1 > c2 || (c1 == c2 && i1 < i2); };
  for (int o = 16; o > 0; o >>= 1) {
    const int oc = __shfl_xor_sync(0xffffffffu, bc, o), oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (better(oc, oi, bc, bi)) {
      bc = oc;
      bi = oi;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    s_c[threadIdx.x >> 5] = bc;
    s_i[threadIdx.x >> 5] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 32; ++w)
      if (better(s_c[w], s_i[w], bc, bi)) {
        bc = s_c[w];
        bi = s_i[w];
      }
    if (bc >= 0) {
      st->best_h = bi / kSol;
      st->best_s = bi % kSol;
      st->best_count = bc;
      for (int q = 0; q < kPose; ++q) st->T[q] = poses64[(size_t)bi * kPose + q];
      st->active = 1;
    } else {
      st->best_h = -1;
      st->best_s = -1;
      st->best_count = 0;
      for (int q = 0; q < kPose; ++q) st->T[q] = Tr.v[q];
      st->active = 0;
    }
    st->steps = 0;
  }
}

// ------------------------------------------------------------------ Gauss-Newton
__device__ __forceinline__ void load_pose32(const State* st, float R[9], float t[3]) {
  for (int q = 0; q < 9; ++q) R[q] = (float)st->T[q];
  for (int q = 0; q < 3; ++q) t[q] = (float)st->T[9 + q];
}

__global__ void __launch_bounds__(kThreads) k_pnp_gn(const float4* __restrict__ X32, const float2* __restrict__ nab,
                                                     const State* __restrict__ st, double* __restrict__ partials,
                                                     float fx, float fy, float tau) {
  __shared__ float s_red[kThreads / 32][kGnVals];
  if (!st->active) return;  // uniform: every block reads the same flag
  float R[9], t[3];
  load_pose32(st, R, t);
  float acc[kGnVals];
#pragma unroll
  for (int k = 0; k < kGnVals; ++k) acc[k] = 0.0f;
  const unsigned K = st->n_valid;
  for (unsigned i = blockIdx.x * kThreads + threadIdx.x; i < K; i += gridDim.x * kThreads) {
    const float4 X = X32[i];
    const float2 ab = nab[i];
    const float x = fmaf(R[0], X.x, fmaf(R[1], X.y, fmaf(R[2], X.z, t[0])));
    const float y = fmaf(R[3], X.x, fmaf(R[4], X.y, fmaf(R[5], X.z, t[1])));
    const float z = fmaf(R[6], X.x, fmaf(R[7], X.y, fmaf(R[8], X.z, t[2])));
    const float du = fmaf(ab.x, z, x), dv = fmaf(ab.y, z, y);
    const float fu = fx * du, fv = fy * dv;
    const float e2 = fmaf(fu, fu, fv * fv);
    const float diff = fmaf(tau * z, -tau * z, e2);
    if (!(z > 0.0f && diff < 0.0f)) continue;
    const float iz = 1.0f / z;
    const float ru = fu * iz, rv = fv * iz;  // (u - px, v - py)
    const float a0 = fx * iz, a2 = -fx * x * iz * iz;
    const float b1 = fy * iz, b2 = -fy * y * iz * iz;
    const float Ju[6] = {a0, 0.0f, a2, a2 * y, a0 * z - a2 * x, -a0 * y};
    const float Jv[6] = {0.0f, b1, b2, b2 * y - b1 * z, -b2 * x, b1 * x};
    int q = 0;
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
      for (int c = r; c < 6; ++c) acc[q++] += Ju[r] * Ju[c] + Jv[r] * Jv[c];
#pragma unroll
    for (int r = 0; r < 6; ++r) acc[21 + r] += Ju[r] * ru + Jv[r] * rv;
    acc[27] += 1.0f;
    acc[28] += ru * ru + rv * rv;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kGnVals; ++k) {
    float s = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) s_red[wid][k] = s;
  }
  __syncthreads();
  if (threadIdx.x < kGnVals) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += (double)s_red[w][threadIdx.x];
    partials[(size_t)blockIdx.x * kGnVals + threadIdx.x] = s;
  }
}

// Left update T <- Exp(xi) T (Rodrigues; V = I + b [phi]x + c [phi]x^2 on rho).
__device__ void se3_left(const double xi[6], double T[kPose]) {
  const double* w = xi + 3;
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  const double th = sqrt(t2);
  double a, b, c;
  if (th < 0.05) {  // Maclaurin series of sin t / t, (1 - cos t) / t^2, (t - sin t) / t^3 to t^8 (< 1e-20 left)
    a = 1.0 + t2 * (-1.0 / 6 + t2 * (1.0 / 120 + t2 * (-1.0 / 5040 + t2 * (1.0 / 362880))));
    b = 0.5 + t2 * (-1.0 / 24 + t2 * (1.0 / 720 + t2 * (-1.0 / 40320 + t2 * (1.0 / 3628800))));
    c = 1.0 / 6 + t2 * (-1.0 / 120 + t2 * (1.0 / 5040 + t2 * (-1.0 / 362880 + t2 * (1.0 / 39916800))));
  } else {
    double sn, cs;
    sincos(th, &sn, &cs);
    a = sn / th;
    b = (1.0 - cs) / t2;
    c = (th - sn) / (t2 * th);
  }
  const double Kx[3][3] = {{0.0, -w[2], w[1]}, {w[2], 0.0, -w[0]}, {-w[1], w[0], 0.0}};
  double E[3][3], V[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double k2 = Kx[i][0] * Kx[0][j] + Kx[i][1] * Kx[1][j] + Kx[i][2] * Kx[2][j];
      const double id = i == j ? 1.0 : 0.0;
      E[i][j] = id + a * Kx[i][j] + b * k2;
      V[i][j] = id + b * Kx[i][j] + c * k2;
    }
  double R[9], t[3];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) R[3 * i + j] = E[i][0] * T[j] + E[i][1] * T[3 + j] + E[i][2] * T[6 + j];
    t[i] = E[i][0] * T[9] + E[i][1] * T[10] + E[i][2] * T[11] + V[i][0] * xi[0] + V[i][1] * xi[1] + V[i][2] * xi[2];
  }
  for (int q = 0; q < 9; ++q) T[q] = R[q];
  for (int q = 0; q < 3; ++q) T[9 + q] = t[q];
}

constexpr int kSolveParts = 8;  // partial sums per component in the solve kernel

__global__ void __launch_bounds__(kGnVals * kSolveParts) k_pnp_gn_solve(const double* __restrict__ partials,
                                                                         State* __restrict__ st) {
  __shared__ double part[kGnVals][kSolveParts];
  __shared__ double s[kGnVals];
  if (!st->active) return;
  {  // component k, blocks j, j + 8, ... in order; then the 8 parts in order
    const int k = threadIdx.x / kSolveParts, j = threadIdx.x % kSolveParts;
    double a = 0.0;
    for (int b = j; b < kGnBlocks; b += kSolveParts) a += partials[(size_t)b * kGnVals + k];
    part[k][j] = a;
  }
  __syncthreads();
  if (threadIdx.x < kGnVals) {
    double a = 0.0;
    for (int j = 0; j < kSolveParts; ++j) a += part[threadIdx.x][j];
    s[threadIdx.x] = a;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  if (s[27] < 3.0) {
    st->active = 0;
    return;
  }
  double H[6][6], L[6][6] = {};
  int q = 0;
  for (int r = 0; r < 6; ++r)
    for (int c = r; c < 6; ++c) {
      H[r][c] = s[q];
      H[c][r] = s[q];
      ++q;
    }
  // Cholesky H = L L^T with the reciprocal diagonal: one reciprocal square
  // root per column and multiplications (fp64 division is a long sequence here)
  double inv[6];
  for (int j = 0; j < 6; ++j) {
    double d = H[j][j];
    for (int m = 0; m < j; ++m) d -= L[j][m] * L[j][m];
    if (!(d > 0.0)) {
      st->active = 0;
      return;
    }
    inv[j] = rsqrt(d);
    L[j][j] = d * inv[j];
    for (int i = j + 1; i < 6; ++i) {
      double e = H[i][j];
      for (int m = 0; m < j; ++m) e -= L[i][m] * L[j][m];
      L[i][j] = e * inv[j];
    }
  }
  double y[6], xi[6];
  for (int i = 0; i < 6; ++i) {  // L y = -g
    double e = -s[21 + i];
    for (int m = 0; m < i; ++m) e -= L[i][m] * y[m];
    y[i] = e * inv[i];
  }
  for (int i = 5; i >= 0; --i) {  // L^T xi = y
    double e = y[i];
    for (int m = i + 1; m < 6; ++m) e -= L[m][i] * xi[m];
    xi[i] = e * inv[i];
  }
  double T[kPose];
  for (int p = 0; p < kPose; ++p) T[p] = st->T[p];
  se3_left(xi, T);
  for (int p = 0; p < kPose; ++p) st->T[p] = T[p];
  st->steps += 1;
}

// ------------------------------------------------------------------ final inliers
__global__ void __launch_bounds__(kThreads) k_pnp_final(const float4* __restrict__ X32, const float2* __restrict__ nab,
                                                        const int32_t* __restrict__ vidx, State* __restrict__ st,
                                                        uint8_t* __restrict__ mask, float fx, float fy, float tau) {
  float R[9], t[3];
  load_pose32(st, R, t);
  const unsigned K = st->n_valid;
  unsigned cnt = 0;
  for (unsigned i = blockIdx.x * kThreads + threadIdx.x; i < K; i += gridDim.x * kThreads) {
    const float4 X = X32[i];
    const float2 ab = nab[i];
    const float x = fmaf(R[0], X.x, fmaf(R[1], X.y, fmaf(R[2], X.z, t[0])));
    const float y = fmaf(R[3], X.x, fmaf(R[4], X.y, fmaf(R[5], X.z, t[1])));
    const float z = fmaf(R[6], X.x, fmaf(R[7], X.y, fmaf(R[8], X.z, t[2])));
    const float du = fmaf(ab.x, z, x), dv = fmaf(ab.y, z, y);
    const float fu = fx * du, fv = fy * dv;
    const float diff = fmaf(tau * z, -tau * z, fmaf(fu, fu, fv * fv));
    if (z > 0.0f && diff < 0.0f) {
      mask[vidx[i]] = 1;
      ++cnt;
    }
  }
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&st->n_inliers, cnt);
}

struct DevBuf {
  void* p = nullptr;
};

}  // namespace

struct gs_pnp {
  int device = 0;
  int sm_count = 1;
  long long max_matches = 0;
  int max_hyp = 0;
  unsigned* blk = nullptr;
  double* X64 = nullptr;
  float4* X32 = nullptr;
  float2* nab = nullptr;
  float2* pix = nullptr;
  int32_t* vidx = nullptr;
  uint8_t* mask = nullptr;
  double* poses64 = nullptr;
  float4* poses32 = nullptr;
  int* counts = nullptr;
  double* partials = nullptr;
  State* st = nullptr;
  State* st_host = nullptr;
  // phase timing (gs_pnp_set_timing): events around lift, P3P, scoring, argmax,
  // refinement and the final inlier pass
  bool timing = false;
  cudaEvent_t ev[GS_PNP_PHASES + 1] = {};
  double kt_ms[GS_PNP_PHASES] = {};
  int64_t kt_n = 0;
};

namespace {

gs_status pnp_fail(gs_status s, const std::string& msg) {
  gsr::set_last_error(msg);
  return s;
}

#define PNP_CUDA(x)                                                                                   \
  do {                                                                                                \
    const cudaError_t e_ = (x);                                                                       \
    if (e_ != cudaSuccess) return pnp_fail(GS_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

extern "C" {

gs_status gs_pnp_set_timing(gs_pnp* s, int enable) {
  gsr::set_last_error("");
  if (!s) return pnp_fail(GS_ERR_INVALID_ARG, "solver is NULL");
  PNP_CUDA(cudaSetDevice(s->device));
  if (enable)
    for (cudaEvent_t& e : s->ev)
      if (!e) PNP_CUDA(cudaEventCreate(&e));
  s->timing = enable != 0;
  return GS_OK;
}

gs_status gs_pnp_phase_times(gs_pnp* s, double* total_ms, int64_t* calls) {
  gsr::set_last_error("");
  if (!s || !total_ms) return pnp_fail(GS_ERR_INVALID_ARG, "solver and total_ms are required");
  for (int k = 0; k < GS_PNP_PHASES; ++k) {
    total_ms[k] = s->kt_ms[k];
    s->kt_ms[k] = 0.0;
  }
  if (calls) *calls = s->kt_n;
  s->kt_n = 0;
  return GS_OK;
}

gs_pnp_opts gs_pnp_defaults(void) {
  gs_pnp_opts o;
  o.tau_px = 2.0f;
  o.min_alpha = 0.5f;
  o.refine_iters = 5;
  return o;
}

void gs_pnp_destroy(gs_pnp* s) {
  if (!s) return;
  cudaSetDevice(s->device);
  cudaDeviceSynchronize();
  for (void* p : {(void*)s->blk, (void*)s->X64, (void*)s->X32, (void*)s->nab, (void*)s->pix, (void*)s->vidx,
                  (void*)s->mask, (void*)s->poses64, (void*)s->poses32, (void*)s->counts, (void*)s->partials,
                  (void*)s->st})
    if (p) cudaFree(p);
  if (s->st_host) cudaFreeHost(s->st_host);
  for (cudaEvent_t e : s->ev)
    if (e) cudaEventDestroy(e);
  delete s;
}

gs_status gs_pnp_create(int64_t max_matches, int max_hypotheses, gs_pnp** out) {
  gsr::set_last_error("");
  if (!out) return pnp_fail(GS_ERR_INVALID_ARG, "out is required");
  *out = nullptr;
  if (max_matches < 1 || max_matches > (1ll << 30))
    return pnp_fail(GS_ERR_INVALID_ARG, "max_matches must be in [1, 2^30]");
  if (max_hypotheses < 1 || max_hypotheses > 65536)
    return pnp_fail(GS_ERR_INVALID_ARG, "max_hypotheses must be in [1, 65536]");
  gs_pnp* s = new gs_pnp();
  s->max_matches = max_matches;
  s->max_hyp = max_hypotheses;
  auto bail = [&](cudaError_t e) {
    cudaGetLastError();
    gs_pnp_destroy(s);
    return pnp_fail(e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA,
                    std::string("gs_pnp_create: ") + cudaGetErrorString(e));
  };
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) return bail(e);
  cudaDeviceProp prop;
  if ((e = cudaGetDeviceProperties(&prop, s->device)) != cudaSuccess) return bail(e);
  s->sm_count = prop.multiProcessorCount;
  const size_t n = (size_t)max_matches, H = (size_t)max_hypotheses;
  const size_t nb = n / kCompact + 1;
  if ((e = cudaMalloc(&s->blk, nb * sizeof(unsigned))) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&s->X64, 3 * n * sizeof(double))) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&s->X32, n * sizeof(float4))) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&s->nab, n * sizeof(float2))) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&s->pix, n * sizeof(float2))) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&s->vidx, n * sizeof(int32_t))) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&s->mask, n)) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&s->poses64, H * kSol * kPose * sizeof(double))) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&s->poses32, H * kSol * 3 * sizeof(float4))) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&s->counts, H * kSol * sizeof(int))) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&s->partials, (size_t)kGnBlocks * kGnVals * sizeof(double))) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&s->st, sizeof(State))) != cudaSuccess) return bail(e);
  if ((e = cudaMallocHost(&s->st_host, sizeof(State))) != cudaSuccess) return bail(e);
  *out = s;
  return GS_OK;
}

gs_status gs_pnp_solve(gs_pnp* s, const gs_camera* cam, const gs_pose* T_render, const float* depth,
                       const float* alpha, const int32_t* matches, int64_t n_matches, const uint32_t* words,
                       int n_hypotheses, const gs_pnp_opts* opts, gs_pnp_result* out, void* stream) {
  gsr::set_last_error("");
  if (!s || !cam || !T_render || !depth || !alpha || !opts || !out)
    return pnp_fail(GS_ERR_INVALID_ARG, "solver, cam, T_render, depth, alpha, opts and out are required");
  if (n_matches < 0 || n_matches > s->max_matches)
    return pnp_fail(GS_ERR_INVALID_ARG, "n_matches outside [0, max_matches]");
  if (n_hypotheses < 0 || n_hypotheses > s->max_hyp)
    return pnp_fail(GS_ERR_INVALID_ARG, "n_hypotheses outside [0, max_hypotheses]");
  if ((n_matches > 0 && !matches) || (n_hypotheses > 0 && !words))
    return pnp_fail(GS_ERR_INVALID_ARG, "matches and words are required when their counts are positive");
  if (!(opts->tau_px > 0.0f) || !std::isfinite(opts->tau_px) || !(opts->min_alpha > 0.0f) ||
      !(opts->min_alpha <= 1.0f) || opts->refine_iters < 0 || opts->refine_iters > 100)
    return pnp_fail(GS_ERR_INVALID_ARG, "options out of range");
  if (cam->width < 1 || cam->height < 1 || (int64_t)cam->width * cam->height >= (1ll << 31) ||
      !(cam->fx > 0.0f) || !(cam->fy > 0.0f) || !std::isfinite(cam->fx) || !std::isfinite(cam->fy) ||
      !std::isfinite(cam->cx) || !std::isfinite(cam->cy))
    return pnp_fail(GS_ERR_INVALID_ARG, "camera out of range");
  for (int k = 0; k < 16; ++k)
    if (!std::isfinite(T_render->T_cw[k])) return pnp_fail(GS_ERR_INVALID_ARG, "T_render has a non-finite entry");
  PNP_CUDA(cudaSetDevice(s->device));
  const cudaStream_t st = (cudaStream_t)stream;
  Cam c;
  c.fx = cam->fx;
  c.fy = cam->fy;
  c.cx = cam->cx;
  c.cy = cam->cy;
  c.ifx = 1.0 / c.fx;
  c.ify = 1.0 / c.fy;
  c.W = cam->width;
  c.H = cam->height;
  Pose12 Tr;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) Tr.v[3 * i + j] = T_render->T_cw[4 * i + j];
    Tr.v[9 + i] = T_render->T_cw[4 * i + 3];
  }
  const float fx = cam->fx, fy = cam->fy, tau = opts->tau_px;
  auto mark = [&](int k) -> cudaError_t { return s->timing ? cudaEventRecord(s->ev[k], st) : cudaSuccess; };
  PNP_CUDA(mark(0));
  PNP_CUDA(cudaMemsetAsync(s->st, 0, sizeof(State), st));
  if (n_matches > 0) PNP_CUDA(cudaMemsetAsync(s->mask, 0, (size_t)n_matches, st));
  const int nb = (int)((n_matches + kCompact - 1) / kCompact);
  if (nb > 0) {
    k_pnp_flags<<<nb, kThreads, 0, st>>>(matches, n_matches, alpha, c.W * c.H, opts->min_alpha, s->blk, s->st);
    PNP_CUDA(cudaGetLastError());
  }
  k_pnp_scan<<<1, 1024, 0, st>>>(s->blk, nb, s->st);
  PNP_CUDA(cudaGetLastError());
  if (nb > 0) {
    k_pnp_lift<<<nb, kThreads, 0, st>>>(matches, n_matches, depth, alpha, c, Tr, opts->min_alpha, s->blk, s->X64,
                                        s->X32, s->nab, s->pix, s->vidx);
    PNP_CUDA(cudaGetLastError());
  }
  PNP_CUDA(mark(1));
  const int n_poses = n_hypotheses * kSol;
  if (n_hypotheses > 0) {
    k_pnp_p3p<<<(n_hypotheses + 31) / 32, 32, 0, st>>>(s->X64, s->pix, s->st, words, n_hypotheses, c,
                                                          s->poses64, s->poses32, s->counts);
    PNP_CUDA(cudaGetLastError());
  }
  PNP_CUDA(mark(2));
  if (n_hypotheses > 0) {
    if (n_matches > 0) {
      const dim3 grid((unsigned)((n_matches + kThreads * kRow - 1) / (kThreads * kRow)),
                      (unsigned)((n_poses + kScorePoses - 1) / kScorePoses));
      k_pnp_score<<<grid, kThreads, 0, st>>>(s->X32, s->nab, s->st, s->poses32, s->counts, n_poses, fx, fy, tau);
      PNP_CUDA(cudaGetLastError());
    }
  }
  PNP_CUDA(mark(3));
  k_pnp_best<<<1, 1024, 0, st>>>(s->counts, n_poses, s->poses64, Tr, s->st);
  PNP_CUDA(cudaGetLastError());
  PNP_CUDA(mark(4));
  for (int it = 0; it < opts->refine_iters; ++it) {
    k_pnp_gn<<<kGnBlocks, kThreads, 0, st>>>(s->X32, s->nab, s->st, s->partials, fx, fy, tau);
    PNP_CUDA(cudaGetLastError());
    k_pnp_gn_solve<<<1, kGnVals * kSolveParts, 0, st>>>(s->partials, s->st);
    PNP_CUDA(cudaGetLastError());
  }
  PNP_CUDA(mark(5));
  if (n_matches > 0) {
    const int g = std::min<int64_t>((n_matches + kThreads - 1) / kThreads, (int64_t)s->sm_count * 8);
    k_pnp_final<<<g, kThreads, 0, st>>>(s->X32, s->nab, s->vidx, s->st, s->mask, fx, fy, tau);
    PNP_CUDA(cudaGetLastError());
  }
  PNP_CUDA(mark(6));
  PNP_CUDA(cudaMemcpyAsync(s->st_host, s->st, sizeof(State), cudaMemcpyDeviceToHost, st));
  PNP_CUDA(cudaStreamSynchronize(st));
  if (s->timing) {
    for (int k = 0; k < GS_PNP_PHASES; ++k) {
      float ms = 0.0f;
      PNP_CUDA(cudaEventElapsedTime(&ms, s->ev[k], s->ev[k + 1]));
      s->kt_ms[k] += ms;
    }
    s->kt_n += 1;
  }
  const State& h = *s->st_host;
  std::memset(out, 0, sizeof(*out));
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) out->T_cw[4 * i + j] = h.T[3 * i + j];
    out->T_cw[4 * i + 3] = h.T[9 + i];
  }
  out->T_cw[15] = 1.0;
  out->n_valid = h.n_valid;
  out->n_inliers = h.n_inliers;
  out->best_hypothesis = h.best_h;
  out->best_solution = h.best_s;
  out->best_count = h.best_count;
  out->refine_steps = h.steps;
  out->inlier = s->mask;
  out->valid_index = s->vidx;
  out->points = s->X64;
  out->hyp_counts = s->counts;
  out->hyp_poses = s->poses64;
  if (h.bad_pixel) return pnp_fail(GS_ERR_INVALID_ARG, "a match has a pixel index outside the image");
  return GS_OK;
}

}  // extern "C"
