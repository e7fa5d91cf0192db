// Per-tile depth sort + front-to-back alpha compositing (forward), the adjoint
// compositor that accumulates the se(3) pose gradient (backward), and the
// fp64 reduction of the per-tile partial sums.
//
// Sec. 3.1 of the paper: colour is alpha-blended over the Gaussians covering a
// pixel, features go through the identical blending; the dense stage of
// Sec. 3.4 renders colour, depth and features at a candidate pose. The
// gradient is the analysis-by-synthesis derivative of the L1 photometric +
// depth loss with respect to the left pose perturbation.
//
// Both compositing kernels are persistent: CTAs pull tiles from a global
// queue spanning every view of the call, so views of different resolution
// share one launch and load-balance.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "gsr_internal.h"

namespace gsr {
namespace {

constexpr float kAlphaFloor = 1.0f / 255.0f;
constexpr float kAlphaCap = 0.99f;
constexpr float kTCut = 1e-4f;
constexpr int kWarps = kTileThreads / 32;

// -0.5 (A dx^2 + C dy^2) - B dx dy with one fixed rounding sequence, shared by
// the forward and backward kernels so that both take identical skip decisions.
__device__ __forceinline__ float gs_power(float A, float B, float C, float dx, float dy) {
  const float q = __fmaf_rn(C, __fmul_rn(dy, dy), __fmul_rn(A, __fmul_rn(dx, dx)));
  return __fmaf_rn(-B, __fmul_rn(dx, dy), __fmul_rn(-0.5f, q));
}

// Record centre (float-float: high parts in a.xy, half2 low parts in c.w)
// relative to the tile origin (X0, Y0): exact subtraction, one rounding.
__device__ __forceinline__ float4 tile_local(float4 a, float cw, float X0, float Y0) {
  const __half2 lo = *reinterpret_cast<const __half2*>(&cw);
  const float2 l = __half22float2(lo);
  return make_float4(__fadd_rn(__fsub_rn(a.x, X0), l.x), __fadd_rn(__fsub_rn(a.y, Y0), l.y), a.z, a.w);
}

__device__ __forceinline__ int find_view(const View* __restrict__ views, int n_views, uint32_t tile) {
  int lo = 0, hi = n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (views[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// exclusive scan of one value per thread over a 256-thread block
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* tmp) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) tmp[wid] = incl;
  __syncthreads();
  uint32_t off = 0;
#pragma unroll
  for (int k = 0; k < kWarps; ++k) off += (k < wid) ? tmp[k] : 0u;
  __syncthreads();
  return off + incl - v;
}

// One stable counting-sort pass on the 8-bit digit at `shift` of key .x, from
// `in` to `out` (shared or global memory). Each warp owns a contiguous run of
// the input; ranks inside a warp come from __match_any_sync, so equal digits
// keep their input order.
__device__ void radix_pass(const uint2* in, uint2* out, int n, int shift, uint32_t* hist, uint32_t* tmp) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = ((n + kTileThreads - 1) / kTileThreads) * 32;
  const int wb = warp * per;
  const int we = min(n, wb + per);
  for (int i = tid; i < kWarps * 256; i += kTileThreads) hist[i] = 0u;
  __syncthreads();
  uint32_t* h = hist + warp * 256;
  for (int b = wb; b < we; b += 32) {
    const int idx = b + lane;
    const bool ok = idx < we;
    const uint32_t d = ok ? ((in[idx].x >> shift) & 255u) : 0u;
    const uint32_t peers = __match_any_sync(0xffffffffu, ok ? d : 256u + lane);
    if (ok && lane == __ffs(peers) - 1) h[d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    const int d = tid;  // one digit per thread (256 threads)
    uint32_t c[kWarps];
    uint32_t tot = 0;
#pragma unroll
    for (int k = 0; k < kWarps; ++k) {
      c[k] = hist[k * 256 + d];
      tot += c[k];
    }
    uint32_t ex = block_excl_scan(tot, tmp);
#pragma unroll
    for (int k = 0; k < kWarps; ++k) {
      hist[k * 256 + d] = ex;
      ex += c[k];
    }
  }
  __syncthreads();
  const uint32_t lt = (1u << lane) - 1u;
  for (int b = wb; b < we; b += 32) {
    const int idx = b + lane;
    const bool ok = idx < we;
    const uint2 kv = ok ? in[idx] : make_uint2(0u, 0u);
    const uint32_t d = ok ? ((kv.x >> shift) & 255u) : 0u;
    const uint32_t peers = __match_any_sync(0xffffffffu, ok ? d : 256u + lane);
    const uint32_t basev = ok ? h[d] : 0u;
    __syncwarp();
    if (ok) {
      out[basev + __popc(peers & lt)] = kv;
      if (lane == __ffs(peers) - 1) h[d] = basev + __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();
}

// Sort the tile's pairs by depth bits, ties by Gaussian index. Returns the
// array holding the result (a or b).
__device__ uint2* sort_tile(uint2* a, uint2* b, int n, uint32_t* hist, uint32_t* tmp, const float4* __restrict__ rec_b) {
  __shared__ uint32_t s_and[kWarps], s_or[kWarps];
  uint32_t kand = 0xffffffffu, kor = 0u;
  for (int i = threadIdx.x; i < n; i += kTileThreads) {
    const uint32_t k = a[i].x;
    kand &= k;
    kor |= k;
  }
  kand = __reduce_and_sync(0xffffffffu, kand);
  kor = __reduce_or_sync(0xffffffffu, kor);
  if ((threadIdx.x & 31) == 0) {
    s_and[threadIdx.x >> 5] = kand;
    s_or[threadIdx.x >> 5] = kor;
  }
  __syncthreads();
  uint32_t diff = 0;
  {
    uint32_t A = 0xffffffffu, O = 0u;
#pragma unroll
    for (int k = 0; k < kWarps; ++k) {
      A &= s_and[k];
      O |= s_or[k];
    }
    diff = (n > 1) ? (A ^ O) : 0u;
  }
  __syncthreads();
  uint2* cur = a;
  uint2* oth = b;
  for (int shift = 0; shift < 32; shift += 8) {
    if (((diff >> shift) & 255u) == 0u) continue;
    radix_pass(cur, oth, n, shift, hist, tmp);
    uint2* t = cur;
    cur = oth;
    oth = t;
  }
  // equal depth bits: order by Gaussian index (rare; runs are short)
  for (int i = threadIdx.x + 1; i < n; i += kTileThreads) {
    if (cur[i].x == cur[i - 1].x && (i == 1 || cur[i - 2].x != cur[i - 1].x)) {
      const int s = i - 1;
      int e = i + 1;
      while (e < n && cur[e].x == cur[s].x) ++e;
      for (int p = s + 1; p < e; ++p) {
        const uint2 v = cur[p];
        const int gv = __float_as_int(rec_b[v.y].w);
        int q = p - 1;
        while (q >= s && __float_as_int(rec_b[cur[q].y].w) > gv) {
          cur[q + 1] = cur[q];
          --q;
        }
        cur[q + 1] = v;
      }
    }
  }
  __syncthreads();
  return cur;
}

// Shared-memory layout of the forward kernel (bytes). The staged batch aliases
// the second sort buffer, which is free once the sorted list sits in bufA.
constexpr int kSmBufA = 0;
constexpr int kSmBufB = kSortCap * 8;
constexpr int kSmHist = 2 * kSortCap * 8;
constexpr int kSmStage = kSmBufB;
constexpr int kSmFwd = kSmHist + kWarps * 256 * 4;
constexpr int kSmFeat = kSmHist;  // 16 KB of BF16 features: hist + 8 KB more
constexpr int kSmFwdFeat = (kSmFeat + kBatchF * 64) > kSmFwd ? (kSmFeat + kBatchF * 64) : kSmFwd;
static_assert(4 * kBatchF * 16 <= kSortCap * 8, "staging must fit in the second sort buffer");

// Warp w covers the 8 x 4 pixel block at (8 (w & 1), 4 (w >> 1)) of the tile.
__device__ __forceinline__ void warp_block(int tid, int& lx, int& ly, int& bx, int& by) {
  const int warp = tid >> 5, lane = tid & 31;
  bx = (warp & 1) * 8;
  by = (warp >> 1) * 4;
  lx = bx + (lane & 7);
  ly = by + (lane >> 3);
}

// Threshold of the alpha-floor test as an ellipse: o exp(power) >= 1/255 with
// power = -q/2, q(d) = A dx^2 + 2 B dx dy + C dy^2, needs q <= 2 ln(255 o).
// Margins (1 % + 0.01 on the log, 0.1 % + 1e-3 on the threshold) cover the
// fp32 evaluation of the per-pixel test; -1 marks a Gaussian whose opacity
// cannot reach the floor anywhere.
__device__ __forceinline__ float floor_threshold(float o) {
  const float Lp = __logf(255.0f * o) * 1.01f + 0.01f;
  return Lp > 0.0f ? 2.0f * Lp * 1.001f + 1e-3f : -1.0f;
}

// Can a staged Gaussian (centre a.xy in tile-local pixels, conic A = a.z,
// B = a.w, C) reach the floor at any pixel centre of the warp's block
// [x0, x1] x [y0, y1]? Exact minimum of the positive-definite quadratic over
// the block (the centre if inside, else the best point of one of the four
// edges). If not, every pixel of the warp would skip the Gaussian, so the warp
// skips it without changing any result.
__device__ __forceinline__ bool ellipse_hits(float4 a, float C, float thr, float x0, float x1, float y0, float y1) {
  if (!(thr > 0.0f)) return false;
  const float A = a.z, B = a.w;
  if (!(A > 0.0f) || !(C > 0.0f)) return true;
  const float dxl = x0 - a.x, dxh = x1 - a.x, dyl = y0 - a.y, dyh = y1 - a.y;
  if (dxl <= 0.0f && dxh >= 0.0f && dyl <= 0.0f && dyh >= 0.0f) return true;
  const float iA = 1.0f / A, iC = 1.0f / C;
  float best = 3.0e38f;
  {
    const float dy0 = fminf(fmaxf(-B * dxl * iC, dyl), dyh), dy1 = fminf(fmaxf(-B * dxh * iC, dyl), dyh);
    best = fminf(best, A * dxl * dxl + 2.0f * B * dxl * dy0 + C * dy0 * dy0);
    best = fminf(best, A * dxh * dxh + 2.0f * B * dxh * dy1 + C * dy1 * dy1);
  }
  {
    const float dx0 = fminf(fmaxf(-B * dyl * iA, dxl), dxh), dx1 = fminf(fmaxf(-B * dyh * iA, dxl), dxh);
    best = fminf(best, A * dx0 * dx0 + 2.0f * B * dx0 * dyl + C * dyl * dyl);
    best = fminf(best, A * dx1 * dx1 + 2.0f * B * dx1 * dyh + C * dyh * dyh);
  }
  return best <= thr;
}

// Bit w set when the staged Gaussian can reach the floor in warp w's 8 x 4
// block (ellipse_hits); a slightly widened bounding box of the ellipse rejects
// most blocks first. Computed once per staged Gaussian by its staging thread.
__device__ __forceinline__ uint32_t warp_hit_mask(float4 a, float C, float thr) {
  if (!(thr > 0.0f)) return 0u;
  const float A = a.z, B = a.w;
  const float detq = A * C - B * B;
  if (!(A > 0.0f) || !(C > 0.0f) || !(detq > 0.0f)) return 0xffu;
  const float ex = sqrtf(thr * C / detq) * 1.0001f + 1e-3f, ey = sqrtf(thr * A / detq) * 1.0001f + 1e-3f;
  uint32_t mask = 0u;
#pragma unroll
  for (int wv = 0; wv < kWarps; ++wv) {
    const float x0 = (float)((wv & 1) * 8) + 0.5f, x1 = x0 + 7.0f;
    const float y0 = (float)((wv >> 1) * 4) + 0.5f, y1 = y0 + 3.0f;
    if (a.x + ex < x0 || a.x - ex > x1 || a.y + ey < y0 || a.y - ey > y1) continue;
    if (ellipse_hits(a, C, thr, x0, x1, y0, y1)) mask |= 1u << wv;
  }
  return mask;
}

template <int FEAT>
__global__ void __launch_bounds__(kTileThreads) k_composite(SceneDev sc, const View* __restrict__ views, int n_views,
                                                            Work w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint2* bufA = reinterpret_cast<uint2*>(smem_raw + kSmBufA);
  uint2* bufB = reinterpret_cast<uint2*>(smem_raw + kSmBufB);
  uint32_t* hist = reinterpret_cast<uint32_t*>(smem_raw + kSmHist);
  float4* sa = reinterpret_cast<float4*>(smem_raw + kSmStage);
  float4* sb = sa + kBatchF;
  float4* scol = sb + kBatchF;
  uint32_t* smask = reinterpret_cast<uint32_t*>(scol + kBatchF);
  uint4* sf = reinterpret_cast<uint4*>(smem_raw + kSmFeat);  // FEAT: kBatchF x 4 (aliases hist)
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_tmp[kWarps];
  if (w.ctr->overflow) return;
  const int tid = threadIdx.x, lane = tid & 31;
  int lx, ly, bxw, byw;
  warp_block(tid, lx, ly, bxw, byw);
  const float pxc = (float)lx + 0.5f, pyc = (float)ly + 0.5f;
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(&w.ctr->fwd_queue, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= w.n_tiles) break;
    const int vi = find_view(views, n_views, tile);
    const View& V = views[vi];
    const uint32_t lt = tile - V.tile_base;
    const int tx = (int)(lt % (uint32_t)V.tiles_x), ty = (int)(lt / (uint32_t)V.tiles_x);
    const uint32_t start = w.tile_offset[tile];
    const int n = (int)(w.tile_offset[tile + 1] - start);

    // ---- depth order of the tile's list (short lists: already sorted by
    // the warp sort that ran before this kernel) ----
    const uint2* list;
    if (n <= kWarpSortMax) {
      list = w.pairs + start;
    } else if (n <= kSortCap) {
      for (int i = tid; i < n; i += kTileThreads) bufA[i] = w.pairs[start + i];
      __syncthreads();
      const uint2* sorted = sort_tile(bufA, bufB, n, hist, s_tmp, w.rec_b);
      if (sorted != bufA) {
        for (int i = tid; i < n; i += kTileThreads) bufA[i] = sorted[i];
        __syncthreads();
      }
      for (int i = tid; i < n; i += kTileThreads) w.pairs[start + i] = bufA[i];
      list = bufA;
    } else {
      uint2* sorted = sort_tile(w.pairs + start, w.pairs_tmp + start, n, hist, s_tmp, w.rec_b);
      if (sorted != w.pairs + start) {
        for (int i = tid; i < n; i += kTileThreads) w.pairs[start + i] = sorted[i];
        __syncthreads();
      }
      list = w.pairs + start;
    }

    // ---- front-to-back blending, one pixel per thread ----
    const int px = tx * kTile + lx, py = ty * kTile + ly;
    const bool inside = px < V.width && py < V.height;
    const float X0 = (float)(tx * kTile), Y0 = (float)(ty * kTile);
    float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
    float F[FEAT > 0 ? FEAT : 1];
#pragma unroll
    for (int c = 0; c < (FEAT > 0 ? FEAT : 1); ++c) F[c] = 0.f;
    uint32_t last = 0;
    bool done = !inside;
    for (int bs = 0; bs < n; bs += kBatchF) {
      if (__syncthreads_count(done) == kTileThreads) break;
      const int bn = min(kBatchF, n - bs);
      if (tid < bn) {
        const uint32_t r = list[bs + tid].y;
        const float4 cc = w.rec_c[r];
        const float4 a = tile_local(w.rec_a[r], cc.w, X0, Y0);
        const float4 bb = w.rec_b[r];
        sa[tid] = a;
        sb[tid] = bb;
        scol[tid] = cc;
        smask[tid] = warp_hit_mask(a, bb.x, floor_threshold(bb.y));
        if (FEAT) {
          const uint4* fp = sc.feat + (size_t)__float_as_int(bb.w) * 4;
#pragma unroll
          for (int q = 0; q < 4; ++q) sf[tid * 4 + q] = __ldg(fp + q);
        }
      }
      __syncthreads();
      // blend one staged Gaussian (power and o exp(power) already evaluated) into
      // this pixel; branch-free: the skip and stop decisions become predicates
      auto blend = [&](int j, float p, float oe, float zj) {
        const float alpha = fminf(kAlphaCap, oe);
        const bool take = !done && !(p > 0.0f) && !(alpha < kAlphaFloor);
        const float Tn = __fmul_rn(T, __fsub_rn(1.0f, alpha));
        const bool stop = take && (Tn < kTCut);
        const bool acc = take && !stop;
        const float wgt = acc ? __fmul_rn(alpha, T) : 0.0f;
        const float4 c = scol[j];
        C0 = fmaf(wgt, c.x, C0);
        C1 = fmaf(wgt, c.y, C1);
        C2 = fmaf(wgt, c.z, C2);
        D = fmaf(wgt, zj, D);
        if (FEAT) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint4 fv = sf[j * 4 + q];
            const uint32_t u4[4] = {fv.x, fv.y, fv.z, fv.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              F[8 * q + 2 * h] = fmaf(wgt, __uint_as_float(u4[h] << 16), F[8 * q + 2 * h]);
              F[8 * q + 2 * h + 1] = fmaf(wgt, __uint_as_float(u4[h] & 0xffff0000u), F[8 * q + 2 * h + 1]);
            }
          }
        }
        T = acc ? Tn : T;
        last = acc ? (uint32_t)(bs + j + 1) : last;
        done = done || stop;
      };
      const uint32_t wbit = 1u << (tid >> 5);
      bool wdone = __all_sync(0xffffffffu, done);
      for (int c0 = 0; c0 < bn && !wdone; c0 += 32) {
        const int jj = c0 + lane;
        uint32_t m = __ballot_sync(0xffffffffu, jj < bn && (smask[jj] & wbit));
        while (m) {  // two hits per step: their exponentials overlap, blending stays in order
          const int j1 = c0 + __ffs(m) - 1;
          m &= m - 1;
          const bool two = m != 0u;
          const int j2 = two ? c0 + __ffs(m) - 1 : j1;
          if (two) m &= m - 1;
          const float4 a1 = sa[j1], b1 = sb[j1], a2 = sa[j2], b2 = sb[j2];
          const float p1 = gs_power(a1.z, a1.w, b1.x, __fsub_rn(a1.x, pxc), __fsub_rn(a1.y, pyc));
          const float p2 = gs_power(a2.z, a2.w, b2.x, __fsub_rn(a2.x, pxc), __fsub_rn(a2.y, pyc));
          const float oe1 = __fmul_rn(b1.y, __expf(p1));
          const float oe2 = __fmul_rn(b2.y, __expf(p2));
          blend(j1, p1, oe1, b1.z);
          if (two) blend(j2, p2, oe2, b2.z);
        }
        wdone = __all_sync(0xffffffffu, done);
      }
    }
    if (inside) {
      const size_t HW = (size_t)V.width * V.height;
      const size_t p = (size_t)py * V.width + px;
      if (V.rgb) {
        V.rgb[p] = C0;
        V.rgb[HW + p] = C1;
        V.rgb[2 * HW + p] = C2;
      }
      if (V.depth) V.depth[p] = D;
      if (V.alpha) V.alpha[p] = 1.0f - T;
      if (V.final_T) V.final_T[p] = T;
      if (V.last_idx) V.last_idx[p] = last;
      if (FEAT && V.feats) {
#pragma unroll
        for (int c = 0; c < (FEAT > 0 ? FEAT : 1); ++c) V.feats[(size_t)c * HW + p] = F[c];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Backward: per pixel, walk the blended Gaussians back to front recomputing
// the transmittance from the stored final value, T_k = T_{k+1} / (1 - a_k);
// chain dL/d(u, v, conic, z, rgb) through the per-Gaussian pose Jacobian and
// accumulate the 6-vector per pixel (fp32); reduce across pixels in fp64.
// The same per-warp footprint test as the forward skips pairs that no pixel of
// the warp blended.
// ---------------------------------------------------------------------------
struct BwdSmem {
  float4 sa[kBatchB], sb[kBatchB], sc[kBatchB];
  uint32_t smask[kBatchB];
  float4 sj[kBatchB * (kJacStride / 4)];
  float red[kWarps][8];
};

__global__ void __launch_bounds__(kTileThreads) k_backward(const View* __restrict__ views, int n_views, Work w,
                                                           double* __restrict__ result) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BwdSmem& S = *reinterpret_cast<BwdSmem*>(smem_raw);
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_max[kWarps];
  __shared__ bool s_last;
  if (w.ctr->overflow) return;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  int lx, ly, bxw, byw;
  warp_block(tid, lx, ly, bxw, byw);
  const float pxc = (float)lx + 0.5f, pyc = (float)ly + 0.5f;
  const uint32_t wbit = 1u << wid;
  const float4* rec_j4 = reinterpret_cast<const float4*>(w.rec_j);
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(&w.ctr->bwd_queue, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= w.n_tiles) break;
    const int vi = find_view(views, n_views, tile);
    const View& V = views[vi];
    const uint32_t lt = tile - V.tile_base;
    const int tx = (int)(lt % (uint32_t)V.tiles_x), ty = (int)(lt / (uint32_t)V.tiles_x);
    const uint32_t start = w.tile_offset[tile];
    const int px = tx * kTile + lx, py = ty * kTile + ly;
    const bool inside = px < V.width && py < V.height;
    const float X0 = (float)(tx * kTile), Y0 = (float)(ty * kTile);
    const size_t HW = (size_t)V.width * V.height;
    const size_t p = (size_t)py * V.width + px;

    uint32_t last = 0;
    float T = 1.0f, gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gD = 0.f;
    float loss = 0.0f;
    if (inside) {
      last = V.last_idx[p];
      T = V.final_T[p];
      const float wpx = V.pixel_weight ? V.pixel_weight[p] : 1.0f;
      const float r0 = V.rgb[p] - V.target_rgb[p];
      const float r1 = V.rgb[HW + p] - V.target_rgb[HW + p];
      const float r2 = V.rgb[2 * HW + p] - V.target_rgb[2 * HW + p];
      const float e = V.depth[p] - V.target_depth[p];
      const float s3 = wpx * V.inv_3p, sd = wpx * V.depth_weight * V.inv_p;
      gC0 = s3 * (float)((r0 > 0.f) - (r0 < 0.f));
      gC1 = s3 * (float)((r1 > 0.f) - (r1 < 0.f));
      gC2 = s3 * (float)((r2 > 0.f) - (r2 < 0.f));
      gD = sd * (float)((e > 0.f) - (e < 0.f));
      loss = s3 * (fabsf(r0) + fabsf(r1) + fabsf(r2)) + sd * fabsf(e);
    }
    // longest list prefix any pixel of the tile (and of this warp) blended
    const uint32_t wm = __reduce_max_sync(0xffffffffu, last);
    if (lane == 0) s_max[wid] = wm;
    __syncthreads();
    uint32_t max_last = 0;
#pragma unroll
    for (int k = 0; k < kWarps; ++k) max_last = max(max_last, s_max[k]);

    // per-tangent partial sums: .x and .y take different Jacobian rows and are
    // added at the end
    float2 xi2[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) xi2[k] = make_float2(0.f, 0.f);
    float sdot = 0.f;
    for (int bend = (int)max_last; bend > 0; bend -= kBatchB) {
      const int bstart = max(0, bend - kBatchB);
      const int bn = bend - bstart;
      __syncthreads();
      if (tid < bn) {
        const uint32_t r = w.pairs[start + bstart + tid].y;
        const float4 cc = w.rec_c[r];
        const float4 a = tile_local(w.rec_a[r], cc.w, X0, Y0);
        const float4 bb = w.rec_b[r];
        S.sa[tid] = a;
        S.sb[tid] = bb;
        S.sc[tid] = cc;
        S.smask[tid] = warp_hit_mask(a, bb.x, floor_threshold(bb.y));
      }
      for (int q = tid; q < bn * (kJacStride / 4); q += kTileThreads) {
        const int jj = q / (kJacStride / 4), k = q % (kJacStride / 4);
        const uint32_t r = w.pairs[start + bstart + jj].y;
        S.sj[q] = rec_j4[(size_t)r * (kJacStride / 4) + k];
      }
      __syncthreads();
      if ((uint32_t)bstart >= wm) continue;  // no pixel of this warp blended this far
      // one Gaussian, back to front: if this pixel blended it, step T and the
      // running sum back and chain its 9 sensitivities through the staged pose
      // Jacobian (48 floats in tangent-major pairs, read as 12 float4).
      // Branch-free: a pixel that skipped the Gaussian contributes zeros.
      auto adjoint = [&](int j, float4 a, float4 b, float dx, float dy, float p, float oe, bool live) {
        const float alpha = fminf(kAlphaCap, oe);
        const bool take = live && !(p > 0.0f) && !(alpha < kAlphaFloor);
        const float Tj = take ? __fdividef(T, 1.0f - alpha) : T;  // transmittance in front of this Gaussian
        const float wgt = take ? alpha * Tj : 0.0f;
        const float4 c = S.sc[j];
        // dL/dalpha = Tj (g . (c, z) - g . acc), where acc, the normalised
        // colour and depth behind this Gaussian, follows acc <- alpha (c, z) +
        // (1 - alpha) acc; only its projection sdot = g . acc is needed
        const float gc = fmaf(gC0, c.x, fmaf(gC1, c.y, fmaf(gC2, c.z, gD * b.z)));
        const float d = gc - sdot;
        sdot = fmaf(take ? alpha : 0.0f, d, sdot);
        T = Tj;
        const float q = (take && oe < kAlphaCap) ? -(Tj * d) * alpha : 0.0f;  // -dL/dpower
        const float dxq = q * dx, dyq = q * dy;
        // the nine sensitivities in pairs; each packed FMA takes one pair
        // against the matching Jacobian pair of one tangent direction
        const float2 g01 = make_float2(dxq, dyq);
        const float2 g23 = make_float2(dxq * dx, dxq * dy);
        const float2 g45 = make_float2(dyq * dy, gD * wgt);
        const float2 g67 = make_float2(gC0 * wgt, gC1 * wgt);
        const float g8 = gC2 * wgt;
        const float4* J4 = S.sj + j * (kJacStride / 4);
#pragma unroll
        for (int q = 0; q < kJacStride / 4; ++q) {
          const float4 v = J4[q];
          const float2 e[2] = {make_float2(v.x, v.y), make_float2(v.z, v.w)};
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const int pr = 2 * q + i;  // pair index
            if (pr < 18) {
              const float2 gg = (pr % 3 == 0) ? g01 : (pr % 3 == 1) ? g23 : g45;
              xi2[pr / 3] = __ffma2_rn(e[i], gg, xi2[pr / 3]);
            } else if (pr < 21) {
              xi2[pr - 18] = __ffma2_rn(e[i], g67, xi2[pr - 18]);
            } else if (pr == 21) {  // floats 42, 43: d blue / d rho_0, rho_1
              xi2[0].x = fmaf(e[i].x, g8, xi2[0].x);
              xi2[1].x = fmaf(e[i].y, g8, xi2[1].x);
            } else if (pr == 22) {  // float 44: d blue / d rho_2
              xi2[2].x = fmaf(e[i].x, g8, xi2[2].x);
            }
          }
        }
      };
      for (int c0 = ((bn - 1) >> 5) << 5; c0 >= 0; c0 -= 32) {
        const int jj = c0 + lane;
        uint32_t m = __ballot_sync(0xffffffffu, jj < bn && (uint32_t)(bstart + jj) < wm && (S.smask[jj] & wbit));
        while (m) {  // two hits per step, back to front
          const int bit1 = 31 - __clz(m);
          m &= ~(1u << bit1);
          const bool two = m != 0u;
          const int bit2 = two ? 31 - __clz(m) : bit1;
          if (two) m &= ~(1u << bit2);
          const int j1 = c0 + bit1, j2 = c0 + bit2;
          const float4 a1 = S.sa[j1], b1 = S.sb[j1], a2 = S.sa[j2], b2 = S.sb[j2];
          const float dx1 = __fsub_rn(a1.x, pxc), dy1 = __fsub_rn(a1.y, pyc);
          const float dx2 = __fsub_rn(a2.x, pxc), dy2 = __fsub_rn(a2.y, pyc);
          const float p1 = gs_power(a1.z, a1.w, b1.x, dx1, dy1);
          const float p2 = gs_power(a2.z, a2.w, b2.x, dx2, dy2);
          const float oe1 = __fmul_rn(b1.y, __expf(p1));
          const float oe2 = __fmul_rn(b2.y, __expf(p2));
          adjoint(j1, a1, b1, dx1, dy1, p1, oe1, inside && (uint32_t)(bstart + j1) < last);
          if (two) adjoint(j2, a2, b2, dx2, dy2, p2, oe2, inside && (uint32_t)(bstart + j2) < last);
        }
      }
    }
    // (loss, xi) of the tile in fp32: a fixed tree over each warp's lanes, then
    // the warps in order. GB300 runs fp64 at 1/64 of the fp32 rate, so fp64
    // starts at the tile sums.
    float v[7];
    v[0] = loss;
#pragma unroll
    for (int k = 0; k < 6; ++k) v[1 + k] = xi2[k].x + xi2[k].y;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 7; ++k) S.red[wid][k] = v[k];
    }
    __syncthreads();
    if (tid < 7) {
      float t = S.red[0][tid];
#pragma unroll
      for (int k = 1; k < kWarps; ++k) t += S.red[k][tid];
      w.partials[(size_t)tile * kPartialStride + tid] = (double)t;
      __threadfence();
    }
    __syncthreads();
    // Deterministic fp64 reduction in two fixed levels, done by whichever CTA
    // finishes the last tile of a chunk (kChunkTiles tiles of one view) and
    // then the last chunk of the view: the order depends only on tile indices,
    // so a view gives the same bits alone or inside a batch.
    const uint32_t nt = (uint32_t)V.tiles_x * (uint32_t)V.tiles_y;
    const uint32_t chunk = lt / kChunkTiles, c0 = chunk * kChunkTiles;
    const uint32_t cn = min((uint32_t)kChunkTiles, nt - c0);
    if (tid == 0) s_last = atomicAdd(&w.chunk_ctr[V.chunk_base + chunk], 1u) == cn - 1u;
    __syncthreads();
    if (!s_last) continue;
    __threadfence();
    if (wid < 7) {  // warp k sums component k; lanes take tiles lane and lane + 32
      const double* src = w.partials + (size_t)(V.tile_base + c0) * kPartialStride + wid;
      double x = (uint32_t)lane < cn ? __ldcg(src + (size_t)lane * kPartialStride) : 0.0;
      if ((uint32_t)lane + 32u < cn) x += __ldcg(src + (size_t)(lane + 32) * kPartialStride);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) {
        w.chunk_part[(size_t)(V.chunk_base + chunk) * kPartialStride + wid] = x;
        __threadfence();
      }
    }
    __syncthreads();
    const uint32_t ncv = (nt + kChunkTiles - 1) / kChunkTiles;
    if (tid == 0) s_last = atomicAdd(&w.view_ctr[vi], 1u) == ncv - 1u;
    __syncthreads();
    if (!s_last) continue;
    __threadfence();
    if (wid < 7) {
      double x = 0.0;
      for (uint32_t c = lane; c < ncv; c += 32)
        x += __ldcg(w.chunk_part + (size_t)(V.chunk_base + c) * kPartialStride + wid);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) result[(size_t)vi * kPartialStride + wid] = x;
    }
  }
}

template <int FEAT>
size_t composite_smem() {
  return FEAT ? (size_t)kSmFwdFeat : (size_t)kSmFwd;
}

template <int FEAT>
int composite_occ() {
  static int occ = -1;
  if (occ < 0) {
    cudaFuncSetAttribute(k_composite<FEAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)composite_smem<FEAT>());
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_composite<FEAT>, kTileThreads, composite_smem<FEAT>()) !=
        cudaSuccess)
      b = 1;
    occ = b > 0 ? b : 1;
  }
  return occ;
}

}  // namespace

int composite_blocks_per_sm(int feat_dim) { return feat_dim ? composite_occ<32>() : composite_occ<0>(); }

int backward_blocks_per_sm() {
  static int occ = -1;
  if (occ < 0) {
    cudaFuncSetAttribute(k_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BwdSmem));
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_backward, kTileThreads, sizeof(BwdSmem)) != cudaSuccess)
      b = 1;
    occ = b > 0 ? b : 1;
  }
  return occ;
}

cudaError_t launch_composite(const SceneDev& sc, const View* views, int n_views, const Work& w, bool feats,
                             int grid, cudaStream_t st) {
  if (w.n_tiles == 0) return cudaSuccess;
  const int g = (uint32_t)grid < w.n_tiles ? grid : (int)w.n_tiles;
  if (sc.feat_dim && feats) {
    composite_occ<32>();
    k_composite<32><<<g, kTileThreads, composite_smem<32>(), st>>>(sc, views, n_views, w);
  } else {
    composite_occ<0>();
    k_composite<0><<<g, kTileThreads, composite_smem<0>(), st>>>(sc, views, n_views, w);
  }
  return cudaGetLastError();
}

cudaError_t launch_backward(const View* views, int n_views, const Work& w, double* result, int grid,
                            cudaStream_t st) {
  if (w.n_tiles == 0) return cudaSuccess;
  backward_blocks_per_sm();
  const int g = (uint32_t)grid < w.n_tiles ? grid : (int)w.n_tiles;
  k_backward<<<g, kTileThreads, sizeof(BwdSmem), st>>>(views, n_views, w, result);
  return cudaGetLastError();
}

}  // namespace gsr
