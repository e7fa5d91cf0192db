// Front-to-back alpha compositing of the depth-sorted tile lists (with the
// block sort of lists too long for the warp sort), optionally carrying the
// six pose tangents through the blend to give the se(3) gradient of the L1
// loss in the same pass, and the fp64 reduction of the per-tile sums.
//
// Sec. 3.1 of the paper: colour is alpha-blended over the Gaussians covering a
// pixel, features go through the identical blending; the dense stage of
// Sec. 3.4 renders colour, depth and features at a candidate pose. The
// gradient is the analysis-by-synthesis derivative of the L1 photometric +
// depth loss with respect to the left pose perturbation.
//
// The kernel is persistent: CTAs pull tiles from a global queue spanning
// every view of the call, so views of different resolution share one launch
// and load-balance.
#include <cuda_bf16.h>
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
// Tangent mode reads the sorted list back from global memory, so after the
// sort the staged pose Jacobians take the two sort buffers and the staged
// batch takes the histogram.
constexpr int kSmJac = 0;
constexpr int kSmStageT = kSmHist;
constexpr int kSmTan = kSmFwd;
// Feature blending on the tensor cores (FEAT): each warp collects the weights
// of its hits in slots of kSlots, transposed (slot-major, one row of 32
// pixels per slot) and split into three bf16 terms w = hi + mid + lo (exact to
// about 2^-24, the binary32 weight's own precision), then adds
// W (32 pixels x kSlots) . f (kSlots x 32 channels) to its accumulator
// fragments with mma.sync (bf16 x bf16 products are exact in fp32, with fp32
// accumulation). Rows of kWtRow bf16 (80 bytes): the eight 16-byte rows an
// ldmatrix reads fall in distinct banks.
// The features of the slots' Gaussians are copied into a per-warp buffer of
// kSlots rows (same 80-byte stride) when a slot is filled, so that slots span
// staging batches: a slot group is every kSlots hits of the warp in depth
// order, whatever the batch size, and the sums come out the same bits under
// every launch configuration.
constexpr int kSlots = 16;
constexpr int kWtRow = 40;
constexpr int kWtTerms = 3;                   // hi, mid, lo
constexpr int kWtWarp = kWtTerms * kSlots * kWtRow;  // bf16 per warp: hi rows, mid rows, lo rows
constexpr int kSmWtBytes = kWarps * kWtWarp * 2;
constexpr int kSmFbBytes = kWarps * kSlots * kWtRow * 2;  // per-warp slot features (bf16 rows)
// Feature-mode layout (blend phase; the sorted list is back in global memory,
// so it may reuse the sort buffers): staged records, staged features, weight
// slots, slot features.
template <int KB>
__host__ __device__ constexpr int feat_off_sf() { return ((KB * 52 + 15) / 16) * 16; }
template <int KB>
__host__ __device__ constexpr int feat_off_wt() { return feat_off_sf<KB>() + KB * 64; }
template <int KB>
__host__ __device__ constexpr int feat_off_fb() { return feat_off_wt<KB>() + kSmWtBytes; }

// dynamic shared memory of a compositor variant (staged batch of KB Gaussians)
template <int FEAT, bool TAN, int KB>
constexpr int comp_smem() {
  return TAN ? kSmTan
             : FEAT ? ((feat_off_fb<KB>() + kSmFbBytes) > kSmFwd ? (feat_off_fb<KB>() + kSmFbBytes) : kSmFwd)
                    : kSmFwd;
}

// four 8 x 8 b16 matrices from shared memory, transposed (lane l gives the
// address of row l % 8 of matrix l / 8)
__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

// d += a . b, m16 n8 k16, bf16 operands, fp32 accumulation
__device__ __forceinline__ void mma_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                          uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

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
// block (ellipse_hits), for the warps w0 <= w < w1; a slightly widened bounding
// box of the ellipse rejects most blocks first. Computed once per staged
// Gaussian and warp block by a staging thread.
template <int W0 = 0, int W1 = kWarps>
__device__ __forceinline__ uint32_t warp_hit_mask(float4 a, float C, float thr, int w0 = W0, int w1 = W1) {
  if (!(thr > 0.0f)) return 0u;
  const float A = a.z, B = a.w;
  const float detq = A * C - B * B;
  if (!(A > 0.0f) || !(C > 0.0f) || !(detq > 0.0f)) return (1u << w1) - (1u << w0);
  const float ex = sqrtf(thr * C / detq) * 1.0001f + 1e-3f, ey = sqrtf(thr * A / detq) * 1.0001f + 1e-3f;
  uint32_t mask = 0u;
#pragma unroll
  for (int wv = W0; wv < W1; ++wv) {
    if (wv < w0 || wv >= w1) continue;
    const float x0 = (float)((wv & 1) * 8) + 0.5f, x1 = x0 + 7.0f;
    const float y0 = (float)((wv >> 1) * 4) + 0.5f, y1 = y0 + 3.0f;
    if (a.x + ex < x0 || a.x - ex > x1 || a.y + ey < y0 || a.y - ey > y1) continue;
    if (ellipse_hits(a, C, thr, x0, x1, y0, y1)) mask |= 1u << wv;
  }
  return mask;
}


// 16-byte asynchronous copy global -> shared (both 16-byte aligned)
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}

// (loss, dL/dxi) of one tile: a fixed fp32 tree over each warp's lanes, then
// the warps in order (GB300 runs fp64 at 1/64 of the fp32 rate, so fp64 starts
// at the tile sums), written to the tile's slot of w.partials. The fixed-order
// fp64 sums over chunks of kChunkTiles tiles and over each view's chunks are
// k_reduce_chunks's, after the pass: the order depends only on tile indices,
// so a view gives the same bits alone or inside a batch. Block-uniform; ends
// past a barrier.
__device__ void tile_partial(float (&v)[7], uint32_t tile, int tid, int lane, int wid, const Work& w,
                             float (&s_red)[kWarps][8]) {
#pragma unroll
  for (int k = 0; k < 7; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 7; ++k) s_red[wid][k] = v[k];
  }
  __syncthreads();
  if (tid < 7) {
    float t = s_red[0][tid];
#pragma unroll
    for (int k = 1; k < kWarps; ++k) t += s_red[k][tid];
    w.partials[(size_t)tile * kPartialStride + tid] = (double)t;
  }
}

// The fp64 reductions of the tangent pass's tile partials: block c sums chunk
// c (kChunkTiles tiles of one view; warp k component k, lanes taking tiles
// lane and lane + 32, then a fixed shuffle tree), and the block that finishes
// the last chunk of a view sums the view's chunks (lane-strided, then the same
// tree) into result.
__global__ void __launch_bounds__(7 * 32) k_reduce_chunks(const View* __restrict__ views, int n_views, Work w,
                                                          double* __restrict__ result) {
  __shared__ bool s_last;
  if (w.ctr->overflow) return;
  const uint32_t chunk = blockIdx.x;
  const int lane = threadIdx.x & 31, k = threadIdx.x >> 5;
  int vi = 0;
  {
    int lo = 0, hi = n_views - 1;  // last view whose first chunk is <= this one
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (views[mid].chunk_base <= chunk) lo = mid; else hi = mid - 1;
    }
    vi = lo;
  }
  const View& V = views[vi];
  const uint32_t nt = (uint32_t)V.tiles_x * (uint32_t)V.tiles_y;
  const uint32_t c0 = (chunk - V.chunk_base) * kChunkTiles;
  const uint32_t cn = min((uint32_t)kChunkTiles, nt - c0);
  {
    const double* src = w.partials + (size_t)(V.tile_base + c0) * kPartialStride + k;
    double x = (uint32_t)lane < cn ? __ldcg(src + (size_t)lane * kPartialStride) : 0.0;
    if ((uint32_t)lane + 32u < cn) x += __ldcg(src + (size_t)(lane + 32) * kPartialStride);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) {
      w.chunk_part[(size_t)chunk * kPartialStride + k] = x;
      __threadfence();
    }
  }
  __syncthreads();
  const uint32_t ncv = (nt + kChunkTiles - 1) / kChunkTiles;
  if (threadIdx.x == 0) s_last = atomicAdd(&w.view_ctr[vi], 1u) == ncv - 1u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double x = 0.0;
  for (uint32_t c = lane; c < ncv; c += 32)
    x += __ldcg(w.chunk_part + (size_t)(V.chunk_base + c) * kPartialStride + k);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  if (lane == 0) result[(size_t)vi * kPartialStride + k] = x;
}

// ---------------------------------------------------------------------------
// Compositing, one persistent CTA per tile at a time (8 warps = 8 blocks of
// 8 x 4 pixels). TAN = false: the forward render (colour, depth, alpha, T,
// last index and, with FEAT = 32, the feature map). TAN = true: the same
// forward values plus the pose gradient of the L1 loss in tangent (forward)
// mode: along each of the six pose directions k every pixel carries
// d(C, D, T)/d xi_k through the front-to-back recursion
//   w = alpha T,  dw = dalpha T + alpha dT,  C += w c  -> dC += dw c + w dc,
//   D += w z -> dD += dw z + w dz,  T' = T (1 - alpha) -> dT' = dT - dw,
// with dalpha = alpha dpower (0 where the 0.99 cap is active) and dpower from
// the pixel offset and the Gaussian's staged pose Jacobian. After the walk,
// dL/dxi = sum over pixels of g . (dC, dD) with g the per-pixel L1
// subgradient, reduced in fp32 per tile (tile_partial) and in fp64 across
// tiles (k_reduce_chunks, launched after the pass).
// ---------------------------------------------------------------------------
// KB: Gaussians staged per batch; MINB: resident CTAs per SM the register
// allocation must allow (the autotuner's compositor variants, all giving the
// same bits: the blending order and every reduction order are fixed by the
// tile lists, not by the batching or the grid)
template <int FEAT, bool TAN, int KB, int MINB>
__global__ void __launch_bounds__(kTileThreads, MINB) k_composite(SceneDev sc, const View* __restrict__ views,
                                                                  int n_views, Work w, double* __restrict__ result) {
  static_assert(!(TAN && FEAT), "tangent mode renders without features");
  static_assert(!TAN || KB * kJacStride * 4 <= kSmHist, "staged Jacobians must fit in the sort buffers");
  static_assert(!TAN || kSmStageT + KB * 48 + kTileThreads * 4 <= kSmTan,
                "tangent staging (records and the per-part hit masks) must fit in the histogram");
  static_assert(!TAN || (kTileThreads % KB == 0 && kWarps % (kTileThreads / KB) == 0),
                "tangent staging splits the warp blocks evenly over the threads of an entry");
  static_assert(TAN || 4 * KB * 16 <= kSortCap * 8, "staging must fit in the second sort buffer");
  constexpr int kB = KB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint2* bufA = reinterpret_cast<uint2*>(smem_raw + kSmBufA);
  uint2* bufB = reinterpret_cast<uint2*>(smem_raw + kSmBufB);
  uint32_t* hist = reinterpret_cast<uint32_t*>(smem_raw + kSmHist);
  float4* sa = reinterpret_cast<float4*>(smem_raw + (TAN ? kSmStageT : FEAT ? 0 : kSmStage));
  float4* sb = sa + kB;
  float4* scol = sb + kB;
  uint32_t* smask = reinterpret_cast<uint32_t*>(scol + kB);
  uint4* sf = reinterpret_cast<uint4*>(smem_raw + feat_off_sf<KB>());  // FEAT: KB x 4
  // FEAT: this warp's transposed weight slots (hi rows, then lo rows) and slot features
  unsigned short* wt = reinterpret_cast<unsigned short*>(smem_raw + feat_off_wt<KB>()) + (threadIdx.x >> 5) * kWtWarp;
  unsigned short* fb = reinterpret_cast<unsigned short*>(smem_raw + feat_off_fb<KB>()) +
                       (threadIdx.x >> 5) * (kSlots * kWtRow);
  if (FEAT) {  // empty slots multiply stale rows by zero weights: keep the rows finite
    for (int i = threadIdx.x & 31; i < kSlots * kWtRow; i += 32) fb[i] = 0;
  }
  float4* sj = reinterpret_cast<float4*>(smem_raw + kSmJac);  // TAN: KB x 12
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_tmp[kWarps];
  __shared__ float s_red[kWarps][8];
  (void)result;  // the tangent pass's fp64 sums are k_reduce_chunks's
  if (w.ctr->overflow) return;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  int lx, ly, bxw, byw;
  warp_block(tid, lx, ly, bxw, byw);
  const float pxc = (float)lx + 0.5f, pyc = (float)ly + 0.5f;
  const float4* rec_j4 = reinterpret_cast<const float4*>(w.rec_j);
  uint32_t n_blend = 0;  // tangent pass: blended (pixel, Gaussian) pairs of this thread
  uint32_t n_eval = 0;   // tangent pass: list entries its pixels examined before their stop
  for (;;) {
    // the tangent pass keeps its own queue: it can follow a feature render
    if (tid == 0) {
      unsigned int* q = w.queue ? w.queue : (TAN ? &w.ctr->tan_queue : &w.ctr->fwd_queue);
      s_tile = w.tile_begin + atomicAdd(q, 1u);
    }
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= min(w.n_tiles, w.tile_end)) {
      if (TAN) {
        const uint32_t nb = __reduce_add_sync(0xffffffffu, n_blend);
        const uint32_t ne = __reduce_add_sync(0xffffffffu, n_eval);
        if (lane == 0 && nb) atomicAdd(&w.ctr->blends, (unsigned long long)nb);
        if (lane == 0 && ne) atomicAdd(&w.ctr->evals, (unsigned long long)ne);
      }
      break;
    }
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
      if (TAN || FEAT) __syncthreads();  // the list is read back from global memory
      list = (TAN || FEAT) ? w.pairs + start : bufA;
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
    // FEAT: accumulator fragments of the warp's 32 pixels x 32 channels
    // (m-tile of 16 pixels, n-tile of 8 channels, the mma.sync C layout)
    float F[FEAT ? 2 : 1][FEAT ? 4 : 1][4];
#pragma unroll
    for (int a = 0; a < (FEAT ? 2 : 1); ++a)
#pragma unroll
      for (int b = 0; b < (FEAT ? 4 : 1); ++b) F[a][b][0] = F[a][b][1] = F[a][b][2] = F[a][b][3] = 0.f;
    int nslot = 0;  // FEAT: slots filled (warp-uniform)
    // FEAT: add the filled slots to the warp's accumulators (empty slots get
    // zero weights)
    auto flush_feats = [&]() {
      for (int sl = nslot; sl < kSlots; ++sl)
#pragma unroll
        for (int t = 0; t < kWtTerms; ++t) wt[(t * kSlots + sl) * kWtRow + lane] = 0;
      __syncwarp();
      // B: the slots' features, k = slot (lane % 16), 8 channels from (lane / 16) * 8
      const uint32_t bb = (uint32_t)__cvta_generic_to_shared(fb + (lane & (kSlots - 1)) * kWtRow) +
                          (uint32_t)(lane >> 4) * 16u;
      uint32_t b[8];
      ldsm_x4_trans(bb, b[0], b[1], b[2], b[3]);       // channels 0..15
      ldsm_x4_trans(bb + 32u, b[4], b[5], b[6], b[7]);  // channels 16..31
      // A: weights, matrix lane / 8 = (pixels +8 if odd, slots +8 if >= 2)
      const int kk = (lane & 7) + ((lane >> 4) << 3), pp = ((lane >> 3) & 1) << 3;
      const uint32_t wa = (uint32_t)__cvta_generic_to_shared(wt) + (uint32_t)(kk * kWtRow + pp) * 2u;
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
        for (int t = kWtTerms - 1; t >= 0; --t) {  // smallest term first
          uint32_t a0, a1, a2, a3;
          ldsm_x4_trans(wa + (uint32_t)(t * kSlots * kWtRow * 2 + mt * 32), a0, a1, a2, a3);
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) mma_16816(F[mt][nt], a0, a1, a2, a3, b[2 * nt], b[2 * nt + 1]);
        }
      }
      __syncwarp();
      nslot = 0;
    };
    // tangents, pairs over the pose directions (0,1), (2,3), (4,5)
    float2 dC0[3], dC1[3], dC2[3], dD[3], dT[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      dC0[k] = dC1[k] = dC2[k] = dD[k] = dT[k] = make_float2(0.f, 0.f);
    }
    uint32_t last = 0;
    uint32_t stop_pos = 0;  // 1 + list position of the entry that stopped the walk (0: none)
    bool done = !inside;
    for (int bs = 0; bs < n; bs += kB) {
      if (__syncthreads_count(done) == kTileThreads) break;
      const int bn = min(kB, n - bs);
      if (TAN) {
        // Pose Jacobians (bn x 12 float4) by cp.async, without registers:
        // consecutive threads copy consecutive 16-byte pieces of a record; the
        // list entries of all of a thread's pieces are loaded first.
        constexpr int kJ4 = kJacStride / 4;
        constexpr int kJPer = (kB * kJ4 + kTileThreads - 1) / kTileThreads;
        uint32_t jr[kJPer];
#pragma unroll
        for (int i = 0; i < kJPer; ++i) {
          const int q = tid + kTileThreads * i;
          jr[i] = q < bn * kJ4 ? list[bs + q / kJ4].y : 0u;
        }
#pragma unroll
        for (int i = 0; i < kJPer; ++i) {
          const int q = tid + kTileThreads * i;
          if (q < bn * kJ4) cp_async16(sj + q, rec_j4 + (size_t)jr[i] * kJ4 + (q % kJ4));
        }
        // records and hit masks: kParts threads per entry, each testing the
        // warp blocks of its part, so that every warp stages
        constexpr int kParts = kTileThreads / kB;
        constexpr int kPW = kWarps / kParts;  // warp blocks per part
        const int e = tid % kB, part = tid / kB;
        if (e < bn) {
          const uint32_t r = list[bs + e].y;
          const float4 cc = w.rec_c[r];
          const float4 a = tile_local(w.rec_a[r], cc.w, X0, Y0);
          const float4 bb = w.rec_b[r];
          if (part == 0) {
            sa[e] = a;
            sb[e] = bb;
            scol[e] = cc;
          }
          smask[part * kB + e] = warp_hit_mask(a, bb.x, floor_threshold(bb.y), part * kPW, part * kPW + kPW);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
      } else if (tid < bn) {
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
      auto blend = [&](int j, float p, float oe, float zj, float dx, float dy) {
        const float alpha = fminf(kAlphaCap, oe);
        const bool take = !done && !(p > 0.0f) && !(alpha < kAlphaFloor);
        const float Tn = __fmul_rn(T, __fsub_rn(1.0f, alpha));
        const bool stop = take && (Tn < kTCut);
        const bool acc = take && !stop;
        const float wgt = acc ? __fmul_rn(alpha, T) : 0.0f;
        const float4 c = scol[j];
        if (TAN) {
          // staged Jacobian: per direction pair k, (P, Q), (dA/2, dB),
          // (dC/2, dz) with P = A du + B dv, Q = B du + C dv; then the colour
          // rows. S_k = dx P + dy Q + dx^2 dA/2 + dx dy dB + dy^2 dC/2 is
          // -dpower/dxi_k.
          const float4* J4 = sj + j * (kJacStride / 4);
          // T dalpha = -alpha T S (0 where the 0.99 cap is active); -alpha T
          // is folded into the monomials of the pixel offset
          const float nat = (acc && oe < kAlphaCap) ? -alpha * T : 0.0f;
          const float qx = nat * dx, qy = nat * dy;
          const float qxx = qx * dx, qxy = qx * dy, qyy = qy * dy;
          const float2 X = make_float2(qx, qx), Y = make_float2(qy, qy);
          const float2 XX = make_float2(qxx, qxx), XY = make_float2(qxy, qxy), YY = make_float2(qyy, qyy);
          const float ae = acc ? alpha : 0.0f;
          const float2 AE = make_float2(ae, ae);
          const float2 CR = make_float2(c.x, c.x), CG = make_float2(c.y, c.y), CB = make_float2(c.z, c.z);
          const float2 ZZ = make_float2(zj, zj), WW = make_float2(wgt, wgt);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const float4 pq = J4[3 * k], ab = J4[3 * k + 1], cz = J4[3 * k + 2];
            float2 tda = __fmul2_rn(make_float2(pq.x, pq.y), X);  // T dalpha
            tda = __ffma2_rn(make_float2(pq.z, pq.w), Y, tda);
            tda = __ffma2_rn(make_float2(ab.x, ab.y), XX, tda);
            tda = __ffma2_rn(make_float2(ab.z, ab.w), XY, tda);
            tda = __ffma2_rn(make_float2(cz.x, cz.y), YY, tda);
            const float2 dw = __ffma2_rn(dT[k], AE, tda);
            dT[k] = __ffma2_rn(dw, make_float2(-1.0f, -1.0f), dT[k]);
            dC0[k] = __ffma2_rn(dw, CR, dC0[k]);
            dC1[k] = __ffma2_rn(dw, CG, dC1[k]);
            dC2[k] = __ffma2_rn(dw, CB, dC2[k]);
            // dz/drho_0 = dz/drho_1 = 0: the first pair has no w dz term
            dD[k] = __ffma2_rn(dw, ZZ, k == 0 ? dD[k] : __ffma2_rn(make_float2(cz.z, cz.w), WW, dD[k]));
          }
          // colour depends on the camera centre only: rho directions 0..2
          const float4 r0 = J4[9], r1 = J4[10], r2 = J4[11];
          dC0[0] = __ffma2_rn(make_float2(r0.x, r0.y), WW, dC0[0]);
          dC0[1].x = fmaf(r0.z, wgt, dC0[1].x);
          dC1[0] = __ffma2_rn(make_float2(r1.x, r1.y), WW, dC1[0]);
          dC1[1].x = fmaf(r1.z, wgt, dC1[1].x);
          dC2[0] = __ffma2_rn(make_float2(r2.x, r2.y), WW, dC2[0]);
          dC2[1].x = fmaf(r2.z, wgt, dC2[1].x);
        }
        C0 = fmaf(wgt, c.x, C0);
        C1 = fmaf(wgt, c.y, C1);
        C2 = fmaf(wgt, c.z, C2);
        D = fmaf(wgt, zj, D);
        if (FEAT && __any_sync(0xffffffffu, wgt != 0.0f)) {  // a slot for a hit some pixel blends
          const __nv_bfloat16 hi = __float2bfloat16_rn(wgt);
          const float r1 = __fsub_rn(wgt, __bfloat162float(hi));  // exact differences
          const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
          const __nv_bfloat16 lo = __float2bfloat16_rn(__fsub_rn(r1, __bfloat162float(mid)));
          wt[nslot * kWtRow + lane] = __bfloat16_as_ushort(hi);
          wt[(kSlots + nslot) * kWtRow + lane] = __bfloat16_as_ushort(mid);
          wt[(2 * kSlots + nslot) * kWtRow + lane] = __bfloat16_as_ushort(lo);
          if (lane < 4) reinterpret_cast<uint4*>(fb + nslot * kWtRow)[lane] = sf[j * 4 + lane];
          if (++nslot == kSlots) flush_feats();
        }
        if (TAN) n_blend += acc ? 1u : 0u;
        T = acc ? Tn : T;
        last = acc ? (uint32_t)(bs + j + 1) : last;
        if (TAN) stop_pos = stop ? (uint32_t)(bs + j + 1) : stop_pos;
        done = done || stop;
      };
      const uint32_t wbit = 1u << wid;
      // tangent mode: this warp's bits sit in the mask array of its part
      const uint32_t* wmask = TAN ? smask + (wid / (kWarps / (kTileThreads / kB))) * kB : smask;
      bool wdone = __all_sync(0xffffffffu, done);
      for (int c0 = 0; c0 < bn && !wdone; c0 += 32) {
        const int jj = c0 + lane;
        uint32_t m = __ballot_sync(0xffffffffu, jj < bn && (wmask[jj] & wbit));
        while (m) {  // two hits per step: their exponentials overlap, blending stays in order
          const int j1 = c0 + __ffs(m) - 1;
          m &= m - 1;
          if (TAN) {  // one hit per step: the tangent update needs the registers
            const float4 a1 = sa[j1], b1 = sb[j1];
            const float dx1 = __fsub_rn(a1.x, pxc), dy1 = __fsub_rn(a1.y, pyc);
            const float p1 = gs_power(a1.z, a1.w, b1.x, dx1, dy1);
            blend(j1, p1, __fmul_rn(b1.y, __expf(p1)), b1.z, dx1, dy1);
            continue;
          }
          const bool two = m != 0u;
          const int j2 = two ? c0 + __ffs(m) - 1 : j1;
          if (two) m &= m - 1;
          const float4 a1 = sa[j1], b1 = sb[j1], a2 = sa[j2], b2 = sb[j2];
          const float dx1 = __fsub_rn(a1.x, pxc), dy1 = __fsub_rn(a1.y, pyc);
          const float dx2 = __fsub_rn(a2.x, pxc), dy2 = __fsub_rn(a2.y, pyc);
          const float p1 = gs_power(a1.z, a1.w, b1.x, dx1, dy1);
          const float p2 = gs_power(a2.z, a2.w, b2.x, dx2, dy2);
          const float oe1 = __fmul_rn(b1.y, __expf(p1));
          const float oe2 = __fmul_rn(b2.y, __expf(p2));
          blend(j1, p1, oe1, b1.z, dx1, dy1);
          if (two) blend(j2, p2, oe2, b2.z, dx2, dy2);
        }
        wdone = __all_sync(0xffffffffu, done);
      }
    }
    if (FEAT && nslot) flush_feats();  // the tile's last, partial slot group
    const size_t HW = (size_t)V.width * V.height;
    const size_t p = (size_t)py * V.width + px;
    // the entries a pixel examines: its list up to the stop, or the whole list
    if (TAN && inside) n_eval += stop_pos ? stop_pos : (uint32_t)n;
    if (inside) {
      if (V.rgb) {
        V.rgb[p] = C0;
        V.rgb[HW + p] = C1;
        V.rgb[2 * HW + p] = C2;
      }
      if (V.depth) V.depth[p] = D;
      if (V.alpha) V.alpha[p] = 1.0f - T;
      if (V.final_T) V.final_T[p] = T;
      if (V.last_idx) V.last_idx[p] = last;
    }
    if (FEAT && V.feats) {  // fragment element (mt, nt, e): pixel 16 mt + lane / 4 (+ 8), channel 8 nt + 2 (lane % 4) (+ 1)
#pragma unroll
      for (int mt = 0; mt < (FEAT ? 2 : 1); ++mt)
#pragma unroll
        for (int e2 = 0; e2 < 2; ++e2) {
          const int q = mt * 16 + (lane >> 2) + e2 * 8;  // the pixel's lane in the warp block
          const int qx = tx * kTile + bxw + (q & 7), qy = ty * kTile + byw + (q >> 3);
          if (qx >= V.width || qy >= V.height) continue;
          const size_t qp = (size_t)qy * V.width + qx;
#pragma unroll
          for (int nt = 0; nt < (FEAT ? 4 : 1); ++nt) {
            const int ch = nt * 8 + (lane & 3) * 2;
            V.feats[(size_t)ch * HW + qp] = F[mt][nt][2 * e2];
            V.feats[(size_t)(ch + 1) * HW + qp] = F[mt][nt][2 * e2 + 1];
          }
        }
    }
    if (TAN) {
      // per-pixel L1 subgradient g (sign(0) = 0) and loss
      float v[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (inside) {
        const float wpx = V.pixel_weight ? V.pixel_weight[p] : 1.0f;
        const float r0 = C0 - V.target_rgb[p];
        const float r1 = C1 - V.target_rgb[HW + p];
        const float r2 = C2 - V.target_rgb[2 * HW + p];
        const float e = D - V.target_depth[p];
        const float s3 = wpx * V.inv_3p, sd = wpx * V.depth_weight * V.inv_p;
        const float g0 = s3 * (float)((r0 > 0.f) - (r0 < 0.f));
        const float g1 = s3 * (float)((r1 > 0.f) - (r1 < 0.f));
        const float g2 = s3 * (float)((r2 > 0.f) - (r2 < 0.f));
        const float gd = sd * (float)((e > 0.f) - (e < 0.f));
        v[0] = s3 * (fabsf(r0) + fabsf(r1) + fabsf(r2)) + sd * fabsf(e);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float2 x = __ffma2_rn(make_float2(g0, g0), dC0[k],
                                      __ffma2_rn(make_float2(g1, g1), dC1[k],
                                                 __ffma2_rn(make_float2(g2, g2), dC2[k],
                                                            __fmul2_rn(make_float2(gd, gd), dD[k]))));
          v[1 + 2 * k] = x.x;
          v[2 + 2 * k] = x.y;
        }
      }
      tile_partial(v, V.tile_base + lt, tid, lane, wid, w, s_red);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Algorithm 1 (render-gradient visibility check): reverse walk of every pixel
// for L = sum of the rendered colours (dL/dC = 1 per channel), from the final
// transmittance and last blended index of a forward render. Walking back,
// with s the channel sum of the normalised colour behind the current
// Gaussian, dL/dalpha_j = T_j (r_j + g_j + b_j - s) and dL/dc_j = alpha_j T_j
// per channel. Per blended pair the record accumulates
//   (e dx, e dy, e dx^2, e dx dy, e dy^2, alpha T),  e = dL/dpower,
// (dx, dy) = centre - pixel: the pose Jacobian's rows contract these with
// (P, Q, dA/2, dB, dC/2) to dL/dxi (see the tangent pass). The six values are
// summed over the warp by a reduce-scatter (8 shuffles) and added to the
// record's accumulator by six lanes, or, when few lanes blended, added by
// those lanes; a Gaussian nobody blended keeps an exact zero. The order of
// the atomic additions varies, so the sums are not bit-reproducible; the test
// the algorithm makes (gradient != 0) is.
// ---------------------------------------------------------------------------
constexpr int kBatchV = kTileThreads;  // entries staged per batch of the reverse pass
constexpr int kVisDirect = 12;         // at most this many blending lanes add without the warp reduction

__global__ void __launch_bounds__(kTileThreads, 7) k_vis_backward(const View* __restrict__ views, int n_views, Work w,
                                                               float* __restrict__ acc) {
  // staged per entry: centre and conic A, B; (C, opacity); channel sum of the colour
  __shared__ float4 sa[kBatchV];
  __shared__ float2 sb[kBatchV];
  __shared__ float sg[kBatchV];
  __shared__ uint32_t smask[kBatchV], srec[kBatchV];
  __shared__ uint32_t s_tile, s_max[kWarps];
  if (w.ctr->overflow) return;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  int lx, ly, bxw, byw;
  warp_block(tid, lx, ly, bxw, byw);
  const float pxc = (float)lx + 0.5f, pyc = (float)ly + 0.5f;
  const uint32_t wbit = 1u << wid;
  uint32_t n_eval = 0, n_take = 0;  // (pixel, Gaussian) pairs evaluated / blended by this thread
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(&w.ctr->tan_queue, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= w.n_tiles) {
      const uint32_t ne = __reduce_add_sync(0xffffffffu, n_eval), nt = __reduce_add_sync(0xffffffffu, n_take);
      if (lane == 0 && ne) atomicAdd(&w.ctr->evals, (unsigned long long)ne);
      if (lane == 0 && nt) atomicAdd(&w.ctr->blends, (unsigned long long)nt);
      break;
    }
    const int vi = find_view(views, n_views, tile);
    const View& V = views[vi];
    const uint32_t lt = tile - V.tile_base;
    const int tx = (int)(lt % (uint32_t)V.tiles_x), ty = (int)(lt / (uint32_t)V.tiles_x);
    const uint32_t start = w.tile_offset[tile];
    const int px = tx * kTile + lx, py = ty * kTile + ly;
    const bool inside = px < V.width && py < V.height;
    const float X0 = (float)(tx * kTile), Y0 = (float)(ty * kTile);
    const size_t p = (size_t)py * V.width + px;
    uint32_t last = 0;
    float T = 1.0f;
    if (inside) {
      last = V.last_idx[p];
      T = V.final_T[p];
    }
    const uint32_t wm = __reduce_max_sync(0xffffffffu, last);
    if (lane == 0) s_max[wid] = wm;
    __syncthreads();
    uint32_t max_last = 0;
#pragma unroll
    for (int k = 0; k < kWarps; ++k) max_last = max(max_last, s_max[k]);
    float sdot = 0.0f;  // sum over channels of the normalised colour behind
    for (int bend = (int)max_last; bend > 0; bend -= kBatchV) {
      const int bstart = max(0, bend - kBatchV);
      const int bn = bend - bstart;
      __syncthreads();
      if (tid < bn) {
        const uint32_t r = w.pairs[start + bstart + tid].y;
        const float4 cc = w.rec_c[r];
        const float4 a = tile_local(w.rec_a[r], cc.w, X0, Y0);
        const float4 bb = w.rec_b[r];
        sa[tid] = a;
        sb[tid] = make_float2(bb.x, bb.y);
        sg[tid] = cc.x + cc.y + cc.z;
        srec[tid] = r;
        smask[tid] = warp_hit_mask(a, bb.x, floor_threshold(bb.y));
      }
      __syncthreads();
      if ((uint32_t)bstart >= wm) continue;
      for (int c0 = ((bn - 1) >> 5) << 5; c0 >= 0; c0 -= 32) {
        const int jj = c0 + lane;
        uint32_t m = __ballot_sync(0xffffffffu, jj < bn && (uint32_t)(bstart + jj) < wm && (smask[jj] & wbit));
        {  // the chunk's hits this pixel evaluates: those before its last blended entry
          const int below = inside ? (int)last - (bstart + c0) : 0;
          n_eval += (uint32_t)__popc(below >= 32 ? m : below <= 0 ? 0u : m & ((1u << below) - 1u));
        }
        while (m) {  // back to front
          const int bit = 31 - __clz(m);
          m &= ~(1u << bit);
          const int j = c0 + bit;
          const float4 a = sa[j];
          const float2 b = sb[j];
          const float dx = __fsub_rn(a.x, pxc), dy = __fsub_rn(a.y, pyc);
          const float pw = gs_power(a.z, a.w, b.x, dx, dy);
          const float oe = __fmul_rn(b.y, __expf(pw));
          const float alpha = fminf(kAlphaCap, oe);
          const bool before = inside && (uint32_t)(bstart + j) < last;
          const bool take = before && !(pw > 0.0f) && !(alpha < kAlphaFloor);
          n_take += take ? 1u : 0u;
          const unsigned tb = __ballot_sync(0xffffffffu, take);
          if (!tb) continue;  // nobody in the warp blended it
          const float Tj = take ? __fdividef(T, 1.0f - alpha) : T;
          const float wgt = take ? alpha * Tj : 0.0f;
          const float d = sg[j] - sdot;  // dL/dalpha = Tj d
          sdot = fmaf(take ? alpha : 0.0f, d, sdot);
          T = Tj;
          const float e = (take && oe < kAlphaCap) ? (Tj * d) * alpha : 0.0f;  // dalpha/dpower = alpha
          const float ex = e * dx, ey = e * dy;
          const float g[6] = {ex, ey, ex * dx, ex * dy, ey * dy, wgt};
          if (__popc(tb) <= kVisDirect) {  // few pixels: their own additions beat the reduction
            if (take) {
              float* ap = acc + (size_t)srec[j] * kVisAcc;
#pragma unroll
              for (int k = 0; k < 6; ++k) atomicAdd(ap + k, g[k]);
            }
            continue;
          }
          // reduce the six sums over the warp's pixels (lane bits b4, b3, b2 =
          // lane & 16, 8, 4): halve the set over b4 (values 3 b4 + 0..2), then
          // over b3 for the first two with the third summed, then over b2
          // between those two, and sum over bits 1, 0. Lane l ends with the
          // total of value 3 b4 + (b2 ? 2 : b3); for b2 both b3 halves hold it.
          const bool u16 = (lane & 16) != 0, u8 = (lane & 8) != 0, u4 = (lane & 4) != 0;
          float h[3];
#pragma unroll
          for (int i = 0; i < 3; ++i)
            h[i] = (u16 ? g[i + 3] : g[i]) + __shfl_xor_sync(0xffffffffu, u16 ? g[i] : g[i + 3], 16);
          h[0] = (u8 ? h[1] : h[0]) + __shfl_xor_sync(0xffffffffu, u8 ? h[0] : h[1], 8);
          h[2] += __shfl_xor_sync(0xffffffffu, h[2], 8);
          float tot = (u4 ? h[2] : h[0]) + __shfl_xor_sync(0xffffffffu, u4 ? h[0] : h[2], 4);
          tot += __shfl_xor_sync(0xffffffffu, tot, 2);
          tot += __shfl_xor_sync(0xffffffffu, tot, 1);
          const int vk = (u16 ? 3 : 0) + (u4 ? 2 : (u8 ? 1 : 0));
          if ((lane & 3) == 0 && !(u4 && u8) && tot != 0.0f) atomicAdd(acc + (size_t)srec[j] * kVisAcc + vk, tot);
        }
      }
    }
    __syncthreads();
  }
}

// The compositor variants of each mode; index 0 is the default.
using CompFn = void (*)(SceneDev, const View*, int, Work, double*);
struct Variant {
  CompFn fn;
  int smem, batch, min_blocks;
};
template <int FEAT, bool TAN, int KB, int MINB>
Variant variant() {
  return {k_composite<FEAT, TAN, KB, MINB>, comp_smem<FEAT, TAN, KB>(), KB, MINB};
}
const Variant* variant_table(int mode) {
  static const Variant fwd[kCompVariants] = {variant<0, false, 256, 5>(), variant<0, false, 128, 5>(),
                                             variant<0, false, 256, 4>(), variant<0, false, 64, 5>()};
  static const Variant feat[kCompVariants] = {variant<32, false, 256, 3>(), variant<32, false, 128, 3>(),
                                              variant<32, false, 128, 4>(), variant<32, false, 64, 4>()};
  static const Variant tan[kCompVariants] = {variant<0, true, 128, 4>(), variant<0, true, 64, 4>(),
                                             variant<0, true, 128, 3>(), variant<0, true, 64, 3>()};
  return mode == kModeTan ? tan : mode == kModeFwdFeat ? feat : fwd;
}

// resident CTAs per SM of a variant (its shared memory and registers), once per process
int variant_occupancy(int mode, int v) {
  static int occ[kModeCount][kCompVariants] = {};
  if (occ[mode][v] == 0) {
    const Variant& V = variant_table(mode)[v];
    cudaFuncSetAttribute(V.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, V.smem);
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, V.fn, kTileThreads, V.smem) != cudaSuccess || b < 1) b = 1;
    occ[mode][v] = b;
  }
  return occ[mode][v];
}

int clamp_variant(int v) { return v >= 0 && v < kCompVariants ? v : 0; }

// persistent grid: per_sm CTAs per SM (0 or above the occupancy: the occupancy), at most one per tile
int comp_grid(int mode, int v, int per_sm, int sm_count, uint32_t n_units) {
  const int occ = variant_occupancy(mode, v);
  const int p = per_sm > 0 && per_sm < occ ? per_sm : occ;
  const uint32_t g = (uint32_t)(p * sm_count);
  return (int)(g < n_units ? g : n_units);
}

}  // namespace

CompVariantInfo composite_variant_info(int mode, int v) {
  mode = mode >= 0 && mode < kModeCount ? mode : 0;
  v = clamp_variant(v);
  const Variant& V = variant_table(mode)[v];
  return {V.batch, V.min_blocks, variant_occupancy(mode, v)};
}

cudaError_t launch_composite(const SceneDev& sc, const View* views, int n_views, const Work& w, bool feats,
                             const LaunchCfg& cfg, int sm_count, cudaStream_t st) {
  if (w.n_tiles == 0) return cudaSuccess;
  const int mode = (sc.feat_dim && feats) ? kModeFwdFeat : kModeFwd;
  const int v = clamp_variant(cfg.variant[mode]);
  const Variant& V = variant_table(mode)[v];
  const int g = comp_grid(mode, v, cfg.per_sm[mode], sm_count, w.n_tiles);
  V.fn<<<g, kTileThreads, V.smem, st>>>(sc, views, n_views, w, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_vis_backward(const View* views, int n_views, const Work& w, float* acc, int sm_count,
                                cudaStream_t st) {
  if (w.n_tiles == 0) return cudaSuccess;
  static int per_sm = 0;  // resident blocks per SM (persistent grid)
  if (per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_vis_backward, kTileThreads, 0) != cudaSuccess || b < 1)
      b = 4;
    per_sm = b;
  }
  const int grid = sm_count * per_sm;
  const int g = (uint32_t)grid < w.n_tiles ? grid : (int)w.n_tiles;
  k_vis_backward<<<g, kTileThreads, 0, st>>>(views, n_views, w, acc);
  return cudaGetLastError();
}

cudaError_t launch_composite_tangent(const SceneDev& sc, const View* views, int n_views, const Work& w,
                                     double* result, const LaunchCfg& cfg, int sm_count, cudaStream_t st) {
  if (w.n_tiles == 0) return cudaSuccess;
  const int v = clamp_variant(cfg.variant[kModeTan]);
  const Variant& V = variant_table(kModeTan)[v];
  const int g = comp_grid(kModeTan, v, cfg.per_sm[kModeTan], sm_count, w.n_tiles);
  V.fn<<<g, kTileThreads, V.smem, st>>>(sc, views, n_views, w, result);
  return cudaGetLastError();
}

cudaError_t launch_reduce_tangent(const View* views, int n_views, const Work& w, double* result, cudaStream_t st) {
  if (w.n_tiles == 0 || w.n_chunks == 0) return cudaSuccess;
  k_reduce_chunks<<<w.n_chunks, 7 * 32, 0, st>>>(views, n_views, w, result);
  return cudaGetLastError();
}

cudaError_t launch_composite_tangent_range(const SceneDev& sc, const View* views, int n_views, const Work& w,
                                           double* result, const LaunchCfg& cfg, int sm_count, cudaStream_t st,
                                           uint32_t tile_begin, uint32_t tile_end, unsigned int* queue) {
  if (tile_end > w.n_tiles) tile_end = w.n_tiles;
  if (tile_begin >= tile_end) return cudaSuccess;
  Work wb = w;
  wb.tile_begin = tile_begin;
  wb.tile_end = tile_end;
  wb.queue = queue;
  const int v = clamp_variant(cfg.variant[kModeTan]);
  const Variant& V = variant_table(kModeTan)[v];
  const int g = comp_grid(kModeTan, v, cfg.per_sm[kModeTan], sm_count, tile_end - tile_begin);
  V.fn<<<g, kTileThreads, V.smem, st>>>(sc, views, n_views, wb, result);
  return cudaGetLastError();
}

}  // namespace gsr
