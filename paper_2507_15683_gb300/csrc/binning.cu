// Tile binning, first level: per-tile pair counts (accumulated by the
// projection) -> exclusive scan -> scatter of (depth bits, record) pairs into
// each tile's segment. This is the most-significant "digit" of the 64-bit
// (tile, depth) key done as one counting pass; the depth order inside each
// tile is finished by the compositor's shared-memory radix sort.
#include <cuda_runtime.h>

#include "gsr_internal.h"

namespace gsr {
namespace {

constexpr int kScanThreads = 1024;

// Exclusive scan of tile_count[0..n) into tile_offset[0..n] and tile_cursor,
// by one CTA: each thread owns a contiguous chunk. Also publishes the total
// and flags an overflow of the pair capacity.
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(Work w) {
  __shared__ unsigned long long warp_tot[kScanThreads / 32];
  const uint32_t n = w.n_tiles;
  const uint32_t per = (n + kScanThreads - 1) / kScanThreads;
  const uint32_t b = threadIdx.x * per;
  const uint32_t e = b + per < n ? b + per : n;
  unsigned long long s = 0;
  for (uint32_t k = b; k < e; ++k) s += w.tile_count[k];
  // block exclusive scan of s
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    unsigned long long x = warp_tot[lane];
    unsigned long long y = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += t;
    }
    warp_tot[lane] = y - x;  // exclusive warp offsets
  }
  __syncthreads();
  unsigned long long run = warp_tot[wid] + incl - s;
  for (uint32_t k = b; k < e; ++k) {
    w.tile_offset[k] = (uint32_t)run;
    w.tile_cursor[k] = (uint32_t)run;
    run += w.tile_count[k];
  }
  // counters of the backward's chunked reduction start at zero every call
  for (uint32_t k = threadIdx.x; k < w.n_chunks; k += kScanThreads) w.chunk_ctr[k] = 0u;
  for (uint32_t k = threadIdx.x; k < w.n_views && w.n_chunks; k += kScanThreads) w.view_ctr[k] = 0u;
  if (threadIdx.x == kScanThreads - 1) {
    const unsigned long long total = run;
    w.tile_offset[n] = (uint32_t)total;
    w.ctr->pair_total = total > 0xffffffffull ? 0xffffffffu : (uint32_t)total;
    if (total > 0xffffffffull) atomicOr(&w.ctr->overflow, 4u);
    if (total > (unsigned long long)w.pair_cap) atomicOr(&w.ctr->overflow, 2u);
  }
}

// Scatter every record's pairs into the segments of the tiles it covers.
// Warp-cooperative: a warp takes 32 record slots, flattens their (record,
// tile) pairs and spreads them over its lanes, so a Gaussian that covers
// hundreds of tiles does not serialise one thread; each lane issues its
// atomics in groups of kScatterUnroll before using any returned slot. Slot
// order inside a segment is arbitrary; the compositor sorts it.
constexpr int kScatterUnroll = 4;

__global__ void __launch_bounds__(256) k_scatter(const View* __restrict__ views, Work w) {
  __shared__ uint32_t s_incl[8][32];
  __shared__ uint4 s_m[8][32];
  if (w.ctr->overflow) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t nw = gridDim.x * 8;
  for (uint32_t base = (blockIdx.x * 8 + wid) * 32; base < w.rec_cap; base += nw * 32) {  // warp-uniform
    const uint32_t r = base + lane;
    uint32_t cnt = 0;
    uint4 m = make_uint4(0u, 0u, 0u, 0u);
    if (r < w.rec_cap) {
      const uint32_t reg = r / w.rec_seg, loc = r - reg * w.rec_seg;
      if (loc < min(w.ctr->rec_region[reg], w.rec_seg)) {
        m = w.rec_m[r];
        cnt = ((m.x >> 16) - (m.x & 0xffffu) + 1u) * ((m.y >> 16) - (m.y & 0xffffu) + 1u);
      }
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0u) continue;
    s_incl[wid][lane] = incl;
    s_m[wid][lane] = m;
    __syncwarp();
    for (uint32_t k0 = 0; k0 < total; k0 += 32u * kScatterUnroll) {
      uint32_t pos[kScatterUnroll];
      uint2 val[kScatterUnroll];
#pragma unroll
      for (int u = 0; u < kScatterUnroll; ++u) {
        const uint32_t k = k0 + (uint32_t)(u * 32 + lane);
        pos[u] = 0xffffffffu;
        if (k < total) {
          int o = 0;  // first lane whose inclusive count exceeds k
#pragma unroll
          for (int step = 16; step > 0; step >>= 1)
            if (s_incl[wid][o + step - 1] <= k) o += step;
          const uint32_t local = k - (o ? s_incl[wid][o - 1] : 0u);
          const uint4 mm = s_m[wid][o];
          const uint32_t x0 = mm.x & 0xffffu, x1 = mm.x >> 16, y0 = mm.y & 0xffffu;
          const uint32_t wdt = x1 - x0 + 1u;
          const uint32_t ty = y0 + local / wdt, tx = x0 + local % wdt;
          const View& V = views[mm.z];
          pos[u] = atomicAdd(&w.tile_cursor[V.tile_base + ty * (uint32_t)V.tiles_x + tx], 1u);
          val[u] = make_uint2(mm.w, base + (uint32_t)o);
        }
      }
#pragma unroll
      for (int u = 0; u < kScatterUnroll; ++u)
        if (pos[u] != 0xffffffffu) w.pairs[pos[u]] = val[u];
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_scan_tiles(const Work& w, cudaStream_t st) {
  k_scan_tiles<<<1, kScanThreads, 0, st>>>(w);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const View* views, const Work& w, int grid, cudaStream_t st) {
  k_scatter<<<grid, 256, 0, st>>>(views, w);
  return cudaGetLastError();
}

}  // namespace gsr
