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
  if (threadIdx.x == kScanThreads - 1) {
    const unsigned long long total = run;
    w.tile_offset[n] = (uint32_t)total;
    w.ctr->pair_total = total > 0xffffffffull ? 0xffffffffu : (uint32_t)total;
    if (total > 0xffffffffull) atomicOr(&w.ctr->overflow, 4u);
    if (total > (unsigned long long)w.pair_cap) atomicOr(&w.ctr->overflow, 2u);
  }
}

// Scatter every record's pairs into the segments of the tiles it covers.
// Slot order inside a segment is arbitrary; the compositor sorts it.
__global__ void __launch_bounds__(256) k_scatter(const View* __restrict__ views, Work w) {
  if (w.ctr->overflow) return;
  const uint32_t n_rec = w.ctr->rec_count < w.rec_cap ? w.ctr->rec_count : w.rec_cap;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n_rec; r += gridDim.x * blockDim.x) {
    const uint4 m = w.rec_m[r];
    const int x0 = m.x & 0xffff, x1 = m.x >> 16, y0 = m.y & 0xffff, y1 = m.y >> 16;
    const View& V = views[m.z];
    const uint32_t tb = V.tile_base;
    const int tx_n = V.tiles_x;
    for (int ty = y0; ty <= y1; ++ty)
      for (int tx = x0; tx <= x1; ++tx) {
        const uint32_t pos = atomicAdd(&w.tile_cursor[tb + ty * tx_n + tx], 1u);
        w.pairs[pos] = make_uint2(m.w, r);
      }
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
