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
constexpr int kScanPer = 8;                             // counts per thread and chunk
constexpr int kScanChunk = kScanThreads * kScanPer;     // counts per chunk (32 KB of shared memory)
static_assert(kScanPer == 8, "a thread reads and writes its counts as two 16-byte vectors");

// Exclusive scan of tile_count[0..n) into tile_offset[0..n] and tile_cursor,
// by one CTA, in chunks of kScanChunk counts with a 64-bit carry: coalesced
// loads into shared memory, each thread then sums kScanPer consecutive counts,
// a block scan of those sums, and coalesced stores of the offsets. Also
// publishes the total and flags an overflow of the pair capacity.
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(Work w) {
  __shared__ __align__(16) uint32_t sv[kScanChunk];
  __shared__ unsigned long long warp_tot[kScanThreads / 32];
  __shared__ unsigned long long s_carry;
  const uint32_t n = w.n_tiles;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_carry = 0ull;
  for (uint32_t base = 0; base < n; base += kScanChunk) {  // block-uniform
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
      const uint32_t k = base + (uint32_t)(i * kScanThreads + tid);
      sv[i * kScanThreads + tid] = k < n ? w.tile_count[k] : 0u;
    }
    __syncthreads();
    // this thread's kScanPer consecutive counts, as two 16-byte reads
    uint32_t c[kScanPer];
    {
      const uint4* v4 = reinterpret_cast<const uint4*>(sv) + tid * (kScanPer / 4);
      const uint4 x = v4[0], y = v4[1];
      c[0] = x.x; c[1] = x.y; c[2] = x.z; c[3] = x.w;
      c[4] = y.x; c[5] = y.y; c[6] = y.z; c[7] = y.w;
    }
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) s += c[i];
    // block exclusive scan of s
    unsigned long long incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const unsigned long long x = warp_tot[lane];
      unsigned long long y = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += t;
      }
      warp_tot[lane] = y - x;  // exclusive warp offsets
    }
    __syncthreads();
    const unsigned long long carry = s_carry;
    unsigned long long run = carry + warp_tot[wid] + incl - s;
    uint32_t o8[kScanPer];
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
      o8[i] = (uint32_t)run;
      run += c[i];
    }
    {
      uint4* v4 = reinterpret_cast<uint4*>(sv) + tid * (kScanPer / 4);
      v4[0] = make_uint4(o8[0], o8[1], o8[2], o8[3]);
      v4[1] = make_uint4(o8[4], o8[5], o8[6], o8[7]);
    }
    __syncthreads();  // every thread has read s_carry and written its offsets
    if (tid == kScanThreads - 1) s_carry = run;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
      const uint32_t k = base + (uint32_t)(i * kScanThreads + tid);
      if (k < n) {
        const uint32_t o = sv[i * kScanThreads + tid];
        w.tile_offset[k] = o;
        w.tile_cursor[k] = o;
      }
    }
    __syncthreads();  // sv and s_carry are reused by the next chunk
  }
  // the view counters of the tangent pass's chunked reduction start at zero every call
  for (uint32_t k = tid; k < w.n_views && w.n_chunks; k += kScanThreads) w.view_ctr[k] = 0u;
  if (tid == 0) {
    const unsigned long long total = s_carry;
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
constexpr int kScatterUnroll = 8;

__global__ void __launch_bounds__(256) k_scatter(const View* __restrict__ views, Work w) {
  __shared__ uint32_t s_incl[8][32];
  __shared__ uint4 s_m[8][32];
  if (w.ctr->overflow) return;
  // every slot a tile cursor hands out lies below the scanned total when the
  // projection's tile counts and the records' rectangles agree; a slot past it
  // is a consistency failure: reported (Counters.error), never written
  const uint32_t pair_total = w.ctr->pair_total;
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
      for (int u = 0; u < kScatterUnroll; ++u) {
        if (pos[u] == 0xffffffffu) continue;
        if (pos[u] < pair_total) w.pairs[pos[u]] = val[u];
        else atomicOr(&w.ctr->error, 1u);
      }
    }
    __syncwarp();
  }
}

// Depth order of the short tile lists, one warp per tile: a bitonic network
// over E elements per lane (element e = E lane + i sits in register i), with
// compare-exchanges inside a lane for strides below E and across lanes by
// shuffles above, on distinct integer keys with branch-free min/max. When the
// tile's depth bits span less than 2^24 the key is the 32-bit
// (depth - smallest depth) << 8 | position, and the records wait in shared
// memory; otherwise the 64-bit (depth << 32 | record). Runs of equal depth
// are then put in Gaussian-index order (the tie-break of the key), which
// happens rarely. Lists longer than kWarpSortMax are left to the compositor's
// block sort.
__device__ __forceinline__ uint64_t kmin(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("min.u64 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t kmax(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("max.u64 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint32_t kmin(uint32_t a, uint32_t b) { return min(a, b); }
__device__ __forceinline__ uint32_t kmax(uint32_t a, uint32_t b) { return max(a, b); }

template <int E, typename K>
__device__ __forceinline__ void bitonic(K (&x)[E], int lane) {
#pragma unroll
  for (int size = 2; size <= 32 * E; size <<= 1) {
#pragma unroll
    for (int j = size >> 1; j > 0; j >>= 1) {
      if (j >= E) {  // partner: lane ^ (j / E), same register
        const int lj = j / E;
        // ascending blocks: the lower element keeps the minimum
        const bool keep_min = ((lane & lj) == 0) == (((lane * E) & size) == 0);
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const K o = __shfl_xor_sync(0xffffffffu, x[i], lj);
          const K mn = kmin(x[i], o), mx = kmax(x[i], o);
          x[i] = keep_min ? mn : mx;
        }
      } else {
#pragma unroll
        for (int i = 0; i < E; ++i) {
          if (i & j) continue;
          const int q = i | j;
          const bool up = ((lane * E + i) & size) == 0;
          const K mn = kmin(x[i], x[q]), mx = kmax(x[i], x[q]);
          x[i] = up ? mn : mx;
          x[q] = up ? mx : mn;
        }
      }
    }
  }
}

template <int E>
__device__ void warp_sort_list(uint2* __restrict__ list, int n, const float4* __restrict__ rec_b, int lane,
                               uint32_t* __restrict__ srec) {
  uint32_t k[E], v[E];
  uint32_t lo = 0xffffffffu, hi = 0u;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int e = lane * E + i;
    const uint2 p = e < n ? list[e] : make_uint2(0xffffffffu, 0xffffffffu);  // pads sort last
    k[i] = p.x;
    v[i] = p.y;
    if (e < n) {
      lo = min(lo, p.x);
      hi = max(hi, p.x);
      srec[e] = p.y;
    }
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  if (hi - lo < (1u << 24)) {  // warp-uniform
    uint32_t x[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int e = lane * E + i;
      x[i] = e < n ? ((k[i] - lo) << 8) | (uint32_t)e : 0xffffffffu;
    }
    bitonic<E>(x, lane);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int e = lane * E + i;
      k[i] = e < n ? (x[i] >> 8) + lo : 0xffffffffu;
      v[i] = e < n ? srec[x[i] & 255u] : 0xffffffffu;
    }
  } else {
    uint64_t x[E];
#pragma unroll
    for (int i = 0; i < E; ++i) x[i] = ((uint64_t)k[i] << 32) | v[i];
    bitonic<E>(x, lane);
#pragma unroll
    for (int i = 0; i < E; ++i) {
      k[i] = (uint32_t)(x[i] >> 32);
      v[i] = (uint32_t)x[i];
    }
  }
  bool tie = false;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int e = lane * E + i;
    if (e < n) list[e] = make_uint2(k[i], v[i]);
    if (i + 1 < E) tie = tie || (e + 1 < n && k[i] == k[i + 1]);
  }
  const uint32_t nxt = __shfl_down_sync(0xffffffffu, k[0], 1);
  const uint32_t prv = __shfl_up_sync(0xffffffffu, k[E - 1], 1);
  tie = tie || (lane < 31 && lane * E + E < n && k[E - 1] == nxt);
  if (!__any_sync(0xffffffffu, tie)) return;
  __syncwarp();
  // the owner of the first element of each run of equal depth puts the run in
  // Gaussian-index order (runs are short: equal binary32 depths are rare)
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int e = lane * E + i;
    const uint32_t before = i > 0 ? k[i > 0 ? i - 1 : 0] : prv;
    const uint32_t after = i + 1 < E ? k[i + 1 < E ? i + 1 : 0] : nxt;
    if (e + 1 < n && after == k[i] && (e == 0 || before != k[i])) {
      int end = e + 1;
      while (end < n && list[end].x == k[i]) ++end;
      for (int p = e + 1; p < end; ++p) {
        const uint2 x = list[p];
        const int gx = __float_as_int(rec_b[x.y].w);
        int q = p - 1;
        while (q >= e && __float_as_int(rec_b[list[q].y].w) > gx) {
          list[q + 1] = list[q];
          --q;
        }
        list[q + 1] = x;
      }
    }
  }
  __syncwarp();
}

__global__ void __launch_bounds__(256, 4) k_sort_tiles(Work w) {
  __shared__ uint32_t s_rec[8][kWarpSortMax];
  if (w.ctr->overflow) return;
  const int lane = threadIdx.x & 31;
  uint32_t* srec = s_rec[threadIdx.x >> 5];
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile < w.n_tiles; tile += nw) {
    const uint32_t start = w.tile_offset[tile];
    const int n = (int)(w.tile_offset[tile + 1] - start);
    if (n <= 1 || n > kWarpSortMax) continue;  // warp-uniform
    uint2* list = w.pairs + start;
    if (n <= 32) warp_sort_list<1>(list, n, w.rec_b, lane, srec);
    else if (n <= 64) warp_sort_list<2>(list, n, w.rec_b, lane, srec);
    else if (n <= 128) warp_sort_list<4>(list, n, w.rec_b, lane, srec);
    else warp_sort_list<8>(list, n, w.rec_b, lane, srec);
  }
}

}  // namespace

cudaError_t launch_sort_tiles(const Work& w, int grid, cudaStream_t st) {
  k_sort_tiles<<<grid, 256, 0, st>>>(w);
  return cudaGetLastError();
}

cudaError_t launch_scan_tiles(const Work& w, cudaStream_t st) {
  k_scan_tiles<<<1, kScanThreads, 0, st>>>(w);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const View* views, const Work& w, int grid, cudaStream_t st) {
  k_scatter<<<grid, 256, 0, st>>>(views, w);
  return cudaGetLastError();
}

}  // namespace gsr
